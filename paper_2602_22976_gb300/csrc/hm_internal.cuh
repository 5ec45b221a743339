// hm_internal.cuh - declarations shared by the translation units of libhm.
//
// Data layout in HBM (one handle; edges relabelled by decreasing priority,
// j = 0 is the highest-priority edge):
//   order  int32[m]     j -> input edge id
//   eoffj  int64[m+1]   edge CSR in j order (E_id of Sec. 4.1)
//   pinsj  int32[kappa] pins in j order (E_p)
//   voff   int64[n+1]   vertex CSR offsets (V_id)
//   vadj   int32[kappa] incident edges of every vertex, ascending j, i.e.
//                       decreasing priority (V_p)
//   alive  uint8[m]     1 = live edge (soft delete, Sec. 3.1)
//   P      uint32[m]    pins of e that have not chosen e yet; e wins when it
//                       reaches 0 (the P counter of Alg. 1 / Sec. 4.1, counted
//                       down). When no edge has more than 65535 pins the
//                       counters are 16 bits wide, two to a word (edge e in
//                       half e & 1 of word e >> 1): half the footprint, so
//                       more of them stay in L2
//   P0     uint32       the initial P words, copied by every match's init
//   vrec   int4[n]      per-vertex record {T[v] as an edge j, cursor of T[v]
//                       relative to the list start, list start, degree}
//                       (Alg. 3's T plus V_id); T[v] = kCurMatched once v is
//                       covered, kCurNone when v has no live edge. One 16-byte
//                       load serves both the liveness check and the advance.
//   firstj int32[n]     first entry of every vertex list (T[v] of round 1; round
//                       1 writes T and the cursor of every record from it)
//   graphs (every edge has two pins), fixed order: an edge is live exactly
//   when neither endpoint is matched, so liveness is read from the vertices
//   and there is no kill step:
//   vpair  int2[kappa]  {edge j, other endpoint} of every list entry, in vadj's
//                       order
//   firstnbr int32[n]   other endpoint of every vertex's first entry
//   vmatch uint8[n]     1 once the vertex is covered by M
//   vrec   int4[n]      {T[v], cursor (absolute position), list end, other
//                       endpoint of T[v]} instead of the layout above
//   list0/list1 int32[nregions*region] active vertex lists (ping-pong). The
//                       list is cut into one region per warp of the argmax
//                       grid; region g holds the active vertices of the
//                       vertex range [g*region, (g+1)*region), compacted in
//                       place, with its length in lcnt[parity][g]
//   lcnt   uint32[2][nregions] region lengths
//   wstage int32[nregions*region] per-region staging of a round's winners
//   win    int32[min(m,n)] winners of the current round, contiguous (the
//                       re-randomised rounds; the fixed order handles its
//                       winners inside the argmax kernel)
//   items  KillItem[n+1] kill ranges of the current round: one per newly
//                       matched vertex, {first list entry, offset of the
//                       range in the round's concatenation of all ranges},
//                       the offsets ascending with the item index
//   wround int32[m]     round in which an edge joined M (input numbering; only
//                       read for matched edges; batches only, which report
//                       each instance's round count)
//   inM    uint8[m]     result mask, input numbering
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>

#include "hm.h"

namespace hm {

constexpr int32_t kCurMatched = -1;  // vertex covered by the matching
constexpr int32_t kCurNone = -2;     // vertex has no live edge (or degree 0)
constexpr int kMinKillChunk = 64;    // smallest kill slice (entries per warp) a launch config may use

// Launch shape of the round kernels; the autotuner picks it per handle.
struct LaunchConfig {
    int kill_chunk = 64;   // least list entries a warp of the kill step takes
    int argmax_bpsm = 0;   // blocks per SM of k_argmax (0 = all that fit)
    int win_bpsm = 0;      // blocks per SM of k_win
    int kill_bpsm = 0;     // blocks per SM of k_kill
    bool operator==(const LaunchConfig &o) const {
        return kill_chunk == o.kill_chunk && argmax_bpsm == o.argmax_bpsm && win_bpsm == o.win_bpsm &&
               kill_bpsm == o.kill_bpsm;
    }
};
constexpr int kStatRounds = 4096;    // per-round counters kept for this many rounds

// Device-resident loop state (one per handle).
struct DevState {
    int32_t round;        // current round, 1-based
    int32_t parity;       // list index read by the current round
    uint32_t cnt[2];      // sizes of list0 / list1
    uint32_t nwin;        // winners of this round
    uint32_t kdone;       // blocks of the kill step that have finished
    int32_t status;       // HM_OK, HM_ETIMEOUT, HM_EINVAL (inconsistent input)
    int32_t rounds_done;  // rounds that started with a live edge
    int32_t finished;     // 1 once the loop has stopped
    int32_t fault;        // nonzero: an internal consistency check failed
    unsigned long long adv;        // counters of the current round
    unsigned long long kills;
    unsigned long long winpins;
    unsigned long long proposals;
    unsigned long long live;       // re-randomised rounds: live entries (pins of live edges) of the round
    unsigned long long sdeg;       // profiled rounds: degrees of the vertices kept
    unsigned long long kpack;      // kill ranges of the round: (entries << 32) | items
    unsigned long long ledges;     // edges live at the start of the round (profiled rounds; every
                                   // re-randomised round from the second on)
    unsigned long long lpins;      // their pins
};

// One kill range: list entries [begin, begin + length) where length is the
// next item's ebase (or the round's total) minus this ebase. kappa < 2^32,
// so both fit 32 bits.
struct KillItem {
    uint32_t begin;
    uint32_t ebase;
};

// Everything a round kernel touches; passed by value.
struct RoundArgs {
    DevState *st;
    const int64_t *voff;
    const int32_t *vadj;
    const int64_t *eoffj;
    const int32_t *pinsj;
    const int32_t *order;
    uint8_t *alive;
    uint32_t *P;
    const uint32_t *P0;    // initial P words (built once per handle)
    int4 *vrec;
    const int32_t *firstj;
    int pairs;             // graph, fixed order: liveness from vmatch, no kill step
    const int2 *vpair;     // pairs: {edge, other endpoint} per list entry
    const int32_t *firstnbr;
    uint8_t *vmatch;
    int32_t *list0;
    int32_t *list1;
    uint32_t *lcnt;
    int32_t *wstage;
    uint32_t nregions;     // == warps of the k_argmax grid
    uint32_t region;       // vertices per region (multiple of 32)
    int32_t *win;
    KillItem *items;
    uint8_t *inM;
    int32_t *wround;
    int64_t *stats;        // [kStatRounds][HM_STATS_COLS]
    int32_t kill_chunk;
    int64_t n;
    int64_t m;
    int64_t cap;           // round cap
    int p16;               // P holds 16-bit counters, two per word
    int graph;             // every edge has exactly two pins: edge j's pins are pinsj[2j], pinsj[2j + 1]
    uint64_t item_cap;     // capacity of items
    uint64_t win_cap;      // capacity of win
    cudaGraphConditionalHandle cond;
    int use_cond;
    // re-randomised rounds only (rrounds.cu)
    float noise_scale;          // amplitude * 2^-24
    uint64_t noise_s0;          // SplitMix64 start state of the priority stream
    const int2 *vadjE;          // round 1's lists as {input edge id, bits(round-1 priority)}
    const int32_t *jof;         // input id -> j
    uint32_t *P2;               // round 1's proposal counters (32-bit words)
    int t_input;                // T[v] holds input edge ids (re-randomised rounds), not j
    int w64;                    // proposal words are 64-bit (some edge has more than 65535 pins)
    const uint32_t *S32;        // |e| << 16 by input id: the proposal words' start value
    const unsigned long long *S64;  // |e| << 32 (w64)
    unsigned long long *W64;    // round 1's 64-bit proposal words (w64)
    const int32_t *vchunk;      // round 1: the vertex owning list entry c * kFlatW, per flat chunk c
    uint64_t kappa;             // list entries
    unsigned long long *rbest;  // largest key offered to each vertex in odd rounds
    unsigned long long *rbest2; // the same in even rounds (rounds >= 2)
    const int4 *erec;           // every edge in j order: {input id, bits(base priority), first pin, size}
    int4 *elist[2];             // rounds >= 2: the live edges of round r (records as erec) at index r & 1,
                                // in eregions regions of eregion records (erec: the same regions, full)
    uint32_t *ecnt;             // [2][eregions]: live records in each region of elist[0] / elist[1]
    uint32_t eregions, eregion;
    int erounds;                // re-randomised rounds: rounds >= 2 are edge rounds (round 1 ends accordingly)
    int profiled;               // the per-kernel replay: edge rounds record their live edges and pins
};

// Stats row of round r (rounds beyond kStatRounds are not recorded).
__device__ inline void write_stats_row(const RoundArgs &a, int r, int64_t active, uint32_t nw, uint32_t next,
                                unsigned long long adv, unsigned long long props, unsigned long long winpins,
                                unsigned long long kills, uint32_t items, unsigned long long live,
                                unsigned long long sdeg, unsigned long long ledges, unsigned long long lpins) {
    if (r >= 1 && r - 1 < kStatRounds) {
        int64_t *row = a.stats + (int64_t)(r - 1) * HM_STATS_COLS;
        row[HM_STAT_ACTIVE] = active;
        row[HM_STAT_ADVANCE] = (int64_t)adv;
        row[HM_STAT_PROPOSALS] = (int64_t)props;
        row[HM_STAT_WINNERS] = nw;
        row[HM_STAT_WINPINS] = (int64_t)winpins;
        row[HM_STAT_KILLS] = (int64_t)kills;
        row[HM_STAT_ITEMS] = items;
        row[HM_STAT_NEXT] = next;
        row[HM_STAT_LIVE] = (int64_t)live;
        row[HM_STAT_DEG] = (int64_t)sdeg;
        row[HM_STAT_LEDGES] = (int64_t)ledges;
        row[HM_STAT_LPINS] = (int64_t)lpins;
    }
}


struct Handle {
    int device = 0;
    int64_t n = 0, m = 0;
    uint64_t kappa = 0;
    bool weighted = true;
    bool p16 = false;           // every edge has at most 65535 pins: 16-bit P counters
    bool graph = false;         // every edge has exactly two pins (d = 2)
    uint64_t seed = 0;
    int sm_count = 0;
    // device buffers (owned)
    int64_t *voff = nullptr;
    int32_t *vadj = nullptr;
    int64_t *eoffj = nullptr;
    int32_t *pinsj = nullptr;
    int32_t *order = nullptr;
    float *weights = nullptr;   // input numbering, for the result weight
    uint8_t *alive = nullptr;
    uint32_t *P = nullptr;
    uint32_t *P0 = nullptr;     // initial P words
    int4 *vrec = nullptr;
    int32_t *firstj = nullptr;
    int2 *vpair = nullptr;      // graphs: {edge, other endpoint} per list entry
    int32_t *firstnbr = nullptr;
    uint8_t *vmatch = nullptr;  // graphs: matched flag per vertex
    int32_t *list0 = nullptr, *list1 = nullptr;
    uint32_t *lcnt = nullptr;
    int32_t *wstage = nullptr;
    uint32_t nregions = 0, region = 0;
    uint64_t list_cap = 0;     // entries in each of list0 / list1 / wstage
    uint32_t regions_cap = 0;  // entries per parity in lcnt
    unsigned argmax_grid = 0, win_grid = 0, kill_grid = 0;
    LaunchConfig cfg, graph_cfg;
    bool edge_rounds = false;   // keep each matched edge's round (batches: rounds per instance)
    int32_t *wround = nullptr;  // allocated when edge_rounds
    // re-randomised rounds (allocated on first use, rrounds.cu)
    float noise = 0.f;          // 0: fixed order; > 0: amplitude of the per-round noise
    float graph_noise = 0.f;    // amplitude exec_rand was built with
    float r1_noise = -1.f;      // amplitude vadjE's round-1 priorities were computed for
    bool last_random = false;   // the last match ran re-randomised rounds
    int4 *vrecR = nullptr;      // round 1: {T[v], 0, list start, list length}
    int2 *vadjE = nullptr;      // round 1's lists as {input edge id, bits(round-1 priority)}
    int4 *erec = nullptr;       // edge records in j order (built once)
    int4 *elist0 = nullptr, *elist1 = nullptr;  // live edge lists of the edge rounds
    uint32_t *ecnt = nullptr;                   // their region lengths
    uint32_t eregions = 0, eregion = 0;
    unsigned long long *rbest2 = nullptr;       // even rounds' largest keys per vertex
    uint8_t *rmatch = nullptr;  // hypergraphs: matched flag per vertex in the edge rounds
    int32_t *jof = nullptr;
    uint32_t *P2 = nullptr;
    uint32_t *S32 = nullptr;              // |e| << 16 by input id (every edge <= 65535 pins)
    unsigned long long *S64 = nullptr;    // |e| << 32 by input id (otherwise)
    unsigned long long *W64 = nullptr;    // 64-bit proposal words (otherwise)
    int32_t *vchunk = nullptr;            // round 1's flat scan: vertex of every chunk's first entry
    unsigned long long *rbest = nullptr;  // re-randomised rounds: largest key offered per vertex (odd rounds)
    unsigned rflat_grid = 0, rpropose_grid = 0, epush_grid = 0, ewin_grid = 0;
    cudaGraphExec_t exec_rand = nullptr;
    int64_t graph_cap_rand = -1;
    LaunchConfig graph_cfg_rand;
    int32_t *win = nullptr;
    KillItem *items = nullptr;
    uint8_t *inM = nullptr;
    int64_t *stats = nullptr;
    DevState *st = nullptr;
    // result scratch
    int32_t *res_idx = nullptr;
    float *res_w = nullptr;
    uint32_t *res_part = nullptr;
    unsigned long long *res_bucket = nullptr;  // [256] exponent buckets of the result weight
    uint64_t item_cap = 0, win_cap = 0;
    int64_t cap = 0;
    // graph
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    int64_t graph_cap = -1;
    cudaEvent_t done = nullptr;
    cudaStream_t last_stream = nullptr;
    bool matched_once = false;
    double create_ms[5] = {0, 0, 0, 0, 0};
    // pinned host staging
    DevState *h_st = nullptr;
};

// ---- error reporting (api.cu) ----
void set_error(const std::string &msg);
hm_status cuda_fail(cudaError_t e, const char *what);

// ---- primitives (prims.cu) ----
// Exclusive scan of n values; out may alias in. If total != nullptr the sum
// of all n values is written there. scratch must hold scan_scratch_elems(n).
size_t scan_scratch_elems(uint64_t n);
cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *total,
                               uint32_t *scratch, cudaStream_t s);
cudaError_t exclusive_scan_i64(const int64_t *in, int64_t *out, uint64_t n, int64_t *total,
                               int64_t *scratch, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs by key bits [0, end_bit).
// Inputs are not modified. tmp_k/tmp_v: n elements each. scratch: radix_scratch_elems(n).
size_t radix_scratch_elems(uint64_t n);
cudaError_t radix_sort_pairs(const uint32_t *keys_in, const uint32_t *vals_in,
                             uint32_t *keys_out, uint32_t *vals_out,
                             uint32_t *tmp_k, uint32_t *tmp_v, uint64_t n, int end_bit,
                             uint32_t *scratch, cudaStream_t s);
// Stable compaction of the indices i with flags[i] != 0 into idx_out (and
// w[i] into w_out when w != nullptr). part: compact_scratch_elems(n) + 1;
// the count is left in part[compact_scratch_elems(n)].
size_t compact_scratch_elems(uint64_t n);
// bucket[E] (256 words, cleared here) <- sum of the integer significands of
// w[i] over the flagged i with exponent field E (exact_sum.cuh rounds them).
cudaError_t weight_buckets(const uint8_t *flags, const float *w, uint64_t n, unsigned long long *bucket,
                           int sm_count, cudaStream_t s);
cudaError_t compact_flags(const uint8_t *flags, uint64_t n, const float *w, int32_t *idx_out,
                          float *w_out, uint32_t *part, cudaStream_t s);

// hm_solve_host below kSmallPins pins (every edge at most kSmallMaxSize
// pins): one thread block runs the whole matching (noalloc.cu).
constexpr uint64_t kSmallPins = uint64_t(1) << 17;
constexpr int64_t kSmallMaxSize = 256;
hm_status solve_small(int64_t n, int64_t m, uint64_t kappa, const int64_t *eoff, const int32_t *pins,
                      const float *weights, uint64_t seed, bool weighted, int32_t *edges_out,
                      int64_t *count_out, int32_t *rounds_out, double *weight_out, cudaStream_t s);

// ---- create (create.cu) ----
// inst_ebase (device, ninst entries): first edge of each instance when the
// input is a union of independent instances (local hash priorities), else null.
// Pins still crossing the host link, in chunks of consecutive pins: chunk c
// covers pins [begin[c], begin[c+1]) (begin[0] = 0, begin[chunks] = kappa,
// every other begin a multiple of kRelabelTile) and event ev[c] marks its
// arrival on the device.
constexpr int kRelabelTile = 2048;
struct PinChunks {
    int chunks;
    const uint64_t *begin;   // host, chunks + 1 entries
    const cudaEvent_t *ev;   // host, chunks entries
};
// feed (or null): the edge phase (validation of offsets and weights, the
// order, the edge offsets) runs first; then each chunk of pins is relabelled
// as soon as it has arrived, the pins are validated on the way, and their
// validity is checked before the vertex CSR is built from them.
hm_status create_structures(Handle *h, const int64_t *eoff, const int32_t *pins,
                            const float *weights, cudaStream_t s, const int64_t *inst_ebase = nullptr,
                            int32_t ninst = 0, const PinChunks *feed = nullptr);

// ---- rounds (rounds.cu) ----
RoundArgs round_args(const Handle *h);
hm_status alloc_round_state(Handle *h, cudaStream_t s);
hm_status launch_match_graph(Handle *h, cudaStream_t s);
hm_status apply_config(Handle *h, const LaunchConfig &c);
// Coordinate-descent search of the launch config; leaves the best applied.
hm_status autotune(Handle *h, cudaStream_t s, LaunchConfig *best, double *best_ms);
// Adds h's whole match (init node + conditional while loop) to graph g as a
// branch with no dependencies.
hm_status add_match_to_graph(Handle *h, cudaGraph_t g);
hm_status profile_match(Handle *h, cudaStream_t s, double *ms, int64_t *launches, double *round_ms,
                        int32_t max_rounds);
cudaError_t launch_vertex_state(const Handle *h, int32_t *out_dev, cudaStream_t s);
void free_handle_buffers(Handle *h);
// a2 - a4 of one round for a loop whose argmax step leaves the winners in
// a.win (the re-randomised rounds): win kernel, then the kill kernel, which
// also ends the round. The kill step reads the edge id of list entry p at
// a.vadj[p * kill_stride]. ev (or null): events 1-4 of a profiled round.
// Profiled rounds only: records ev[5] (the end of the argmax span), then
// counts the degrees of the vertices the argmax step kept (HM_STAT_DEG).
void launch_kept_degrees(const Handle *h, const RoundArgs &a, cudaStream_t s, cudaEvent_t *ev);
// Profiled rounds only, before the round's timed kernels: counts the edges
// live at the start of the round and their pins (HM_STAT_LEDGES/LPINS).
void launch_live_edges(const Handle *h, const RoundArgs &a, cudaStream_t s, int random);
void launch_win_kill_end(const Handle *h, const RoundArgs &a, cudaStream_t s, cudaEvent_t *ev,
                         int kill_stride = 1);
// Captures `capture(stream)` into g after the current nodes and returns the
// one new node nothing depends on (the end of the captured chain).
hm_status capture_chain(Handle *h, cudaGraph_t g, void (*capture)(Handle *, cudaStream_t, void *), void *ctx,
                        cudaGraphNode_t *tail);
// Adds a conditional while node after `after` whose body is `body(stream)`.
hm_status add_while_loop(Handle *h, cudaGraph_t g, cudaGraphNode_t after, cudaGraphConditionalHandle cond,
                         void (*body)(Handle *, cudaStream_t, void *), void *ctx);

// ---- re-randomised rounds (rrounds.cu) ----
// Allocates the extra buffers on first use and builds the j -> input maps.
hm_status rand_prepare(Handle *h, cudaStream_t s);
hm_status launch_match_graph_rand(Handle *h, cudaStream_t s);
hm_status profile_match_rand(Handle *h, cudaStream_t s, double *ms, int64_t *launches, double *round_ms,
                             int32_t max_rounds);
void free_rand_buffers(Handle *h);
// The per-vertex state after the last re-randomised match (hm_vertex_state).
cudaError_t launch_rand_vertex_state(const Handle *h, int32_t *out_dev, cudaStream_t s);

// SplitMix64 (Steele, Lea, Flood 2014): output number k (k >= 1) of the
// generator whose state starts at s0. The first output for a seed is
// splitmix64_at(seed, 1).
__host__ __device__ inline uint64_t splitmix64_at(uint64_t s0, uint64_t k) {
    uint64_t x = s0 + k * 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}
__host__ __device__ inline uint64_t splitmix64_first(uint64_t seed) { return splitmix64_at(seed, 1); }

// MurmurHash3 32-bit finaliser (Appleby): a bijection on 32-bit words. The
// unweighted priority of edge e is fmix32(e ^ s), s = low 32 bits of
// splitmix64_first(seed); every path that orders edges uses this one copy.
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// True when p is device memory usable by kernels of the current device:
// memory of the current device, or managed memory. Memory of another GPU
// is refused (without peer access a kernel would fault on it).
bool usable_device_pointer(const void *p);

// Stream-ordered device allocation of `count` elements (at least one);
// HM_ENOMEM with a message naming `what` on failure.
template <typename T>
hm_status dalloc(T **p, uint64_t count, cudaStream_t s, const char *what) {
    cudaError_t e = cudaMallocAsync((void **)p, (size_t)(count > 0 ? count : 1) * sizeof(T), s);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error(std::string("out of device memory allocating ") + what + " (" +
                  std::to_string((unsigned long long)(count * sizeof(T))) + " bytes)");
        return HM_ENOMEM;
    }
    return HM_OK;
}

inline unsigned grid_for(uint64_t work, int threads, int sm_count, int per_sm) {
    uint64_t need = (work + threads - 1) / threads;
    uint64_t cap = (uint64_t)sm_count * per_sm;
    if (need < 1) need = 1;
    return (unsigned)(need < cap ? need : cap);
}

}  // namespace hm
