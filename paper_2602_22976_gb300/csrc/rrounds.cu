// rrounds.cu - the paper's re-randomised rounds on the device: before every
// round each live edge draws a fresh random priority (Sec. 3.1; Sec. 5.1
// draws random weights per round), here
//     p_r(e) = base_e + a * U_r(e)   in float32,
//     key_r(e) = (bits(p_r(e)) << 32) | (0xFFFFFFFF - e),
// base_e = w_e (1.0f unweighted), U_r(e) = top 24 bits of output number
// (r << 32) + e + 1 of a SplitMix64 stream started at the first output for
// the seed, times 2^-24. Nothing random is stored: every key is recomputed
// from (seed, r, e) where it is needed.
//
// With priorities that change every round there is no fixed list order for
// a cursor to walk. Every round each active vertex scans its live list,
// takes the largest key among the live entries (Alg. 3's argmax), and
// compacts it, so an entry is read at most once after its edge died. List
// entries carry what the key needs, {input edge id e, bits(base_e)}, so
// round 1 streams the lists with no random read at all (every edge is live
// then); later rounds add one 1-byte live-flag read per entry, from an
// array indexed by input id (m bytes, L2-resident). Round 1 reads the
// immutable lists (vadjE) and writes nothing (it keeps every entry); round 2
// reads vadjE and writes the compacted lists to the working copy (vadjR);
// later rounds compact vadjR in place. Lists are scheduled by length:
//   - at most kLong entries: the 32 vertices of a warp tile are scanned as
//     one concatenated sequence, each lane taking kE consecutive entries of
//     a batch (scan_tile: per-list maxima folded in shared memory, one warp
//     scan per batch for the compaction offsets), so short and medium lists
//     keep every lane busy;
//   - longer lists: queued with their chunk count (one 64-bit atomic hands
//     out the queue slot and the first chunk); k_rlong scans the chunks of
//     kChunk entries with one warp each and combines them per list with a
//     64-bit atomicMax. Long lists are not compacted: they are scanned from vadjE,
//     and their part of vadjR (read by the kill step) is copied once when
//     the handle first runs this mode and never written.
// Proposals use the P counter of Alg. 1 counted up and double-buffered by
// round parity, indexed by input edge id and packed with the edge's size
// (propose): a vertex adds 1 to P_r[T[v]] and learns from the same atomic
// whether the count reached |e| (the edge wins); it clears the count it
// added in the previous round in the other buffer, which the next round
// reuses. Every vertex that proposed a still-live edge is active in the
// next round and clears it; stale counts are left only on dead edges, which
// nobody proposes again. T[v] holds the input id; the winner list holds
// relabelled ids j (looked up for the winners only). The scans leave each
// vertex's largest key of the round in rbest; k_rpropose then makes all
// proposals of the round, one vertex per thread, so a proposal's random
// access is not on the scans' critical path.
// The win kernel and the kill kernel (which ends the round) of rounds.cu
// run on this handle's re-randomised vertex records and lists: the cursor
// field stays 0, so the kill range of a matched vertex is its whole
// (compacted) list, and the kill step (reading every second word: the edge
// ids of the pairs; from vadjE in round 1) clears the flags of the input ids
// there. Graphs (every edge has two pins) need no kill: each list entry
// also has its edge's other endpoint (vnbrE, compacted into vnbrR with the
// pairs), an entry is live while that endpoint is unmatched, the win step
// only sets the matched flags of the winners' endpoints, and a vertex whose
// own flag is set drops out.
#include "hm_internal.cuh"

#include <algorithm>
#include <cmath>

namespace hm {
namespace {

constexpr int kT = 256;
constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kLong = 2048;   // lists longer than this are scanned in chunks
constexpr uint32_t kChunk = 2048;  // entries per chunk of a long list

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

__device__ __forceinline__ void block_add_u64(unsigned long long x, unsigned long long *s_red,
                                              unsigned long long *dst) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(kFull, x, d);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s_red[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kT / 32; ++w) t += s_red[w];
        if (t) atomicAdd(dst, t);
    }
    __syncthreads();
}

// key_r(e) of input edge e whose base priority is `base`: p_r(e) = base +
// scale * U_r(e), the product and the sum rounded separately (no fused
// multiply-add), as the definition's float32 operations are. U_r(e) comes
// from output number (r << 32) + e + 1 of the SplitMix64 stream started at
// s0, computed in fewer operations than splitmix64_at: cr = s0 + ((r << 32)
// + 1) * gamma (one value per round), so that output's state is cr + e *
// gamma; and the output's last step, x ^ (x >> 31), leaves bits 33..63
// unchanged, so the top 24 bits are those of x itself.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;
__device__ __forceinline__ uint64_t round_counter_base(uint64_t s0, int r) {
    return s0 + ((((uint64_t)(uint32_t)r) << 32) + 1u) * kGamma;
}
__device__ __forceinline__ unsigned long long scan_key(uint64_t cr, float scale, uint32_t e, float base) {
    uint64_t x = cr + (uint64_t)e * kGamma;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    const float u = __uint2float_rn((uint32_t)(x >> 40));
    const float p = __fadd_rn(base, __fmul_rn(u, scale));
    return ((unsigned long long)__float_as_uint(p) << 32) | (unsigned long long)(0xFFFFFFFFu - e);
}

__device__ __forceinline__ int32_t edge_of_key(unsigned long long k) {
    return (int32_t)(0xFFFFFFFFu - (uint32_t)k);
}

// The P counter of round r for input edge e, packed with the edge's size:
// word = (|e| << H) | count, H = 16 when no edge has more than 65535 pins
// (two 32-bit buffers), else H = 32 (two 64-bit buffers). A proposal adds 1
// and gets the size back with the old count from the same atomic, so no
// other read is needed to see whether it completed the edge; the clear of
// the previous round's count keeps the size half. The buffers start each
// match as copies of the sizes (k_rinit). A graph's edges all have two
// pins: its counts are 8-bit, four to a 32-bit word, with no size beside
// them (the count an edge reaches is at most 2), so the counters of m edges
// take m bytes and stay in L2.
__device__ __forceinline__ bool propose(const RoundArgs &a, int r, int32_t e) {
    if (a.pairs) {  // graphs: every edge has two pins; four 8-bit counts a word, no size needed
        uint32_t *W = (r & 1) ? a.P2 : a.P;
        const int sh = (e & 3) * 8;
        const uint32_t old = atomicAdd(W + (e >> 2), 1u << sh);
        return ((old >> sh) & 0xFFu) == 1u;
    }
    if (a.w64) {
        unsigned long long *W = (r & 1) ? a.W64b : a.W64a;
        const unsigned long long old = atomicAdd(W + e, 1ull);
        return (old & 0xFFFFFFFFull) + 1ull == (old >> 32);
    }
    uint32_t *W = (r & 1) ? a.P2 : a.P;
    const uint32_t old = atomicAdd(W + e, 1u);
    return (old & 0xFFFFu) + 1u == (old >> 16);
}

// Clears the count a vertex added to edge e in round r - 1 (its T then).
__device__ __forceinline__ void clear_previous(const RoundArgs &a, int r, int32_t e) {
    if (a.pairs) atomicAnd(((r & 1) ? a.P : a.P2) + (e >> 2), ~(0xFFu << ((e & 3) * 8)));
    else if (a.w64) atomicAnd(((r & 1) ? a.W64a : a.W64b) + e, 0xFFFFFFFF00000000ull);
    else atomicAnd(((r & 1) ? a.P : a.P2) + e, 0xFFFF0000u);
}

__global__ void __launch_bounds__(kT) k_rinit(RoundArgs a) {
    const int64_t total = a.n > a.m ? a.n : a.m;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < total; i += (int64_t)gridDim.x * kT) {
        if (i < a.m) {
            a.alive[i] = 1;
            if (a.pairs) {  // four 8-bit counts a word
                if (i < (a.m + 3) / 4) {
                    a.P[i] = 0;
                    a.P2[i] = 0;
                }
            } else if (a.w64) {
                const unsigned long long z = __ldg(a.S64 + i);
                a.W64a[i] = z;
                a.W64b[i] = z;
            } else {
                const uint32_t z = __ldg(a.S32 + i);
                a.P[i] = z;
                a.P2[i] = z;
            }
            a.inM[i] = 0;
        }
        if (i < a.n) {
            if (a.pairs) a.vmatch[i] = 0;
            a.rbest[i] = 0;  // round 1 folds list pieces into it with atomicMax
            const int64_t b = a.voff[i], e = a.voff[i + 1];
            a.vrec[i] = make_int4(a.firstj[i], 0, (int32_t)(uint32_t)b, (int32_t)(uint32_t)(e - b));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        DevState *st = a.st;
        st->round = 1;
        st->parity = 0;
        st->cnt[0] = st->cnt[1] = 0;
        st->nwin = 0;
        st->kdone = 0;
        st->rgrab = 0;
        st->status = HM_OK;
        st->rounds_done = 0;
        st->finished = 0;
        st->fault = 0;
        st->adv = st->kills = st->winpins = st->proposals = 0;
        st->lpack = st->live = st->kpack = st->sdeg = 0;
        st->ledges = st->lpins = 0;
    }
}

// Adds a warp's counter to *dst with one atomic.
__device__ __forceinline__ void warp_add_u64(unsigned long long x, unsigned long long *dst) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(kFull, x, d);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(dst, x);
}

// Appends a region's staged winners to the round's list with one atomic
// (one counter word for the whole GPU: an atomic per winning step would
// serialise on it). Kept out of line: inlined into k_rargmax it changed the
// code of the scan loop and cost 0.3-0.5 ms in the scan-heavy rounds.
__device__ __noinline__ void flush_winners(const RoundArgs &a, uint64_t base, uint32_t won) {
    const int lane = threadIdx.x & 31;
    uint32_t wb = 0;
    if (lane == 0) wb = atomicAdd(&a.st->nwin, won);
    wb = __shfl_sync(kFull, wb, 0);
    __syncwarp();
    for (uint32_t x = lane; x < won; x += 32) {
        const uint64_t idx = (uint64_t)wb + x;
        if (idx < a.win_cap) a.win[idx] = a.wstage[base + x];
        else a.st->fault = 2;
    }
}

constexpr int kE = 4;  // consecutive entries a lane takes per batch of the tile scan
constexpr int kFlatC = 32;              // round 1: consecutive entries a lane takes per chunk
constexpr uint64_t kFlatW = 32 * kFlatC;  // round 1: entries per warp chunk
constexpr int kFlatSpan = 192;          // round 1: a chunk's vertex offsets staged in shared memory up to this many

// Per-warp tile state of the scan in shared memory: for each lane's vertex
// (its owner index) the start and end of its list in the tile's
// concatenated sequence, the list's first entry in memory, the running
// maximum key and live count, and the tile's live count before the list
// (compaction offsets).
struct TileSmem {
    uint32_t pre[32], end[32], base[32], gst[32], live[32];
    unsigned long long best[32];
};
// round 1 stages up to kFlatSpan vertex offsets in a warp's TileSmem
static_assert(kFlatSpan * sizeof(uint32_t) <= sizeof(TileSmem), "the staged offsets must fit a warp's tile state");

// The short and medium lists of a tile of 32 vertices (L = list length of
// this lane's vertex, 0 when it takes no part; lb = its first entry), read
// as one concatenated sequence in batches of 32 * kE entries: lane l takes
// the kE consecutive positions from batch start + l * kE, finds the list
// holding its first one by a binary search over the lists' starts, and
// walks on (a run rarely crosses more than one list end). Each lane keeps
// the maximum key and live count of every list piece in its run and folds
// them into the list's shared entries with one atomic per piece. From round
// 2 on the live entries are compacted: a warp scan of the lanes' live counts
// gives every entry its place among the tile's live entries, and the live
// count at each list's start (recorded by the lane holding that start)
// turns it into the place in the list's own compacted copy. All reads of a
// batch precede its writes (__syncwarp), and compacted entries land at or
// before the positions they were read from, so compaction in place is safe.
// Returns the list's maximum key (0: nothing live) and live count.
template <bool kPairs>
__device__ __forceinline__ void scan_tile(const RoundArgs &a, int r, const int2 *src, int2 *dst,
                                          const int32_t *nsrc, int32_t *ndst, uint32_t L, uint32_t lb,
                                          TileSmem &sm, unsigned long long &best, uint32_t &live,
                                          unsigned long long &scanned) {
    const int lane = threadIdx.x & 31;
    const uint32_t inc = warp_inclusive_scan(L);
    const uint32_t total = __shfl_sync(kFull, inc, 31);
    best = 0;
    live = 0;
    if (total == 0) return;  // warp-uniform
    sm.pre[lane] = inc - L;
    sm.end[lane] = inc;
    sm.base[lane] = lb;
    sm.best[lane] = 0;
    sm.live[lane] = 0;
    __syncwarp();
    uint32_t gbase = 0;  // live entries of the tile before this batch
    const uint64_t cr = round_counter_base(a.noise_s0, r);
    for (uint32_t s0 = 0; s0 < total; s0 += 32 * kE) {
        const uint32_t p0 = s0 + (uint32_t)lane * kE;
        // the list holding p0: the largest x with pre[x] <= p0 (a non-empty
        // list whenever p0 < total)
        int x = 0;
#pragma unroll
        for (int bit = 16; bit; bit >>= 1)
            if (sm.pre[x + bit] <= p0) x += bit;
        int own[kE];
        bool lv[kE], first[kE];
        int2 ev[kE];
        int32_t nb[kE];
        {
            int o = x;
            uint32_t cend = sm.end[o], cpre = sm.pre[o], cbase = sm.base[o];
#pragma unroll
            for (int k = 0; k < kE; ++k) {
                const uint32_t p = p0 + k;
                const bool valid = p < total;
                if (valid)
                    while (p >= cend) {  // past this list's end (empty lists end where they start)
                        ++o;
                        cend = sm.end[o];
                        cpre = sm.pre[o];
                        cbase = sm.base[o];
                    }
                own[k] = o;
                first[k] = valid && p == cpre;
                const uint64_t at = (uint64_t)cbase + (p - cpre);
                // plain loads: from round 3 on this kernel rewrites the lists behind the reads
                ev[k] = valid ? src[at] : make_int2(0, 0);
                if (kPairs) nb[k] = valid ? nsrc[at] : 0;
                lv[k] = valid;
            }
        }
        if (r > 1) {
#pragma unroll
            for (int k = 0; k < kE; ++k)
                lv[k] = lv[k] && (kPairs ? __ldg(a.vmatch + nb[k]) == 0 : __ldg(a.alive + ev[k].x) != 0);
        }
        // the run's pieces: maximum key and live count per list, each piece
        // folded into its list's shared entries with one atomic
        uint32_t lcnt = 0;
        {
            unsigned long long m = 0;
            uint32_t c = 0;
            int co = own[0];
#pragma unroll
            for (int k = 0; k < kE; ++k) {
                if (own[k] != co) {
                    if (c) {
                        atomicMax(&sm.best[co], m);
                        atomicAdd(&sm.live[co], c);
                    }
                    co = own[k];
                    m = 0;
                    c = 0;
                }
                if (lv[k]) {
                    const unsigned long long key = scan_key(cr, a.noise_scale, (uint32_t)ev[k].x,
                                                            __int_as_float(ev[k].y));
                    m = key > m ? key : m;
                    ++c;
                }
                lcnt += lv[k] ? 1u : 0u;
            }
            scanned += p0 < total ? min(total - p0, (uint32_t)kE) : 0u;
            if (c) {
                atomicMax(&sm.best[co], m);
                atomicAdd(&sm.live[co], c);
            }
        }
        if (r > 1) {  // compaction
            const uint32_t incl = warp_inclusive_scan(lcnt);
            const uint32_t g0 = gbase + incl - lcnt;  // live entries of the tile before this lane's run
            uint32_t g = g0;
#pragma unroll
            for (int k = 0; k < kE; ++k) {
                if (first[k]) sm.gst[own[k]] = g;
                g += lv[k] ? 1u : 0u;
            }
            __syncwarp();  // every read of this batch and every list start precede the writes
            g = g0;
#pragma unroll
            for (int k = 0; k < kE; ++k)
                if (lv[k]) {
                    const uint64_t at = (uint64_t)sm.base[own[k]] + (g - sm.gst[own[k]]);
                    dst[at] = ev[k];
                    if (kPairs) ndst[at] = nb[k];
                    ++g;
                }
            gbase += __shfl_sync(kFull, incl, 31);
        }
        __syncwarp();
    }
    best = sm.best[lane];
    live = sm.live[lane];
    __syncwarp();  // the next tile rewrites the shared state
}

// Round 1 of the re-randomised rounds: every entry is live, so each
// vertex's largest key is a plain maximum over its whole list. The lists
// (vadjE, in vertex order) are read as one flat array: a warp takes chunks
// of kFlatW consecutive entries, each lane kFlatC of them (16-byte loads),
// whatever lists they belong to. A lane finds the vertex of its first entry
// by a binary search over the vertex offsets between the vertices owning
// this chunk's and the next chunk's first entries (vchunk, built once), and
// walks on through the lists its run touches. A list that lies wholly inside
// the run is stored at once; a piece of a longer list is folded into the
// vertex's largest key with a 64-bit atomicMax (rbest starts at 0), one per
// warp when the whole chunk lies inside one list. The proposals follow in
// k_rpropose; nothing else is written.
template <bool kPairs>
__device__ __forceinline__ void flat_round1(const RoundArgs &a, uint32_t *s_off) {
    // list positions are below kappa < 2^32: 32-bit arithmetic throughout
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * (uint32_t)kT + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * (uint32_t)kT) >> 5;
    const uint32_t kappa = (uint32_t)a.kappa;
    const uint32_t nchunks = (uint32_t)((a.kappa + kFlatW - 1) / kFlatW);
    const uint64_t cr = round_counter_base(a.noise_s0, 1);
    const float scale = a.noise_scale;
    for (uint32_t c = warp; c < nchunks; c += nwarps) {  // uniform in the warp
        const uint32_t cb = c * (uint32_t)kFlatW;
        const uint32_t p0 = cb + (uint32_t)lane * kFlatC;
        // this lane's positions p0 .. p0 + len - 1 (none when p0 >= kappa);
        // cb is a multiple of kFlatW below kappa <= 2^32 - 1, so p0 <=
        // 2^32 - 32 does not wrap
        const uint32_t len = p0 < kappa ? min((uint32_t)kFlatC, kappa - p0) : 0u;
        // the chunk's vertices lie in [vlo, vhi]; when there are fewer than
        // kFlatSpan of them their offsets are staged in this warp's shared
        // array (the search and the walk then read shared memory)
        const int32_t vlo = __ldg(a.vchunk + c);
        const int32_t vhi = c + 1 < nchunks ? __ldg(a.vchunk + c + 1) : (int32_t)(a.n - 1);
        const bool staged = vhi - vlo + 1 < kFlatSpan;  // uniform: offsets vlo .. vhi + 1 fit
        __syncwarp();  // the previous chunk's reads of the shared array are done
        if (staged) {
            for (int32_t i = lane; i <= vhi - vlo + 1; i += 32) s_off[i] = (uint32_t)__ldg(a.voff + vlo + i);
            __syncwarp();
        }
        auto vo = [&](int32_t v) -> uint32_t {
            return staged ? s_off[v - vlo] : (uint32_t)__ldg(a.voff + v);
        };
        int32_t cur = 0;
        uint32_t cs = 0, ce = 0;
        if (len) {
            // the vertex whose list holds p0: the largest v with voff[v] <= p0
            // (its list is not empty: a later vertex with the same offset
            // would be larger)
            int32_t lo = vlo, hi = vhi;
            while (lo < hi) {
                const int32_t mid = (int32_t)(((int64_t)lo + hi + 1) >> 1);
                if (vo(mid) <= p0) lo = mid;
                else hi = mid - 1;
            }
            cur = lo;
            cs = vo(cur);
            ce = vo(cur + 1);
        }
        // a chunk inside one list (the lists of hubs): one atomic per warp
        // (every lane takes part in every shuffle: none sits behind a condition)
        const uint32_t cs0 = __shfl_sync(kFull, cs, 0), cs31 = __shfl_sync(kFull, cs, 31);
        const uint32_t ce0 = __shfl_sync(kFull, ce, 0);
        const bool one = cs0 == cs31 && len == (uint32_t)kFlatC && ce0 - cb >= (uint32_t)kFlatW;
        const bool all_one = __all_sync(kFull, one);
        unsigned long long m = 0;
#pragma unroll 1
        for (uint32_t k0 = 0; k0 < len; k0 += 8) {
            int2 ev[8];
            if (k0 + 8 <= len) {  // four 16-byte loads: p0 + k0 is even, so 16-byte aligned
                const int4 *v4 = reinterpret_cast<const int4 *>(a.vadjE + p0 + k0);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int4 x = __ldg(v4 + u);
                    ev[2 * u] = make_int2(x.x, x.y);
                    ev[2 * u + 1] = make_int2(x.z, x.w);
                }
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) ev[u] = k0 + u < len ? __ldg(a.vadjE + p0 + k0 + u) : make_int2(0, 0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (k0 + u >= len) break;
                const uint32_t p = p0 + k0 + u;
                if (!all_one)
                    while (p >= ce) {  // the list of cur ends before p: store or fold its piece
                        if (cs >= p0) a.rbest[cur] = m;  // the whole list lay inside this run
                        else if (m) atomicMax(a.rbest + cur, m);
                        m = 0;
                        ++cur;
                        cs = ce;
                        ce = vo(cur + 1);
                    }
                const unsigned long long key = scan_key(cr, scale, (uint32_t)ev[u].x, __int_as_float(ev[u].y));
                m = key > m ? key : m;
            }
        }
        if (all_one) {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                const unsigned long long y = __shfl_xor_sync(kFull, m, d);
                m = y > m ? y : m;
            }
            if (lane == 0) atomicMax(a.rbest + cur, m);
        } else if (len) {  // the run's last piece
            if (cs >= p0 && ce - p0 <= len) a.rbest[cur] = m;
            else if (m) atomicMax(a.rbest + cur, m);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // round 1 scans and finds live every entry
        atomicAdd(&a.st->adv, (unsigned long long)a.kappa);
        atomicAdd(&a.st->live, (unsigned long long)a.kappa);
    }
}

// a1 of a re-randomised round for the vertices of the active list. The
// regions are those of the fixed-order loop; warps of a persistent grid
// take them one at a time from a counter, so that regions with long lists
// do not leave other warps idle.
template <bool kPairs>
__global__ void __launch_bounds__(kT, 4) k_rargmax(RoundArgs a) {
    __shared__ TileSmem s_tile[kT / 32];
    DevState *st = a.st;
    const int r = st->round;
    const int par = st->parity;
    const int32_t *in = par ? a.list1 : a.list0;
    int32_t *out = par ? a.list0 : a.list1;
    const uint32_t *cnt_in = a.lcnt + (size_t)par * a.nregions;
    uint32_t *cnt_out = a.lcnt + (size_t)(par ^ 1) * a.nregions;
    // round 1 keeps every entry: it reads the immutable lists and writes
    // nothing; round 2 compacts them into the working copy; later rounds
    // compact the working copy in place
    const int2 *src = r <= 2 ? a.vadjE : a.vadjR;
    int2 *dst = a.vadjR;
    const int32_t *nsrc = r <= 2 ? a.vnbrE : a.vnbrR;  // graphs
    int32_t *ndst = a.vnbrR;
    if (r == 1) {  // uniform: round 1 is a flat scan of every list (k_rpropose builds the kept list)
        flat_round1<kPairs>(a, reinterpret_cast<uint32_t *>(&s_tile[threadIdx.x >> 5]));
        return;
    }
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    unsigned long long scanned = 0, nlive = 0;
    for (;;) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(&st->rgrab, 1u);
        g = __shfl_sync(kFull, g, 0);
        if (g >= a.nregions) break;
        const uint64_t base = (uint64_t)g * a.region;
        uint32_t count;
        if (r == 1) {
            const int64_t left = a.n - (int64_t)base;
            count = left <= 0 ? 0u : (uint32_t)(left < (int64_t)a.region ? left : (int64_t)a.region);
        } else {
            count = cnt_in[g];
        }
        uint32_t kept = 0;
        for (uint32_t i0 = 0; i0 < count; i0 += 32) {
            const uint32_t i = i0 + lane;
            const bool ok = i < count;
            const int32_t v = ok ? (r == 1 ? (int32_t)(base + i) : in[base + i]) : 0;
            const bool mine = kPairs && ok && __ldg(a.vmatch + v) != 0;  // graphs: v is matched
            const int4 rec = ok ? a.vrec[v] : make_int4(kCurNone, 0, 0, 0);
            const bool act = rec.x >= 0 && !mine;
            const bool lng = act && (uint32_t)rec.w > kLong;
            if (lng) {  // queue slot and first chunk from one atomic, so both ascend together
                const uint32_t nch = ((uint32_t)rec.w + kChunk - 1) / kChunk;
                const unsigned long long old = atomicAdd(&st->lpack, (1ull << 32) | nch);
                const uint32_t slot = (uint32_t)(old >> 32);
                if (slot < a.lq_cap) a.lq[slot] = make_int2(v, (int32_t)(uint32_t)old);
                else st->fault = 3;
                a.rbest[v] = 0;  // k_rlong folds the chunks' maxima in
            }
            // the short and medium lists of the tile as one sequence
            const uint32_t L = act && !lng ? (uint32_t)rec.w : 0u;
            unsigned long long best = 0;
            uint32_t live = 0;
            scan_tile<kPairs>(a, r, src, dst, nsrc, ndst, L, (uint32_t)rec.z, s_tile[threadIdx.x >> 5], best, live,
                              scanned);
            // the vertex's best key goes to k_rpropose, which makes every
            // proposal of the round (a dependent chain of random reads that
            // would otherwise sit in this scan's critical path)
            bool keep = false;
            if (act && !lng) {
                if (r > 1) clear_previous(a, r, rec.x);  // T[v] of the previous round is what v counted there
                a.rbest[v] = best;
                if (best != 0) {
                    reinterpret_cast<int2 *>(a.vrec + v)[1] = make_int2(rec.z, (int32_t)live);
                    keep = true;
                    nlive += live;
                } else {
                    reinterpret_cast<int2 *>(a.vrec + v)[0] = make_int2(kCurNone, 0);
                }
            }
            const unsigned km = __ballot_sync(kFull, keep);
            if (keep) out[base + kept + __popc(km & lt)] = v;
            kept += __popc(km);
            const unsigned lgm = __ballot_sync(kFull, lng);  // long lists stay; k_rpropose may drop them
            if (lng) out[base + kept + __popc(lgm & lt)] = v;
            kept += __popc(lgm);
        }
        if (lane == 0) {
            cnt_out[g] = kept;
            if (kept) atomicAdd(&st->cnt[par ^ 1], kept);
        }
    }
    warp_add_u64(scanned, &st->adv);
    warp_add_u64(nlive, &st->live);
}

// Chunks of the long lists: one warp per chunk of kChunk entries, maximum
// key of the live entries combined per list with atomicMax.
template <bool kPairs>
__global__ void __launch_bounds__(kT) k_rlong(RoundArgs a) {
    __shared__ unsigned long long s_red[kT / 32];
    DevState *st = a.st;
    const unsigned long long lp = st->lpack;
    const uint32_t nl = (uint32_t)(lp >> 32), nchunks = (uint32_t)lp;
    unsigned long long scanned = 0, nlive = 0;
    if (nl > 0 && nl <= a.lq_cap) {
        const int r = st->round;
        const int lane = threadIdx.x & 31;
        const uint32_t warp = (blockIdx.x * kT + threadIdx.x) >> 5;
        const uint32_t nwarps = (gridDim.x * kT) >> 5;
        for (uint32_t c = warp; c < nchunks; c += nwarps) {
            uint32_t lo = 0, hi = nl - 1;  // the last list whose first chunk is <= c
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if ((uint32_t)a.lq[mid].y <= c) lo = mid; else hi = mid - 1;
            }
            const int2 q = a.lq[lo];  // {vertex, its first chunk}
            const int4 rec = a.vrec[q.x];
            const int64_t lb = (int64_t)(uint32_t)rec.z;
            const int64_t b = lb + (int64_t)(c - (uint32_t)q.y) * kChunk;
            const int64_t e = min(lb + (int64_t)(uint32_t)rec.w, b + (int64_t)kChunk);
            unsigned long long mx = 0;
            const uint64_t cr = round_counter_base(a.noise_s0, r);
            int64_t p = b + lane;
            for (; p + 96 < e; p += 128) {  // four entries per lane in flight
                int2 x[4];
                bool lv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = __ldg(a.vadjE + p + 32 * u);  // long lists are never compacted
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    lv[u] = r == 1 || (kPairs ? __ldg(a.vmatch + __ldg(a.vnbrE + p + 32 * u)) == 0
                                              : __ldg(a.alive + x[u].x) != 0);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (lv[u]) {
                        const unsigned long long k = scan_key(cr, a.noise_scale, (uint32_t)x[u].x,
                                                              __int_as_float(x[u].y));
                        if (k > mx) mx = k;
                        ++nlive;
                    }
            }
            for (; p < e; p += 32) {
                const int2 x = __ldg(a.vadjE + p);
                if (r == 1 || (kPairs ? __ldg(a.vmatch + __ldg(a.vnbrE + p)) == 0 : __ldg(a.alive + x.x) != 0)) {
                    const unsigned long long k = scan_key(cr, a.noise_scale, (uint32_t)x.x, __int_as_float(x.y));
                    if (k > mx) mx = k;
                    ++nlive;
                }
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                const unsigned long long y = __shfl_xor_sync(kFull, mx, d);
                if (y > mx) mx = y;
            }
            if (lane == 0) {
                if (mx) atomicMax(a.rbest + q.x, mx);
                scanned += (unsigned long long)(e - b);
            }
        }
    }
    block_add_u64(scanned, s_red, &st->adv);
    block_add_u64(nlive, s_red, &st->live);
}

// Every proposal of the round: for each vertex the argmax step kept (one
// warp per region of the kept list), its largest key of the round (rbest,
// from the scan or from the chunks of a long list) names its new T[v]; the
// vertex counts itself in P_r of that edge, and the count that completes the
// edge makes it a winner. A long list with nothing live left drops out here
// (T[v] = none; the vertex leaves the active count). Winners are staged per
// region and appended with one atomic.
__global__ void __launch_bounds__(kT) k_rpropose(RoundArgs a) {
    __shared__ unsigned long long s_red[kT / 32];
    DevState *st = a.st;
    const int r = st->round, par = st->parity;
    int32_t *out = par ? a.list0 : a.list1;
    uint32_t *cnt_out = a.lcnt + (size_t)(par ^ 1) * a.nregions;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const uint64_t warp = (blockIdx.x * (uint64_t)kT + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * kT) >> 5;
    unsigned long long props = 0;
    if (r == 1) {  // uniform: the flat scan left every vertex's largest key; keep those with a list
        int32_t *keep_out = out;
        for (uint64_t g = warp; g < a.nregions; g += nwarps) {
            const uint64_t base = g * a.region;
            const int64_t left = a.n - (int64_t)base;
            const uint32_t c = left <= 0 ? 0u : (uint32_t)(left < (int64_t)a.region ? left : (int64_t)a.region);
            uint32_t won = 0, kept = 0;
            for (uint32_t i0 = 0; i0 < c; i0 += 32) {
                const uint32_t i = i0 + lane;
                bool w = false, keep = false;
                int32_t nb = -1;
                const int32_t v = (int32_t)(base + i);
                if (i < c) {
                    const unsigned long long best = a.rbest[v];
                    if (best != 0) {
                        const int32_t e = edge_of_key(best);  // T[v], input id
                        reinterpret_cast<int2 *>(a.vrec + v)[0] = make_int2(e, 0);
                        w = propose(a, r, e);
                        if (w) nb = __ldg(a.jof + e);
                        keep = true;
                        ++props;
                    }
                }
                const unsigned km = __ballot_sync(kFull, keep);
                if (keep) keep_out[base + kept + __popc(km & lt)] = v;
                kept += __popc(km);
                const unsigned wm = __ballot_sync(kFull, w);
                if (w) a.wstage[base + won + __popc(wm & lt)] = nb;
                won += __popc(wm);
            }
            if (lane == 0) {
                cnt_out[g] = kept;
                if (kept) atomicAdd(&st->cnt[par ^ 1], kept);
            }
            if (won) flush_winners(a, base, won);
        }
        block_add_u64(props, s_red, &st->proposals);
        return;
    }
    for (uint64_t g = warp; g < a.nregions; g += nwarps) {
        const uint32_t c = cnt_out[g];
        const uint64_t base = g * a.region;
        uint32_t won = 0;
        for (uint32_t i0 = 0; i0 < c; i0 += 32) {
            const uint32_t i = i0 + lane;
            bool w = false;
            int32_t nb = -1;
            if (i < c) {
                const int32_t v = out[base + i];
                const unsigned long long best = a.rbest[v];
                const int4 rec = a.vrec[v];
                // a long list (never compacted: its length field stays above
                // kLong) clears what it counted in the previous round here
                if ((uint32_t)rec.w > kLong && r > 1) clear_previous(a, r, rec.x);
                if (best == 0) {  // a long list with nothing live left
                    reinterpret_cast<int2 *>(a.vrec + v)[0] = make_int2(kCurNone, 0);
                    atomicSub(&st->cnt[par ^ 1], 1u);
                } else {
                    const int32_t e = edge_of_key(best);  // T[v], input id
                    reinterpret_cast<int2 *>(a.vrec + v)[0] = make_int2(e, 0);
                    w = propose(a, r, e);
                    if (w) nb = __ldg(a.jof + e);  // winners are listed by relabelled id
                    ++props;
                }
            }
            const unsigned wm = __ballot_sync(kFull, w);
            if (w) a.wstage[base + won + __popc(wm & lt)] = nb;
            won += __popc(wm);
        }
        if (won) flush_winners(a, base, won);
    }
    block_add_u64(props, s_red, &st->proposals);
}

// Graphs: the other endpoint of every list entry (the second word of the
// fixed order's {edge, endpoint} pairs, in the same list order).
__global__ void __launch_bounds__(kT) k_pair_endpoints(const int2 *vpair, uint64_t kappa, int32_t *vnbrE) {
    for (uint64_t i = blockIdx.x * (uint64_t)kT + threadIdx.x; i < kappa; i += (uint64_t)gridDim.x * kT)
        vnbrE[i] = vpair[i].y;
}

// Round 1's flat scan: the vertex whose list holds entry c * kFlatW, for
// every chunk c (the largest v with voff[v] <= c * kFlatW).
__global__ void __launch_bounds__(kT) k_vchunk(const int64_t *voff, int64_t n, uint64_t nchunks, int32_t *vchunk) {
    for (uint64_t c = blockIdx.x * (uint64_t)kT + threadIdx.x; c < nchunks; c += (uint64_t)gridDim.x * kT) {
        const uint64_t p = c * kFlatW;
        int64_t lo = 0, hi = n - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if ((uint64_t)voff[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        vchunk[c] = (int32_t)lo;
    }
}

// The proposal words' start value by input id: |e| in the upper half.
__global__ void __launch_bounds__(kT) k_size_words(const int32_t *order, const int64_t *eoffj, int64_t m, int graph,
                                                   uint32_t *S32, unsigned long long *S64) {
    for (int64_t j = blockIdx.x * (int64_t)kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT) {
        const int32_t e = __ldg(order + j);
        const uint64_t size = graph ? 2u : (uint64_t)(eoffj[j + 1] - eoffj[j]);
        if (S32) S32[e] = (uint32_t)size << 16;
        else S64[e] = (unsigned long long)size << 32;
    }
}

// Lists as {input edge id, bits(base priority)} pairs, both copies, and
// the inverse of the edge order (built once per handle).
__global__ void __launch_bounds__(kT) k_map(const int32_t *order, const int32_t *vadj, const float *w, int64_t m,
                                          uint64_t kappa, int2 *vadjE, int2 *vadjR, int32_t *jof) {
    const uint64_t stride = (uint64_t)gridDim.x * kT;
    for (uint64_t i = blockIdx.x * (uint64_t)kT + threadIdx.x; i < kappa; i += stride) {
        const int32_t e = __ldg(order + __ldg(vadj + i));
        const int2 x = make_int2(e, __float_as_int(w ? __ldg(w + e) : 1.0f));
        vadjE[i] = x;
        vadjR[i] = x;
    }
    for (uint64_t j = blockIdx.x * (uint64_t)kT + threadIdx.x; j < (uint64_t)m; j += stride)
        jof[order[j]] = (int32_t)j;
}

template <typename K>
int fit_per_sm(K kernel) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kT, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 2;
    }
    return per_sm;
}

RoundArgs rand_args(const Handle *h) {
    RoundArgs a = round_args(h);
    a.vrec = h->vrecR;
    a.pairs = h->graph ? 1 : 0;  // graphs: liveness from vmatch, flag-only win, no kill
    a.vnbrE = h->vnbrE;
    a.vnbrR = h->vnbrR;
    a.vadj = reinterpret_cast<const int32_t *>(h->vadjR);  // for the kill step: stride 2
    a.vadjE = h->vadjE;
    a.vadjR = h->vadjR;
    a.noise_scale = h->noise * (1.0f / 16777216.0f);
    a.noise_s0 = splitmix64_first(h->seed);
    a.jof = h->jof;
    a.P2 = h->P2;
    a.t_input = 1;
    a.w64 = h->p16 ? 0 : 1;
    a.S32 = h->S32;
    a.S64 = h->S64;
    a.W64a = h->W64a;
    a.W64b = h->W64b;
    a.vchunk = h->vchunk;
    a.kappa = h->kappa;
    a.lq = h->lq;
    a.rbest = h->rbest;
    a.lq_cap = h->lq_cap;
    return a;
}

unsigned rinit_grid(const Handle *h) {
    return grid_for((uint64_t)std::max(h->n, h->m), kT, h->sm_count, 16);
}

void launch_rinit(const Handle *h, const RoundArgs &a, cudaStream_t s) {
    k_rinit<<<rinit_grid(h), kT, 0, s>>>(a);
}

void launch_rround(const Handle *h, const RoundArgs &a, cudaStream_t s, cudaEvent_t *ev) {
    if (ev) cudaEventRecord(ev[0], s);
    if (a.pairs) {
        k_rargmax<true><<<h->rargmax_grid, kT, 0, s>>>(a);
        k_rlong<true><<<h->rlong_grid, kT, 0, s>>>(a);
    } else {
        k_rargmax<false><<<h->rargmax_grid, kT, 0, s>>>(a);
        k_rlong<false><<<h->rlong_grid, kT, 0, s>>>(a);
    }
    k_rpropose<<<h->rpropose_grid, kT, 0, s>>>(a);
    if (ev) launch_kept_degrees(h, a, s, ev, 1);
    launch_win_kill_end(h, a, s, ev, 2);
}

void capture_rinit(Handle *h, cudaStream_t s, void *ctx) {
    launch_rinit(h, *static_cast<const RoundArgs *>(ctx), s);
}

void capture_rround(Handle *h, cudaStream_t s, void *ctx) {
    launch_rround(h, *static_cast<const RoundArgs *>(ctx), s, nullptr);
}

hm_status build_graph_rand(Handle *h) {
    cudaError_t e;
    if (h->exec_rand) {
        cudaGraphExecDestroy(h->exec_rand);
        h->exec_rand = nullptr;
    }
    cudaGraph_t g = nullptr;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
    struct G {
        cudaGraph_t g;
        ~G() { cudaGraphDestroy(g); }
    } guard{g};
    cudaGraphConditionalHandle cond;
    if ((e = cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphConditionalHandleCreate");
    RoundArgs a = rand_args(h);
    a.cond = cond;
    a.use_cond = 1;
    cudaGraphNode_t tail = nullptr;
    hm_status st = capture_chain(h, g, capture_rinit, &a, &tail);
    if (st != HM_OK) return st;
    if ((st = add_while_loop(h, g, tail, cond, capture_rround, &a)) != HM_OK) return st;
    if ((e = cudaGraphInstantiate(&h->exec_rand, g, 0)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphInstantiate");
    h->graph_cap_rand = h->cap;
    h->graph_cfg_rand = h->cfg;
    h->graph_noise = h->noise;
    return HM_OK;
}

}  // namespace

hm_status rand_prepare(Handle *h, cudaStream_t s) {
    h->rargmax_grid = (unsigned)(h->sm_count * (h->graph ? fit_per_sm(k_rargmax<true>) : fit_per_sm(k_rargmax<false>)));
    h->rlong_grid = (unsigned)(h->sm_count * (h->graph ? fit_per_sm(k_rlong<true>) : fit_per_sm(k_rlong<false>)));
    h->rpropose_grid = (unsigned)(h->sm_count * fit_per_sm(k_rpropose));
    if (h->vrecR) return HM_OK;
    const uint64_t n = (uint64_t)h->n, m = (uint64_t)h->m;
    h->lq_cap = (uint32_t)(std::min<uint64_t>(n, h->kappa / kLong) + 1);
    hm_status st;
    if ((st = dalloc(&h->vrecR, n, s, "re-randomised vertex records")) != HM_OK ||
        (st = dalloc(&h->vadjE, h->kappa, s, "vertex lists in edge ids")) != HM_OK ||
        (st = dalloc(&h->vadjR, h->kappa, s, "re-randomised vertex lists")) != HM_OK ||
        (st = dalloc(&h->jof, m, s, "inverse edge order")) != HM_OK ||
        (st = dalloc(&h->P2, m, s, "second proposal counters")) != HM_OK ||
        (h->p16 && !h->graph && (st = dalloc(&h->S32, m, s, "edge sizes")) != HM_OK) ||
        (!h->p16 && ((st = dalloc(&h->S64, m, s, "edge sizes")) != HM_OK ||
                     (st = dalloc(&h->W64a, m, s, "proposal counters")) != HM_OK ||
                     (st = dalloc(&h->W64b, m, s, "proposal counters")) != HM_OK)) ||
        (st = dalloc(&h->lq, h->lq_cap, s, "long-list queue")) != HM_OK ||
        (st = dalloc(&h->rbest, n, s, "largest keys of the round")) != HM_OK ||
        (st = dalloc(&h->vchunk, (h->kappa + kFlatW - 1) / kFlatW + 1, s, "flat chunk vertices")) != HM_OK ||
        (h->graph && ((st = dalloc(&h->vnbrE, h->kappa, s, "list endpoints")) != HM_OK ||
                      (st = dalloc(&h->vnbrR, h->kappa, s, "re-randomised list endpoints")) != HM_OK))) {
        free_rand_buffers(h);
        return st;
    }
    if (h->graph && h->kappa)  // the endpoints in list order, from the fixed order's pair lists
        k_pair_endpoints<<<grid_for(h->kappa, kT, h->sm_count, 16), kT, 0, s>>>(h->vpair, h->kappa, h->vnbrE);
    if (m) {
        k_map<<<grid_for(std::max<uint64_t>(m, h->kappa), kT, h->sm_count, 16), kT, 0, s>>>(
            h->order, h->vadj, h->weighted ? h->weights : nullptr, h->m, h->kappa, h->vadjE, h->vadjR, h->jof);
        if (!h->graph)  // graphs count in bytes and need no sizes
            k_size_words<<<grid_for(m, kT, h->sm_count, 16), kT, 0, s>>>(h->order, h->eoffj, h->m, 0, h->S32,
                                                                        h->S64);
        const uint64_t nchunks = (h->kappa + kFlatW - 1) / kFlatW;
        if (nchunks)
            k_vchunk<<<grid_for(nchunks, kT, h->sm_count, 16), kT, 0, s>>>(h->voff, h->n, nchunks, h->vchunk);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            free_rand_buffers(h);
            return cuda_fail(e, "edge id maps");
        }
    }
    return HM_OK;
}

hm_status launch_match_graph_rand(Handle *h, cudaStream_t s) {
    hm_status st = rand_prepare(h, s);
    if (st != HM_OK) return st;
    if (!h->exec_rand || h->graph_cap_rand != h->cap || !(h->graph_cfg_rand == h->cfg) ||
        h->graph_noise != h->noise) {
        if ((st = build_graph_rand(h)) != HM_OK) return st;
    }
    cudaError_t e = cudaGraphLaunch(h->exec_rand, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return HM_OK;
}

hm_status profile_match_rand(Handle *h, cudaStream_t s, double *ms, int64_t *launches, double *round_ms,
                             int32_t max_rounds) {
    hm_status st = rand_prepare(h, s);
    if (st != HM_OK) return st;
    for (int k = 0; k < HM_K_COUNT; ++k) {
        ms[k] = 0;
        launches[k] = 0;
    }
    cudaEvent_t ev[6];
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    struct E {
        cudaEvent_t *ev;
        ~E() {
            for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
        }
    } guard{ev};
    RoundArgs a = rand_args(h);
    float t = 0;
    cudaEventRecord(ev[5], s);
    launch_rinit(h, a, s);
    cudaEventRecord(ev[0], s);
    cudaError_t e = cudaEventSynchronize(ev[0]);
    if (e != cudaSuccess) return cuda_fail(e, "profile init");
    cudaEventElapsedTime(&t, ev[5], ev[0]);
    ms[HM_K_INIT] += t;
    launches[HM_K_INIT] += 1;
    for (int32_t r = 0;; ++r) {
        launch_live_edges(h, a, s, 1);  // untimed: before the round's first event
        launch_rround(h, a, s, ev);
        cudaMemcpyAsync(h->h_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "profile round");
        for (int k = 0; k < 4; ++k) {
            cudaEventElapsedTime(&t, ev[k], k == 0 ? ev[5] : ev[k + 1]);
            ms[HM_K_ARGMAX + k] += t;
            // the argmax step is three kernels here; the round end is part of the kill kernel
            launches[HM_K_ARGMAX + k] += k == 0 ? 3 : (k == 3 ? 0 : 1);
            if (r < max_rounds) round_ms[(int64_t)r * 4 + k] = t;
        }
        if (h->h_st->finished) break;
    }
    cudaEventRecord(h->done, s);
    return HM_OK;
}

void free_rand_buffers(Handle *h) {
    void *bufs[] = {h->vrecR, h->vadjE, h->vadjR, h->jof, h->P2, h->lq, h->rbest, h->vnbrE, h->vnbrR,
                    h->S32, h->S64, h->W64a, h->W64b, h->vchunk};
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, h->cap_stream);
    h->vrecR = nullptr;
    h->vadjE = nullptr;
    h->vadjR = nullptr;
    h->jof = nullptr;
    h->P2 = nullptr;
    h->lq = nullptr;
    h->rbest = nullptr;
    h->S32 = nullptr;
    h->S64 = nullptr;
    h->W64a = nullptr;
    h->W64b = nullptr;
    h->vchunk = nullptr;
    h->vnbrE = nullptr;
    h->vnbrR = nullptr;
    if (h->exec_rand) cudaGraphExecDestroy(h->exec_rand);
    h->exec_rand = nullptr;
}

}  // namespace hm
