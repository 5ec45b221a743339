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
// A round is Alg. 1's three steps with these keys: every vertex takes the
// largest key among its live edges (T[v]), an edge chosen by all of its
// pins joins the matching, and edges with a matched pin die. Two
// formulations compute it, each where its cost is lowest.
//
// Round 1 (every edge live) is vertex-driven. The vertex lists, stored as
// {input edge id e, bits(p_1(e))} pairs (vadjE: round 1's priority of the
// entry's edge, computed once per handle and amplitude, so the scan hashes
// nothing), are read as one flat array (flat_round1) with no random read at
// all; each vertex's largest key goes to rbest. k_rpropose then makes every proposal (the P counter of Alg. 1,
// counted up by input id and packed with the edge's size, so one atomic
// tells whether the count reached |e|), and the win and kill kernels of
// rounds.cu finish the round: the winners' vertices are marked, and every
// entry of their lists is cleared in the m-byte live-flag array.
//
// Rounds 2 on are edge-driven, on a list of the edges still live (records
// {e, bits(base_e), first pin, |e|}, in j order for round 2: erec). After
// round 1 most list entries belong to dead edges (on the power-law bench
// instance 3.7e7 of the 1.78e8 entries of the vertices still active), so a
// vertex-driven round would pay one random live-flag read per dead entry;
// here a round touches only the pins of the edges live in the round before:
//   k_epush: the previous round's live list (round 2: every edge) is
//     filtered - an edge is live while none of its pins is matched (in
//     round 2 of a hypergraph: while the live flag that round 1's kill step
//     maintained is set) - and compacted into this round's list, and every
//     live edge offers key_r(e) to each pin with a 64-bit atomicMax on the
//     vertex's slot of this round's buffer: the slot ends as the key of
//     T[v] (step 1).
//   k_ewin: an edge whose key is in the slot of every pin won (step 2): it
//     joins the matching and its pins are marked matched; the deaths this
//     causes are found by the next round's filter (step 3). It also clears
//     the other buffer whole (a streaming pass: cheaper than a random store
//     per live pin), so that the next round starts from zero slots and a
//     nonzero slot after a round means the vertex was offered a key in it;
//     its last block ends the round.
// Small edges (at most kSmall pins) are handled by one lane, which keeps
// their pins in registers between the test and the offer; larger ones by
// the whole warp, 32 pins at a time. The lists are split into fixed regions
// (those of erec: eregion consecutive records each), a warp owns a region
// at a time, and a region's live records are compacted to the front of the
// same region of the next list with ballots: no counter shared by the whole
// GPU (one such atomic per 32 records serialised the round on a graph).
#include "hm_internal.cuh"

#include <algorithm>
#include <cmath>

namespace hm {
namespace {

constexpr int kT = 256;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kSmall = 8;  // edges with at most this many pins are handled by one lane

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
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

// Round 1's P counter for input edge e, packed with the edge's size: word
// = (|e| << H) | count, H = 16 when no edge has more than 65535 pins (a
// 32-bit word), else H = 32 (a 64-bit word). A proposal adds 1 and gets
// the size back with the old count from the same atomic, so no other read
// is needed to see whether it completed the edge. The words start each
// match as copies of the sizes (k_rinit). A graph's edges all have two
// pins: its counts are 8-bit, four to a 32-bit word, with no size beside
// them (the count an edge reaches is at most 2), so the counters of m edges
// take m bytes and stay in L2.
__device__ __forceinline__ bool propose(const RoundArgs &a, int32_t e) {
    if (a.pairs) {
        const int sh = (e & 3) * 8;
        const uint32_t old = atomicAdd(a.P2 + (e >> 2), 1u << sh);
        return ((old >> sh) & 0xFFu) == 1u;
    }
    if (a.w64) {
        const unsigned long long old = atomicAdd(a.W64 + e, 1ull);
        return (old & 0xFFFFFFFFull) + 1ull == (old >> 32);
    }
    const uint32_t old = atomicAdd(a.P2 + e, 1u);
    return (old & 0xFFFFu) + 1u == (old >> 16);
}

__global__ void __launch_bounds__(kT) k_rinit(RoundArgs a) {
    const int64_t total = a.n > a.m ? a.n : a.m;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < total; i += (int64_t)gridDim.x * kT) {
        if (i < a.m) {
            a.alive[i] = 1;
            if (a.pairs) {  // four 8-bit counts a word
                if (i < (a.m + 3) / 4) a.P2[i] = 0;
            } else if (a.w64) {
                a.W64[i] = __ldg(a.S64 + i);
            } else {
                a.P2[i] = __ldg(a.S32 + i);
            }
            a.inM[i] = 0;
        }
        if (i < a.n) {
            a.vmatch[i] = 0;
            a.rbest[i] = 0;   // round 1 folds list pieces into it with atomicMax
            a.rbest2[i] = 0;  // round 2 offers its keys into it
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        DevState *st = a.st;
        st->round = 1;
        st->parity = 0;
        st->cnt[0] = st->cnt[1] = 0;
        st->nwin = 0;
        st->kdone = 0;
        st->status = HM_OK;
        st->rounds_done = 0;
        st->finished = 0;
        st->fault = 0;
        st->adv = st->kills = st->winpins = st->proposals = 0;
        st->live = st->kpack = st->sdeg = 0;
        st->ledges = st->lpins = 0;
    }
}

constexpr int kFlatC = 32;                // round 1: consecutive entries a lane takes per chunk
constexpr uint64_t kFlatW = 32 * kFlatC;  // round 1: entries per warp chunk
constexpr int kFlatSpan = 192;            // round 1: a chunk's vertex offsets staged in shared memory up to this many

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
__device__ __forceinline__ void flat_round1(const RoundArgs &a, uint32_t *s_off) {
    // list positions are below kappa < 2^32: 32-bit arithmetic throughout
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * (uint32_t)kT + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * (uint32_t)kT) >> 5;
    const uint32_t kappa = (uint32_t)a.kappa;
    const uint32_t nchunks = (uint32_t)((a.kappa + kFlatW - 1) / kFlatW);
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
                // the entry holds bits(p_1(e)): key_1(e) needs no hash here
                const unsigned long long key = ((unsigned long long)(uint32_t)ev[u].y << 32) |
                                               (unsigned long long)(0xFFFFFFFFu - (uint32_t)ev[u].x);
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

// Round 1's scan: one flat pass over every list.
__global__ void __launch_bounds__(kT) k_rflat(RoundArgs a) {
    __shared__ uint32_t s_off[kT / 32][kFlatSpan];
    flat_round1(a, s_off[threadIdx.x >> 5]);
}

// Round 1's proposals: for every vertex with a list (the flat scan left its
// largest key in rbest), T[v] is the edge of that key; the vertex counts
// itself in that edge's P counter, and the count that completes the edge
// makes it a winner. A flat grid-stride loop, two vertices a lane in
// flight. Winners are staged in a per-warp shared buffer and appended to
// the round's list with one atomic per kWinStage of them (a graph has
// millions of winners in round 1: one atomic on the list counter per warp
// step serialised the kernel). The proposers are counted (the vertices
// kept for round 2).
constexpr int kWinStage = 256;

__device__ __forceinline__ void flush_staged(const RoundArgs &a, const int32_t *buf, uint32_t cnt) {
    const int lane = threadIdx.x & 31;
    uint32_t wb = 0;
    if (lane == 0) wb = atomicAdd(&a.st->nwin, cnt);
    wb = __shfl_sync(kFull, wb, 0);
    for (uint32_t x = lane; x < cnt; x += 32) {
        const uint64_t idx = (uint64_t)wb + x;
        if (idx < a.win_cap) a.win[idx] = buf[x];
        else a.st->fault = 2;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kT) k_rpropose(RoundArgs a) {
    __shared__ unsigned long long s_red[kT / 32];
    __shared__ int32_t s_win[kT / 32][kWinStage];
    __shared__ unsigned int s_cnt;
    DevState *st = a.st;
    const unsigned lt = lanemask_lt();
    int32_t *wbuf = s_win[threadIdx.x >> 5];
    uint32_t staged = 0;  // uniform in the warp
    const uint64_t stride = (uint64_t)gridDim.x * kT;
    unsigned long long props = 0;
    for (uint64_t v0 = blockIdx.x * (uint64_t)kT * 2 + threadIdx.x;; v0 += 2 * stride) {
        if (v0 - threadIdx.x >= (uint64_t)a.n) break;  // uniform in the block: no vertex left for it
        unsigned long long best[2];
        bool w[2] = {false, false};
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const uint64_t v = v0 + (uint64_t)u * kT;
            best[u] = v < (uint64_t)a.n ? a.rbest[v] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (best[u] != 0) {
                const uint64_t v = v0 + (uint64_t)u * kT;
                const int32_t e = edge_of_key(best[u]);  // T[v], input id
                reinterpret_cast<int2 *>(a.vrec + v)[0] = make_int2(e, 0);
                w[u] = propose(a, e);
                ++props;
            }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const unsigned wm = __ballot_sync(kFull, w[u]);
            if (staged + __popc(wm) > (uint32_t)kWinStage) {  // uniform
                flush_staged(a, wbuf, staged);
                staged = 0;
            }
            if (w[u]) wbuf[staged + __popc(wm & lt)] = __ldg(a.jof + edge_of_key(best[u]));  // listed by relabelled id
            staged += __popc(wm);
            __syncwarp();
        }
    }
    if (staged) flush_staged(a, wbuf, staged);
    block_add_u64(props, s_red, &st->proposals);
    // the proposers are the vertices kept for round 2 (the round end reads
    // cnt[1]): one 32-bit atomic a block
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    if (props) atomicAdd(&s_cnt, (unsigned int)props);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(&st->cnt[1], s_cnt);
}

// Profiled replay only, between round 1's timed spans: the sum of the
// degrees of the vertices kept for round 2 (every vertex with a list, the
// ones the flat scan gave a key), into the round's counter.
__global__ void __launch_bounds__(kT) k_rdeg1(RoundArgs a) {
    __shared__ unsigned long long s_red[kT / 32];
    unsigned long long sum = 0;
    for (int64_t v = blockIdx.x * (int64_t)kT + threadIdx.x; v < a.n; v += (int64_t)gridDim.x * kT)
        if (a.rbest[v] != 0) sum += (unsigned long long)(a.voff[v + 1] - a.voff[v]);
    block_add_u64(sum, s_red, &a.st->sdeg);
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
__global__ void __launch_bounds__(kT) k_size_words(const int32_t *order, const int64_t *eoffj, int64_t m,
                                                   uint32_t *S32, unsigned long long *S64) {
    for (int64_t j = blockIdx.x * (int64_t)kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT) {
        const int32_t e = __ldg(order + j);
        const uint64_t size = (uint64_t)(eoffj[j + 1] - eoffj[j]);
        if (S32) S32[e] = (uint32_t)size << 16;
        else S64[e] = (unsigned long long)size << 32;
    }
}

// ---------------------------------------------------------------- edge rounds

// Offers key to a vertex slot. In a hypergraph the slot is read first: it
// only rises during the pass, so a read that finds it at or above the key
// makes the atomic unnecessary (a stale read can only be lower: then the
// atomic runs and decides). In a random order about ln d of the d offers to
// a vertex raise its slot, and a random L2 load costs less than a 64-bit
// atomic: round 2 of the power-law instance 1.18 -> 0.68 ms. A graph's
// vertices get a few offers each, and there the extra dependent load cost
// more than it saved (2.69 -> 3.10 ms a match).
template <bool kPairs>
__device__ __forceinline__ void offer(unsigned long long *slot, unsigned long long key) {
    if (kPairs || __ldcg(slot) < key) atomicMax(slot, key);
}

// An edge record is {input id, bits(base priority), first pin, size}, or,
// for an edge of two pins, {input id, bits(base priority), pin, pin | 2^31}
// (the pins in place: a negative last word; vertex ids are below 2^31).
// A graph's records all have their pins in place (kPairs: known at compile
// time, which keeps the other form out of its kernels).
template <bool kPairs>
__device__ __forceinline__ uint32_t record_size(const int4 &rec) {
    return (kPairs || rec.w < 0) ? 2u : (uint32_t)rec.w;
}

// The pins of a small edge (size <= kSmall) in registers: in the record,
// or loaded from the edge CSR.
template <bool kPairs>
__device__ __forceinline__ void record_pins(const int32_t *__restrict__ pinsj, const int4 &rec, uint32_t size,
                                            int32_t (&pv)[kSmall]) {
    const bool in_place = kPairs || rec.w < 0;
#pragma unroll
    for (int k = 0; k < kSmall; ++k) {
        if (in_place) pv[k] = k == 0 ? rec.z : (k == 1 ? (rec.w & 0x7FFFFFFF) : 0);
        else pv[k] = (uint32_t)k < size ? __ldg(pinsj + (uint32_t)rec.z + k) : 0;
    }
}

// Step 1 of round r >= 2 (see the file comment). Past the round cap the
// kernel only counts the live edges (the round end decides between done and
// HM_ETIMEOUT) and writes nothing. The next record of a region is loaded
// while the current one is worked on.
template <bool kPairs>
__global__ void __launch_bounds__(kT) k_epush(RoundArgs a) {
    __shared__ unsigned long long s_red[kT / 32];
    DevState *st = a.st;
    const int r = st->round;
    const bool over = r > a.cap;
    const bool first = r == 2;
    const bool by_flag = first && !kPairs;
    const int4 *__restrict__ in = first ? a.erec : a.elist[(r - 1) & 1];
    const uint32_t *cnt_in = a.ecnt + (size_t)((r - 1) & 1) * a.eregions;
    int4 *__restrict__ out = a.elist[r & 1];
    uint32_t *cnt_out = a.ecnt + (size_t)(r & 1) * a.eregions;
    unsigned long long *cur = (r & 1) ? a.rbest : a.rbest2;
    const uint64_t cr = round_counter_base(a.noise_s0, r);
    const float scale = a.noise_scale;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const uint32_t warp = (blockIdx.x * (uint32_t)kT + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * (uint32_t)kT) >> 5;
    unsigned long long nedges = 0, npins = 0, nscan = 0, ndead = 0;
    for (uint32_t g = warp; g < a.eregions; g += nwarps) {  // uniform in the warp
        const uint64_t base = (uint64_t)g * a.eregion;
        uint32_t cnt;
        if (first) {
            const int64_t left = a.m - (int64_t)base;
            cnt = left <= 0 ? 0u : (uint32_t)(left < (int64_t)a.eregion ? left : (int64_t)a.eregion);
        } else {
            cnt = cnt_in[g];
        }
        uint32_t kept = 0;
        int4 nrec = lane < cnt ? in[base + lane] : make_int4(0, 0, 0, 0);
        for (uint32_t i0 = 0; i0 < cnt; i0 += 32) {
            const uint32_t i = i0 + lane;
            const bool ok = i < cnt;
            const int4 rec = nrec;
            if (i + 32 < cnt) nrec = in[base + i + 32];
            const uint32_t start = (uint32_t)rec.z, size = ok ? record_size<kPairs>(rec) : 0u;
            const bool big = size > (uint32_t)kSmall;
            bool live = ok;
            int32_t pv[kSmall];
            if (by_flag) {
                live = ok && a.alive[rec.x] != 0;
                if (live && !big) record_pins<kPairs>(a.pinsj, rec, size, pv);
                if (live) nscan += size;
            } else {
                if (ok && !big) {
                    record_pins<kPairs>(a.pinsj, rec, size, pv);
                    bool any = false;
#pragma unroll
                    for (int k = 0; k < kSmall; ++k)
                        if ((uint32_t)k < size) any |= a.vmatch[pv[k]] != 0;
                    live = !any;
                }
                nscan += size;
                unsigned bm = __ballot_sync(kFull, ok && big);
                while (bm) {  // the warp tests each big edge's pins together
                    const int k = __ffs(bm) - 1;
                    bm &= bm - 1;
                    const uint32_t bs = __shfl_sync(kFull, start, k), bn = __shfl_sync(kFull, size, k);
                    bool any = false;
                    for (uint32_t p = lane; p < bn; p += 32) any |= a.vmatch[__ldg(a.pinsj + bs + p)] != 0;
                    const bool dead = __any_sync(kFull, any);
                    if (lane == k) live = !dead;
                }
                if (ok && !live) ndead += size;
            }
            if (live) {
                nedges += 1;
                npins += size;
            }
            if (over) continue;  // uniform
            // this round's live list: compacted to the front of the same region
            const unsigned lm = __ballot_sync(kFull, live);
            if (live) out[base + kept + __popc(lm & lt)] = rec;
            kept += __popc(lm);
            // every live edge offers its key to each of its pins
            const unsigned long long key = scan_key(cr, scale, (uint32_t)rec.x, __int_as_float(rec.y));
            if (live && !big) {
#pragma unroll
                for (int k = 0; k < kSmall; ++k)
                    if ((uint32_t)k < size) offer<kPairs>(cur + pv[k], key);
            }
            unsigned bm = __ballot_sync(kFull, live && big);
            while (bm) {
                const int k = __ffs(bm) - 1;
                bm &= bm - 1;
                const uint32_t bs = __shfl_sync(kFull, start, k), bn = __shfl_sync(kFull, size, k);
                const unsigned long long kk = __shfl_sync(kFull, key, k);
                for (uint32_t p = lane; p < bn; p += 32) offer<kPairs>(cur + __ldg(a.pinsj + bs + p), kk);
            }
        }
        if (lane == 0 && !over) cnt_out[g] = kept;
    }
    block_add_u64(nedges, s_red, &st->ledges);
    block_add_u64(npins, s_red, &st->lpins);
    block_add_u64(nscan, s_red, &st->adv);
    block_add_u64(ndead, s_red, &st->kills);
}

// The end of an edge round (one thread, after every block of k_ewin has
// finished): records the round and decides whether another one runs. A
// round with no live edge did not happen (the one before ended the
// matching); past the cap, a live edge means HM_ETIMEOUT.
__device__ void eround_end(const RoundArgs &a) {
    DevState *st = a.st;
    const int r = st->round;
    const uint32_t nw = st->nwin;
    const unsigned long long ledges = st->ledges;
    int cont = 0;
    if (r > a.cap) {
        st->rounds_done = r - 1;
        if (ledges > 0) st->status = HM_ETIMEOUT;
    } else {
        // proposals: the keys offered (one per live pin). The vertices
        // offered a key (active, next) and their degrees are counted by the
        // profiled replay (k_ekept), which also records the live edges and
        // pins, as in round 1
        const bool prof = a.profiled != 0;
        write_stats_row(a, r, 0, nw, 0u, st->adv, st->lpins, st->winpins, st->kills, 0u, st->lpins, 0ull,
                        prof ? ledges : 0ull, prof ? st->lpins : 0ull);
        if (st->fault) {
            st->status = HM_ECUDA;
        } else if (ledges == 0) {
            st->rounds_done = r - 1;
        } else if (nw == 0) {  // the live edge with the largest key always wins: inconsistent input
            st->rounds_done = r;
            st->status = HM_EINVAL;
        } else {
            st->rounds_done = r;
            cont = ledges > nw;  // the edges that did not win may still be live
        }
    }
    st->nwin = 0;
    st->kdone = 0;
    st->adv = st->kills = st->winpins = st->proposals = 0;
    st->live = st->kpack = st->sdeg = 0;
    st->ledges = st->lpins = 0;
    if (cont) st->round = r + 1;
    else st->finished = 1;
    if (a.use_cond) cudaGraphSetConditional(a.cond, cont ? 1u : 0u);
}

// Step 2 of round r >= 2: an edge wins when every pin's slot holds its key;
// it joins the matching and marks its pins matched. The other buffer is
// cleared on the way. The block that finishes last (a ticket counter) ends
// the round.
template <bool kPairs>
__global__ void __launch_bounds__(kT) k_ewin(RoundArgs a) {
    __shared__ unsigned long long s_red[kT / 32];
    __shared__ int s_last;
    DevState *st = a.st;
    const int r = st->round;
    unsigned long long nw = 0, wp = 0;
    if (r <= a.cap) {  // uniform
        const int4 *__restrict__ in = a.elist[r & 1];
        const uint32_t *cnt_in = a.ecnt + (size_t)(r & 1) * a.eregions;
        const unsigned long long *cur = (r & 1) ? a.rbest : a.rbest2;
        unsigned long long *other = (r & 1) ? a.rbest2 : a.rbest;
        // the other buffer must be zero at every vertex the next round
        // offers a key to, and nonzero only there afterwards (the vertex
        // state reads it): cleared whole, one streaming pass of 8n bytes
        // (a round with no live edge ends the matching and keeps it)
        if (st->lpins > 0) {
            ulonglong2 *o2 = reinterpret_cast<ulonglong2 *>(other);  // cudaMalloc'd: 16-byte aligned
            const uint64_t n2 = (uint64_t)a.n / 2;
            for (uint64_t x = blockIdx.x * (uint64_t)kT + threadIdx.x; x < n2; x += (uint64_t)gridDim.x * kT)
                o2[x] = make_ulonglong2(0ull, 0ull);
            if (blockIdx.x == 0 && threadIdx.x == 0 && (a.n & 1)) other[a.n - 1] = 0;
        }
        const uint64_t cr = round_counter_base(a.noise_s0, r);
        const float scale = a.noise_scale;
        const int lane = threadIdx.x & 31;
        const uint32_t warp = (blockIdx.x * (uint32_t)kT + threadIdx.x) >> 5;
        const uint32_t nwarps = (gridDim.x * (uint32_t)kT) >> 5;
        for (uint32_t g = warp; g < a.eregions; g += nwarps) {  // uniform in the warp
            const uint32_t cnt = cnt_in[g];
            for (uint32_t i0 = 0; i0 < cnt; i0 += 32) {
                const uint32_t i = i0 + lane;
                const bool ok = i < cnt;
                const int4 rec = ok ? in[(uint64_t)g * a.eregion + i] : make_int4(0, 0, 0, 0);
                const uint32_t start = (uint32_t)rec.z, size = ok ? record_size<kPairs>(rec) : 0u;
                const bool big = size > (uint32_t)kSmall;
                const unsigned long long key = scan_key(cr, scale, (uint32_t)rec.x, __int_as_float(rec.y));
                bool win = ok;
                int32_t pv[kSmall];
                if (ok && !big) {
                    record_pins<kPairs>(a.pinsj, rec, size, pv);
#pragma unroll
                    for (int k = 0; k < kSmall; ++k)
                        if ((uint32_t)k < size) {
                            win &= cur[pv[k]] == key;
                        }
                }
                unsigned bm = __ballot_sync(kFull, ok && big);
                while (bm) {  // the warp tests each big edge's pins together
                    const int k = __ffs(bm) - 1;
                    bm &= bm - 1;
                    const uint32_t bs = __shfl_sync(kFull, start, k), bn = __shfl_sync(kFull, size, k);
                    const unsigned long long kk = __shfl_sync(kFull, key, k);
                    bool miss = false;
                    for (uint32_t p = lane; p < bn; p += 32) {
                        const int32_t v = __ldg(a.pinsj + bs + p);
                        miss |= cur[v] != kk;
                    }
                    const bool lost = __any_sync(kFull, miss);
                    if (lane == k) win = !lost;
                }
                if (win) {
                    a.inM[rec.x] = 1;
                    if (a.wround) a.wround[rec.x] = r;
                    nw += 1;
                    wp += size;
                    if (!big) {
#pragma unroll
                        for (int k = 0; k < kSmall; ++k)
                            if ((uint32_t)k < size) a.vmatch[pv[k]] = 1;
                    }
                }
                bm = __ballot_sync(kFull, win && big);
                while (bm) {  // a big winner's pins, marked by the warp
                    const int k = __ffs(bm) - 1;
                    bm &= bm - 1;
                    const uint32_t bs = __shfl_sync(kFull, start, k), bn = __shfl_sync(kFull, size, k);
                    for (uint32_t p = lane; p < bn; p += 32) a.vmatch[__ldg(a.pinsj + bs + p)] = 1;
                }
            }
        }
    }
    {
        uint32_t x = (uint32_t)nw;  // winners: one atomic per warp
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(kFull, x, d);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&st->nwin, x);
    }
    block_add_u64(wp, s_red, &st->winpins);
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&st->kdone, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        eround_end(a);
    }
}

// Profiled edge rounds only, after round r's k_ewin: the vertices offered a
// key in round r (the pins of its live edges: the vertices active at its
// start, unmatched with a live edge), counted as both the active and the
// kept vertices, and the sum of their degrees, added to round r's stats row
// (zero there until now).
__global__ void __launch_bounds__(kT) k_ekept(RoundArgs a, int r) {
    __shared__ unsigned long long s_red[kT / 32];
    const unsigned long long *cur = (r & 1) ? a.rbest : a.rbest2;
    unsigned long long kept = 0, deg = 0;
    for (int64_t v = blockIdx.x * (int64_t)kT + threadIdx.x; v < a.n; v += (int64_t)gridDim.x * kT) {
        if (cur[v] == 0) continue;
        kept += 1;
        deg += (unsigned long long)(a.voff[v + 1] - a.voff[v]);
    }
    if (r - 1 < kStatRounds) {
        int64_t *row = a.stats + (int64_t)(r - 1) * HM_STATS_COLS;
        block_add_u64(kept, s_red, reinterpret_cast<unsigned long long *>(row + HM_STAT_ACTIVE));
        block_add_u64(kept, s_red, reinterpret_cast<unsigned long long *>(row + HM_STAT_NEXT));
        block_add_u64(deg, s_red, reinterpret_cast<unsigned long long *>(row + HM_STAT_DEG));
    }
}

// The per-vertex state after the last round run: HM_VERTEX_MATCHED, T[v]
// (input id) or HM_VERTEX_NONE. After round 1 it is the round-1 record;
// after an edge round R, T[v] is the edge of v's slot in round R's buffer
// (zero: v was offered no key in round R).
__global__ void __launch_bounds__(kT) k_rvertex_state(RoundArgs a, int32_t *out) {
    const int R = a.st->rounds_done;
    const unsigned long long *buf = (R & 1) ? a.rbest : a.rbest2;
    for (int64_t v = blockIdx.x * (int64_t)kT + threadIdx.x; v < a.n; v += (int64_t)gridDim.x * kT) {
        const int32_t t = a.vrec[v].x;
        int32_t s;
        if (a.vmatch[v] || t == kCurMatched) {
            s = HM_VERTEX_MATCHED;
        } else if (R <= 1) {
            s = t >= 0 ? t : HM_VERTEX_NONE;
        } else {
            const unsigned long long k = buf[v];
            s = k != 0 ? edge_of_key(k) : HM_VERTEX_NONE;
        }
        out[v] = s;
    }
}

// The round-1 vertex records {T[v], 0, list start, list length}, built once
// per handle: a match rewrites T[v] of every vertex with a list in round 1
// (k_rpropose) and of the winners' pins (k_win) and nothing else, and a
// vertex without a list keeps T = none.
__global__ void __launch_bounds__(kT) k_rrec(const int64_t *voff, int64_t n, int4 *vrec) {
    for (int64_t v = blockIdx.x * (int64_t)kT + threadIdx.x; v < n; v += (int64_t)gridDim.x * kT) {
        const int64_t b = voff[v], e = voff[v + 1];
        vrec[v] = make_int4(kCurNone, 0, (int32_t)(uint32_t)b, (int32_t)(uint32_t)(e - b));
    }
}

// Every edge's record (record_size), in j order: the input of round 2. An
// edge of two pins (every edge of a graph) carries them, so the edge
// rounds read no pins for it.
__global__ void __launch_bounds__(kT) k_erec(const int32_t *order, const int64_t *eoffj, const int32_t *pinsj,
                                           const float *w, int64_t m, int graph, int4 *erec) {
    for (int64_t j = blockIdx.x * (int64_t)kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT) {
        const int32_t e = __ldg(order + j);
        const int32_t wb = __float_as_int(w ? __ldg(w + e) : 1.0f);
        const int64_t b = graph ? 2 * j : eoffj[j];
        const int64_t size = graph ? 2 : eoffj[j + 1] - b;
        if (size == 2)
            erec[j] = make_int4(e, wb, __ldg(pinsj + b), (int32_t)(0x80000000u | (uint32_t)__ldg(pinsj + b + 1)));
        else
            erec[j] = make_int4(e, wb, (int32_t)(uint32_t)b, (int32_t)size);
    }
}

// The inverse of the edge order (built once per handle).
__global__ void __launch_bounds__(kT) k_jof(const int32_t *order, int64_t m, int32_t *jof) {
    for (int64_t j = blockIdx.x * (int64_t)kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT)
        jof[order[j]] = (int32_t)j;
}

// Round 1's lists as {input edge id e, bits(p_1(e))}: the round-1 priority
// of every entry's edge, computed with scan_key's arithmetic (so round 1's
// keys are bit for bit those the hash gives), once per handle and noise
// amplitude. Round 1 then reads its keys instead of hashing every list
// entry (an edge appears in the lists of all its pins).
__global__ void __launch_bounds__(kT) k_r1keys(const int32_t *order, const int32_t *vadj, const float *w,
                                             uint64_t kappa, uint64_t s0, float scale, int2 *vadjE) {
    const uint64_t cr = round_counter_base(s0, 1);
    for (uint64_t i = blockIdx.x * (uint64_t)kT + threadIdx.x; i < kappa; i += (uint64_t)gridDim.x * kT) {
        const int32_t e = __ldg(order + __ldg(vadj + i));
        const unsigned long long key = scan_key(cr, scale, (uint32_t)e, w ? __ldg(w + e) : 1.0f);
        vadjE[i] = make_int2(e, (int32_t)(uint32_t)(key >> 32));
    }
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
    a.pairs = h->graph ? 1 : 0;  // graphs: round 1 sets matched flags and needs no kill
    a.vmatch = h->graph ? h->vmatch : h->rmatch;
    a.vadj = reinterpret_cast<const int32_t *>(h->vadjE);  // round 1's kill step: every second word
    a.vadjE = h->vadjE;
    a.noise_scale = h->noise * (1.0f / 16777216.0f);
    a.noise_s0 = splitmix64_first(h->seed);
    a.jof = h->jof;
    a.P2 = h->P2;
    a.t_input = 1;
    a.w64 = h->p16 ? 0 : 1;
    a.S32 = h->S32;
    a.S64 = h->S64;
    a.W64 = h->W64;
    a.vchunk = h->vchunk;
    a.kappa = h->kappa;
    a.rbest = h->rbest;
    a.rbest2 = h->rbest2;
    a.erec = h->erec;
    a.elist[0] = h->elist0;
    a.elist[1] = h->elist1;
    a.ecnt = h->ecnt;
    a.eregions = h->eregions;
    a.eregion = h->eregion;
    a.erounds = 1;
    a.profiled = 0;
    return a;
}

unsigned rinit_grid(const Handle *h) {
    return grid_for((uint64_t)std::max(h->n, h->m), kT, h->sm_count, 16);
}

// Round 1 (vertex-driven; the kill kernel's last block ends it). ev (or
// null): the profiled replay's events, as in the fixed order's rounds.
void launch_round1(const Handle *h, const RoundArgs &a, cudaStream_t s, cudaEvent_t *ev) {
    if (ev) cudaEventRecord(ev[0], s);
    k_rflat<<<h->rflat_grid, kT, 0, s>>>(a);
    k_rpropose<<<h->rpropose_grid, kT, 0, s>>>(a);
    if (ev) {  // the end of the argmax span, then the untimed degree count
        cudaEventRecord(ev[5], s);
        k_rdeg1<<<grid_for((uint64_t)h->n, kT, h->sm_count, 8), kT, 0, s>>>(a);
    }
    launch_win_kill_end(h, a, s, ev, 2);
}

// An edge round (round 2 on): the offers, then the win test and the round end.
void launch_eround(const Handle *h, const RoundArgs &a, cudaStream_t s, cudaEvent_t *ev) {
    if (ev) cudaEventRecord(ev[0], s);
    if (a.pairs) k_epush<true><<<h->epush_grid, kT, 0, s>>>(a);
    else k_epush<false><<<h->epush_grid, kT, 0, s>>>(a);
    if (ev) {
        cudaEventRecord(ev[5], s);
        cudaEventRecord(ev[1], s);
    }
    if (a.pairs) k_ewin<true><<<h->ewin_grid, kT, 0, s>>>(a);
    else k_ewin<false><<<h->ewin_grid, kT, 0, s>>>(a);
    if (ev) {  // no kill kernel (the next round's filter finds the deaths); the round end is part of k_ewin
        cudaEventRecord(ev[2], s);
        cudaEventRecord(ev[3], s);
        cudaEventRecord(ev[4], s);
    }
}

void capture_rfirst(Handle *h, cudaStream_t s, void *ctx) {
    const RoundArgs &a = *static_cast<const RoundArgs *>(ctx);
    k_rinit<<<rinit_grid(h), kT, 0, s>>>(a);
    launch_round1(h, a, s, nullptr);
}

void capture_eround(Handle *h, cudaStream_t s, void *ctx) {
    launch_eround(h, *static_cast<const RoundArgs *>(ctx), s, nullptr);
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
    hm_status st = capture_chain(h, g, capture_rfirst, &a, &tail);
    if (st != HM_OK) return st;
    if ((st = add_while_loop(h, g, tail, cond, capture_eround, &a)) != HM_OK) return st;
    if ((e = cudaGraphInstantiate(&h->exec_rand, g, 0)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphInstantiate");
    h->graph_cap_rand = h->cap;
    h->graph_cfg_rand = h->cfg;
    h->graph_noise = h->noise;
    return HM_OK;
}

}  // namespace

namespace {

// The mode's buffers and the maps built once per handle.
hm_status alloc_rand(Handle *h, cudaStream_t s) {
    const uint64_t n = (uint64_t)h->n, m = (uint64_t)h->m;
    // regions of the edge lists: four per warp of the offer kernel's grid,
    // whole 32-record steps
    h->eregions = h->epush_grid * (kT / 32) * 4;
    h->eregion = (uint32_t)std::max<uint64_t>(32, (m + h->eregions - 1) / h->eregions);
    h->eregion = (h->eregion + 31) / 32 * 32;
    hm_status st;
    if ((st = dalloc(&h->vrecR, n, s, "re-randomised vertex records")) != HM_OK ||
        (st = dalloc(&h->vadjE, h->kappa, s, "vertex lists in edge ids")) != HM_OK ||
        (st = dalloc(&h->jof, m, s, "inverse edge order")) != HM_OK ||
        (st = dalloc(&h->P2, m, s, "proposal counters")) != HM_OK ||
        (h->p16 && !h->graph && (st = dalloc(&h->S32, m, s, "edge sizes")) != HM_OK) ||
        (!h->p16 && ((st = dalloc(&h->S64, m, s, "edge sizes")) != HM_OK ||
                     (st = dalloc(&h->W64, m, s, "proposal counters")) != HM_OK)) ||
        (st = dalloc(&h->rbest, n, s, "largest keys (odd rounds)")) != HM_OK ||
        (st = dalloc(&h->rbest2, n, s, "largest keys (even rounds)")) != HM_OK ||
        (st = dalloc(&h->vchunk, (h->kappa + kFlatW - 1) / kFlatW + 1, s, "flat chunk vertices")) != HM_OK ||
        (st = dalloc(&h->erec, m, s, "edge records")) != HM_OK ||
        (st = dalloc(&h->elist0, m, s, "live edge list")) != HM_OK ||
        (st = dalloc(&h->elist1, m, s, "live edge list")) != HM_OK ||
        (st = dalloc(&h->ecnt, 2 * (uint64_t)h->eregions, s, "live edge list regions")) != HM_OK ||
        (!h->graph && (st = dalloc(&h->rmatch, n, s, "matched flags")) != HM_OK)) {
        free_rand_buffers(h);
        return st;
    }
    if (n)
        k_rrec<<<grid_for(n, kT, h->sm_count, 16), kT, 0, s>>>(h->voff, h->n, h->vrecR);
    if (m) {
        const float *w = h->weighted ? h->weights : nullptr;
        k_jof<<<grid_for(m, kT, h->sm_count, 16), kT, 0, s>>>(h->order, h->m, h->jof);
        k_erec<<<grid_for(m, kT, h->sm_count, 16), kT, 0, s>>>(h->order, h->eoffj, h->pinsj, w, h->m,
                                                               h->graph ? 1 : 0, h->erec);
        if (!h->graph)  // graphs count in bytes and need no sizes
            k_size_words<<<grid_for(m, kT, h->sm_count, 16), kT, 0, s>>>(h->order, h->eoffj, h->m, h->S32, h->S64);
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

}  // namespace

hm_status rand_prepare(Handle *h, cudaStream_t s) {
    h->rflat_grid = (unsigned)(h->sm_count * fit_per_sm(k_rflat));
    h->rpropose_grid = (unsigned)(h->sm_count * fit_per_sm(k_rpropose));
    h->epush_grid = (unsigned)(h->sm_count * (h->graph ? fit_per_sm(k_epush<true>) : fit_per_sm(k_epush<false>)));
    h->ewin_grid = (unsigned)(h->sm_count * (h->graph ? fit_per_sm(k_ewin<true>) : fit_per_sm(k_ewin<false>)));
    hm_status st;
    if (!h->vrecR && (st = alloc_rand(h, s)) != HM_OK) return st;
    if (h->r1_noise != h->noise && h->kappa) {  // round 1's keys for this amplitude
        k_r1keys<<<grid_for(h->kappa, kT, h->sm_count, 16), kT, 0, s>>>(
            h->order, h->vadj, h->weighted ? h->weights : nullptr, h->kappa, splitmix64_first(h->seed),
            h->noise * (1.0f / 16777216.0f), h->vadjE);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "round-1 keys");
    }
    h->r1_noise = h->noise;
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

cudaError_t launch_rand_vertex_state(const Handle *h, int32_t *out_dev, cudaStream_t s) {
    const RoundArgs a = rand_args(h);
    k_rvertex_state<<<grid_for((uint64_t)h->n, kT, h->sm_count, 16), kT, 0, s>>>(a, out_dev);
    return cudaGetLastError();
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
    k_rinit<<<rinit_grid(h), kT, 0, s>>>(a);
    cudaEventRecord(ev[0], s);
    cudaError_t e = cudaEventSynchronize(ev[0]);
    if (e != cudaSuccess) return cuda_fail(e, "profile init");
    cudaEventElapsedTime(&t, ev[5], ev[0]);
    ms[HM_K_INIT] += t;
    launches[HM_K_INIT] += 1;
    a.profiled = 1;  // the edge rounds record their live edges and pins
    for (int32_t r = 0;; ++r) {
        // per kernel class: launches of round 1 (scan, proposals | win | kill with the round
        // end | -) and of an edge round (offers | win test with the round end | - | -)
        static const int kLaunches[2][4] = {{2, 1, 1, 0}, {1, 1, 0, 0}};
        const int edge = r > 0;
        if (!edge) {
            launch_live_edges(h, a, s, 1);  // untimed: before the round's first event
            launch_round1(h, a, s, ev);
        } else {
            launch_eround(h, a, s, ev);
            k_ekept<<<grid_for((uint64_t)h->n, kT, h->sm_count, 8), kT, 0, s>>>(a, r + 1);  // untimed
        }
        cudaMemcpyAsync(h->h_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "profile round");
        for (int k = 0; k < 4; ++k) {
            cudaEventElapsedTime(&t, ev[k], k == 0 ? ev[5] : ev[k + 1]);
            ms[HM_K_ARGMAX + k] += t;
            launches[HM_K_ARGMAX + k] += kLaunches[edge][k];
            if (r < max_rounds) round_ms[(int64_t)r * 4 + k] = t;
        }
        if (h->h_st->finished) break;
    }
    cudaEventRecord(h->done, s);
    return HM_OK;
}

void free_rand_buffers(Handle *h) {
    void *bufs[] = {h->vrecR, h->vadjE, h->jof, h->P2, h->rbest, h->rbest2, h->S32, h->S64, h->W64,
                    h->vchunk, h->erec, h->elist0, h->elist1, h->ecnt, h->rmatch};
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, h->cap_stream);
    h->vrecR = nullptr;
    h->vadjE = nullptr;
    h->jof = nullptr;
    h->P2 = nullptr;
    h->rbest = nullptr;
    h->rbest2 = nullptr;
    h->S32 = nullptr;
    h->S64 = nullptr;
    h->W64 = nullptr;
    h->vchunk = nullptr;
    h->erec = nullptr;
    h->elist0 = nullptr;
    h->elist1 = nullptr;
    h->ecnt = nullptr;
    h->rmatch = nullptr;
    h->r1_noise = -1.f;
    if (h->exec_rand) cudaGraphExecDestroy(h->exec_rand);
    h->exec_rand = nullptr;
}

}  // namespace hm
