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
//     one concatenated sequence, kU steps of 32 entries at a time (all their
//     loads in flight together; segmented maximum and ballot compaction),
//     so short and medium lists keep every lane busy;
//   - longer lists: queued with their chunk count (one 64-bit atomic hands
//     out the queue slot and the first chunk); k_rlong scans the chunks of
//     kChunk entries with one warp each and combines them per list with a
//     64-bit atomicMax; k_rfin turns each list's maximum into the vertex's
//     proposal. Long lists are not compacted: they are scanned from vadjE,
//     and their part of vadjR (read by the kill step) is copied once when
//     the handle first runs this mode and never written.
// Proposals use the P counter of Alg. 1 counted up and double-buffered by
// round parity: a vertex adds 1 to P_r[T[v]], the edge wins when the count
// reaches |e|, and the vertex clears the entry it counted in the previous
// round in the other buffer, which the next round reuses. Every vertex that
// proposed a still-live edge is active in the next round and clears it;
// stale counts are left only on dead edges, which nobody proposes again.
// The clear is a plain store: all vertices of a large edge clear the same
// word, and same-address stores cost far less than same-address atomics
// (an undo by atomic add measured 5-30 % slower per round). T[v] and the
// winner list hold relabelled ids j.
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
constexpr uint32_t kSeqMax = 64;   // graphs, round 1: tiles whose lists are all this short go one list per lane
constexpr int kU = 4;              // 32-entry steps with loads in flight together

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

// key_r(e) of input edge e whose base priority is `base`. The product and
// the sum are rounded separately (no fused multiply-add), as the
// definition's float32 operations are.
__device__ __forceinline__ unsigned long long round_key_of(uint64_t s0, float scale, int r, uint32_t e, float base) {
    const uint64_t x = splitmix64_at(s0, ((uint64_t)(uint32_t)r << 32) + e + 1u);
    const float u = __uint2float_rn((uint32_t)(x >> 40));
    const float p = __fadd_rn(base, __fmul_rn(u, scale));
    return ((unsigned long long)__float_as_uint(p) << 32) | (unsigned long long)(0xFFFFFFFFu - e);
}

__device__ __forceinline__ unsigned long long round_key(const RoundArgs &a, int r, uint32_t e, float base) {
    return round_key_of(a.noise_s0, a.noise_scale, r, e, base);
}

// Round 1 of a graph, a tile whose lists are all short: each lane takes the
// largest key of its own list, read from the immutable lists (every entry
// is live in round 1, and nothing is written). Kept out of line so that the
// tile path of k_rargmax keeps its own code.
__device__ __noinline__ unsigned long long first_round_max(const int2 *vadjE, int64_t lb, uint32_t len, uint64_t s0,
                                                           float scale) {
    unsigned long long best = 0;
    for (uint32_t i = 0; i < len; ++i) {
        const int2 ev = __ldg(vadjE + lb + i);
        const unsigned long long key = round_key_of(s0, scale, 1, (uint32_t)ev.x, __int_as_float(ev.y));
        if (key > best) best = key;
    }
    return best;
}

__device__ __forceinline__ int32_t edge_of_key(unsigned long long k) {
    return (int32_t)(0xFFFFFFFFu - (uint32_t)k);
}

// Proposal of a vertex for edge j (relabelled id) in round r: counts in the
// round's buffer; returns whether it completed the count (j wins).
__device__ __forceinline__ bool propose(const RoundArgs &a, uint32_t *Pc, int32_t j) {
    const uint32_t size = a.graph ? 2u : (uint32_t)(a.eoffj[j + 1] - a.eoffj[j]);
    return atomicAdd(Pc + j, 1u) + 1u == size;
}

// Appends the winners of a warp (lanes with w set, edge nb) to the list.
__device__ __forceinline__ void append_winners(const RoundArgs &a, bool w, int32_t nb) {
    const int lane = threadIdx.x & 31;
    const unsigned wm = __ballot_sync(kFull, w);
    if (!wm) return;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&a.st->nwin, (uint32_t)__popc(wm));
    base = __shfl_sync(kFull, base, 0);
    if (w) {
        const uint64_t idx = (uint64_t)base + __popc(wm & lanemask_lt());
        if (idx < a.win_cap) a.win[idx] = nb;
        else a.st->fault = 2;
    }
}

__global__ void __launch_bounds__(kT) k_rinit(RoundArgs a) {
    const int64_t total = a.n > a.m ? a.n : a.m;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < total; i += (int64_t)gridDim.x * kT) {
        if (i < a.m) {
            a.alive[i] = 1;
            a.P[i] = 0;
            a.P2[i] = 0;
            a.inM[i] = 0;
        }
        if (i < a.n) {
            if (a.pairs) a.vmatch[i] = 0;
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

// a1 of a re-randomised round for the vertices of the active list. The
// regions are those of the fixed-order loop; warps of a persistent grid
// take them one at a time from a counter, so that regions with long lists
// do not leave other warps idle.
template <bool kPairs>
__global__ void __launch_bounds__(kT, 4) k_rargmax(RoundArgs a) {
    DevState *st = a.st;
    const int r = st->round;
    const int par = st->parity;
    const int32_t *in = par ? a.list1 : a.list0;
    int32_t *out = par ? a.list0 : a.list1;
    const uint32_t *cnt_in = a.lcnt + (size_t)par * a.nregions;
    uint32_t *cnt_out = a.lcnt + (size_t)(par ^ 1) * a.nregions;
    uint32_t *Pc = (r & 1) ? a.P2 : a.P;  // counts of this round
    uint32_t *Po = (r & 1) ? a.P : a.P2;  // counts of the previous round
    // round 1 keeps every entry: it reads the immutable lists and writes
    // nothing; round 2 compacts them into the working copy; later rounds
    // compact the working copy in place
    const int2 *src = r <= 2 ? a.vadjE : a.vadjR;
    int2 *dst = a.vadjR;
    const int32_t *nsrc = r <= 2 ? a.vnbrE : a.vnbrR;  // graphs
    int32_t *ndst = a.vnbrR;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    unsigned long long scanned = 0, props = 0, nlive = 0;
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
        uint32_t kept = 0, won = 0;
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
                if (slot < a.lq_cap) {
                    a.lq[slot] = make_int2(v, (int32_t)(uint32_t)old);
                    a.lbest[slot] = 0;
                } else {
                    st->fault = 3;
                }
            }
            // the short and medium lists of the tile as one sequence
            const uint32_t L = act && !lng ? (uint32_t)rec.w : 0u;
            unsigned long long best = 0;
            uint32_t live = 0;
            uint32_t Lmax = 0;
            if (kPairs && r == 1) {
                Lmax = L;
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) Lmax = max(Lmax, __shfl_xor_sync(kFull, Lmax, d));
            }
            if (kPairs && r == 1 && Lmax <= kSeqMax) {  // warp-uniform
                if (L) best = first_round_max(a.vadjE, (int64_t)(uint32_t)rec.z, L, a.noise_s0, a.noise_scale);
                live = L;
                scanned += L;
            } else {
            const uint32_t inc = warp_inclusive_scan(L);
            const uint32_t pre = inc - L;
            const uint32_t total = __shfl_sync(kFull, inc, 31);
            for (uint32_t s0 = 0; s0 < total; s0 += 32 * kU) {
                int o[kU];
                uint32_t opre[kU];
                int64_t ob[kU];
                int2 ev[kU];
                int32_t nbv[kU];  // graphs: the other endpoint of each entry
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    // owner of position p: the largest lane x with pre_x <= p
                    // (it has L_x > 0 when p < total)
                    const uint32_t p = s0 + 32 * u + lane;
                    int x = 0;
#pragma unroll
                    for (int bit = 16; bit; bit >>= 1) {
                        const uint32_t pc = __shfl_sync(kFull, pre, x + bit);
                        if (pc <= p) x += bit;
                    }
                    o[u] = x;
                    opre[u] = __shfl_sync(kFull, pre, x);
                    ob[u] = (int64_t)(uint32_t)__shfl_sync(kFull, rec.z, x);
                }
                // plain loads: from round 3 on this kernel rewrites the lists behind the reads
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const uint32_t p = s0 + 32 * u + lane;
                    ev[u] = p < total ? src[ob[u] + (int64_t)(p - opre[u])] : make_int2(0, 0);
                    if (kPairs) nbv[u] = p < total ? nsrc[ob[u] + (int64_t)(p - opre[u])] : 0;
                }
                bool lvv[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const uint32_t p = s0 + 32 * u + lane;
                    lvv[u] = p < total &&
                             (r == 1 || (kPairs ? __ldg(a.vmatch + nbv[u]) == 0 : __ldg(a.alive + ev[u].x) != 0));
                }
                __syncwarp();  // every read of this batch precedes its compaction writes
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const uint32_t su = s0 + 32 * u;
                    if (su < total) {  // warp-uniform
                        const bool lv = lvv[u];
                        const unsigned long long key =
                            lv ? round_key(a, r, (uint32_t)ev[u].x, __int_as_float(ev[u].y)) : 0ull;
                        // lanes [sst, lane) of this step hold earlier entries of the same list
                        const uint32_t sst = opre[u] > su ? opre[u] - su : 0u;
                        const unsigned seg_lt = lt & ~((1u << sst) - 1u);
                        const unsigned lm = __ballot_sync(kFull, lv);
                        const uint32_t carried = __shfl_sync(kFull, live, o[u]);
                        if (lv && r > 1) {  // compaction
                            dst[ob[u] + carried + __popc(lm & seg_lt)] = ev[u];
                            if (kPairs) ndst[ob[u] + carried + __popc(lm & seg_lt)] = nbv[u];
                        }
                        // segmented running maximum over the step
                        unsigned long long mx = key;
#pragma unroll
                        for (int d = 1; d < 32; d <<= 1) {
                            const unsigned long long y = __shfl_up_sync(kFull, mx, d);
                            if (lane >= d && (uint32_t)(lane - d) >= sst && y > mx) mx = y;
                        }
                        // each owner takes the maximum at the last lane of its piece
                        const bool mine = L > 0 && pre < su + 32 && pre + L > su;
                        const uint32_t tail = mine ? min(pre + L - su, 32u) - 1u : (uint32_t)lane;
                        const unsigned long long tmx = __shfl_sync(kFull, mx, (int)tail);
                        if (mine) {
                            if (tmx > best) best = tmx;
                            const uint32_t lo = pre > su ? pre - su : 0u;
                            const unsigned upto = tail == 31u ? kFull : ((2u << tail) - 1u);
                            live += __popc(lm & upto & ~((1u << lo) - 1u));
                        }
                        scanned += su + lane < total ? 1u : 0u;
                    }
                }
            }
            }
            bool keep = false, w = false;
            int32_t nb = -1;
            if (act && !lng) {
                if (r > 1) Po[rec.x] = 0;  // T[v] of the previous round is what v counted there
                if (best != 0) {
                    nb = __ldg(a.jof + edge_of_key(best));
                    a.vrec[v] = make_int4(nb, 0, rec.z, (int32_t)live);
                    w = propose(a, Pc, nb);
                    keep = true;
                    ++props;
                    nlive += live;
                } else {
                    reinterpret_cast<int2 *>(a.vrec + v)[0] = make_int2(kCurNone, 0);
                }
            }
            const unsigned km = __ballot_sync(kFull, keep);
            if (keep) out[base + kept + __popc(km & lt)] = v;
            kept += __popc(km);
            const unsigned lgm = __ballot_sync(kFull, lng);  // long lists stay; k_rfin may drop them
            if (lng) out[base + kept + __popc(lgm & lt)] = v;
            kept += __popc(lgm);
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
    warp_add_u64(scanned, &st->adv);
    warp_add_u64(props, &st->proposals);
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
            const int2 q = a.lq[lo];
            const int4 rec = a.vrec[q.x];
            const int64_t lb = (int64_t)(uint32_t)rec.z;
            const int64_t b = lb + (int64_t)(c - (uint32_t)q.y) * kChunk;
            const int64_t e = min(lb + (int64_t)(uint32_t)rec.w, b + (int64_t)kChunk);
            unsigned long long mx = 0;
            for (int64_t p = b + lane; p < e; p += 32) {
                const int2 x = __ldg(a.vadjE + p);  // long lists are never compacted
                if (r == 1 || (kPairs ? __ldg(a.vmatch + __ldg(a.vnbrE + p)) == 0 : __ldg(a.alive + x.x) != 0)) {
                    const unsigned long long k = round_key(a, r, (uint32_t)x.x, __int_as_float(x.y));
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
                if (mx) atomicMax(a.lbest + lo, mx);
                scanned += (unsigned long long)(e - b);
            }
        }
    }
    block_add_u64(scanned, s_red, &st->adv);
    block_add_u64(nlive, s_red, &st->live);
}

// Proposals of the long lists (one thread per list).
__global__ void __launch_bounds__(kT) k_rfin(RoundArgs a) {
    __shared__ unsigned long long s_red[kT / 32];
    DevState *st = a.st;
    const unsigned long long lp = st->lpack;
    const uint32_t nl = (uint32_t)(lp >> 32);
    unsigned long long props = 0;
    if (nl <= a.lq_cap) {
        const int r = st->round, par = st->parity;
        uint32_t *Pc = (r & 1) ? a.P2 : a.P;
        uint32_t *Po = (r & 1) ? a.P : a.P2;
        const uint32_t stride = gridDim.x * kT;
        // whole warps iterate, so that winners can be appended with ballots
        for (uint32_t s0 = blockIdx.x * kT + (threadIdx.x & ~31u); s0 < nl; s0 += stride) {
            const uint32_t s = s0 + (threadIdx.x & 31);
            bool w = false;
            int32_t nb = -1;
            if (s < nl) {
                const int32_t v = a.lq[s].x;
                const int32_t prev = a.vrec[v].x;
                if (r > 1) Po[prev] = 0;
                const unsigned long long k = a.lbest[s];
                if (k == 0) {  // no live entry left: v leaves the active list
                    reinterpret_cast<int2 *>(a.vrec + v)[0] = make_int2(kCurNone, 0);
                    atomicSub(&st->cnt[par ^ 1], 1u);
                } else {
                    nb = __ldg(a.jof + edge_of_key(k));
                    reinterpret_cast<int2 *>(a.vrec + v)[0] = make_int2(nb, 0);
                    w = propose(a, Pc, nb);
                    ++props;
                }
            }
            append_winners(a, w, nb);
        }
    }
    block_add_u64(props, s_red, &st->proposals);
}

// Graphs: the other endpoint of every list entry (the second word of the
// fixed order's {edge, endpoint} pairs, in the same list order).
__global__ void __launch_bounds__(kT) k_pair_endpoints(const int2 *vpair, uint64_t kappa, int32_t *vnbrE) {
    for (uint64_t i = blockIdx.x * (uint64_t)kT + threadIdx.x; i < kappa; i += (uint64_t)gridDim.x * kT)
        vnbrE[i] = vpair[i].y;
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
    a.lq = h->lq;
    a.lbest = h->lbest;
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
    k_rfin<<<(unsigned)h->sm_count, kT, 0, s>>>(a);
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
    if (h->vrecR) return HM_OK;
    const uint64_t n = (uint64_t)h->n, m = (uint64_t)h->m;
    h->lq_cap = (uint32_t)(std::min<uint64_t>(n, h->kappa / kLong) + 1);
    hm_status st;
    if ((st = dalloc(&h->vrecR, n, s, "re-randomised vertex records")) != HM_OK ||
        (st = dalloc(&h->vadjE, h->kappa, s, "vertex lists in edge ids")) != HM_OK ||
        (st = dalloc(&h->vadjR, h->kappa, s, "re-randomised vertex lists")) != HM_OK ||
        (st = dalloc(&h->jof, m, s, "inverse edge order")) != HM_OK ||
        (st = dalloc(&h->P2, m, s, "second proposal counters")) != HM_OK ||
        (st = dalloc(&h->lq, h->lq_cap, s, "long-list queue")) != HM_OK ||
        (st = dalloc(&h->lbest, h->lq_cap, s, "long-list maxima")) != HM_OK ||
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
    void *bufs[] = {h->vrecR, h->vadjE, h->vadjR, h->jof, h->P2, h->lq, h->lbest, h->vnbrE, h->vnbrR};
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, h->cap_stream);
    h->vrecR = nullptr;
    h->vadjE = nullptr;
    h->vadjR = nullptr;
    h->jof = nullptr;
    h->P2 = nullptr;
    h->lq = nullptr;
    h->lbest = nullptr;
    h->vnbrE = nullptr;
    h->vnbrR = nullptr;
    if (h->exec_rand) cudaGraphExecDestroy(h->exec_rand);
    h->exec_rand = nullptr;
}

}  // namespace hm
