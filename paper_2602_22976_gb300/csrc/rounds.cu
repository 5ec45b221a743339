// rounds.cu - the round loop of locally-maximal hypergraph matching
// (Sec. 3.1, Alg. 1, Alg. 3) on the device.
//
// One round is three kernels:
//   k_argmax    a1: every active vertex v makes T[v] the highest-priority
//               live edge of its list. The list is sorted by decreasing
//               priority and edges only ever die, so T[v] is a cursor that
//               moves forward past dead entries (Alg. 3's argmax; Sec. 4.1
//               keeps T across rounds). When T[v] moves to a new edge e the
//               vertex counts down P[e]; the vertex that brings P[e] to 0 has
//               seen e chosen by all |e| of its vertices (the test P[e] = |e|
//               of Alg. 1, Sec. 4.1) and appends e to the winners.
//   k_win       a2: winners join M; their vertices become matched and each
//               emits the rest of its list (from its cursor on) as one kill
//               range.
//   k_kill      a3 + a4: every entry of every kill range is deactivated (the
//               vertex-side deactivation of Alg. 1; the writes race benignly,
//               Sec. 4.2). The ranges are read as one concatenated sequence
//               split evenly over the warps. The block that finishes last
//               ends the round: counters, termination test, and the
//               conditional of the CUDA graph's while node.
// The active vertex list is compacted inside k_argmax (vertices that are
// matched or have no live edge left drop out), each warp in place in its own
// region of the list.
// Graphs (every edge has two pins) skip the kill: an edge is live exactly
// when neither endpoint is matched, so k_argmax reads each list entry with
// its other endpoint and that endpoint's matched flag, k_win only sets the
// flags of the winners' endpoints, and the kill step is one block that ends
// the round.
#include "hm_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <new>
#include <vector>

namespace hm {
namespace {

constexpr int kT = 256;        // threads per block of the round kernels
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

// Sum over the block, added once per block to *dst.
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

// Per-match reset: live flags (matched flags of the vertices for graphs),
// result mask, and the P counters from their initial copy (P0). The vertex
// records' T and cursor are set by round 1.
__global__ void __launch_bounds__(kT) k_init(RoundArgs a) {
    const int64_t pw = a.p16 ? (a.m + 1) / 2 : a.m;  // words of P
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < a.m; i += (int64_t)gridDim.x * kT) {
        if (!a.pairs) a.alive[i] = 1;
        a.inM[i] = 0;
        if (i < pw) a.P[i] = __ldg(a.P0 + i);
    }
    if (a.pairs)
        for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * kT)
            a.vmatch[i] = 0;
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

// Initial P counters: |e| of every edge (two 16-bit halves a word when
// p16), computed once per handle.
__global__ void __launch_bounds__(kT) k_p0(RoundArgs a, uint32_t *__restrict__ p0) {
    const int64_t pw = a.p16 ? (a.m + 1) / 2 : a.m;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < pw; i += (int64_t)gridDim.x * kT) {
        uint32_t x;
        if (a.graph) {  // every edge has two pins
            x = 2 * i + 1 < a.m ? 0x00020002u : 2u;
        } else if (!a.p16) {
            x = (uint32_t)(a.eoffj[i + 1] - a.eoffj[i]);
        } else {  // edges 2i and 2i + 1
            const int64_t e = 2 * i;
            const uint32_t lo = (uint32_t)(a.eoffj[e + 1] - a.eoffj[e]);
            const uint32_t hi = e + 1 < a.m ? (uint32_t)(a.eoffj[e + 2] - a.eoffj[e + 1]) : 0u;
            x = lo | (hi << 16);
        }
        p0[i] = x;
    }
}

// Requests the 16-byte line holding *p into L2 (no register is written).
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

constexpr int kLaneSteps = 4;  // a lane walks at most 4 x 4 entries before its warp helps

// First live entry of vadj[c, end) within kLaneSteps steps of four entries
// (their loads are independent, so a step costs two dependent memory trips).
// Returns its position (j = the edge), or end if the list ran out; sets
// `more` when the budget ran out first. List positions are below kappa <
// 2^32, so they are kept in 32 bits (fewer registers: more warps resident).
__device__ __forceinline__ uint32_t next_live_bounded(const int32_t *__restrict__ vadj,
                                                      const uint8_t *__restrict__ alive, uint32_t c, uint32_t end,
                                                      int32_t &j, bool &more) {
    more = false;
#pragma unroll 1
    for (int step = 0; step < kLaneSteps; ++step) {
        if (c >= end) return end;
        const uint32_t left = end - c;
        const int32_t e0 = __ldg(vadj + c);
        const int32_t e1 = left > 1 ? __ldg(vadj + c + 1) : -1;
        const int32_t e2 = left > 2 ? __ldg(vadj + c + 2) : -1;
        const int32_t e3 = left > 3 ? __ldg(vadj + c + 3) : -1;
        const bool a0 = __ldg(alive + e0) != 0;
        const bool a1 = e1 >= 0 && __ldg(alive + e1) != 0;
        const bool a2 = e2 >= 0 && __ldg(alive + e2) != 0;
        const bool a3 = e3 >= 0 && __ldg(alive + e3) != 0;
        if (a0) { j = e0; return c; }
        if (a1) { j = e1; return c + 1; }
        if (a2) { j = e2; return c + 2; }
        if (a3) { j = e3; return c + 3; }
        if (left <= 4) return end;
        c += 4;
    }
    more = true;
    return end;
}

// The same walk over a graph's pair list: entry c is live when the other
// endpoint of its edge is unmatched (the list's own vertex is active, so it
// is unmatched too). Returns the position, with j = the edge and o = that
// endpoint; end and `more` as above.
__device__ __forceinline__ uint32_t next_live_pair(const int2 *__restrict__ vpair, const uint8_t *__restrict__ vmatch,
                                                   uint32_t c, uint32_t end, int32_t &j, int32_t &o, bool &more) {
    more = false;
#pragma unroll 1
    for (int step = 0; step < kLaneSteps; ++step) {
        if (c >= end) return end;
        const uint32_t left = end - c;
        const int2 e0 = __ldg(vpair + c);
        const int2 e1 = left > 1 ? __ldg(vpair + c + 1) : make_int2(-1, -1);
        const int2 e2 = left > 2 ? __ldg(vpair + c + 2) : make_int2(-1, -1);
        const int2 e3 = left > 3 ? __ldg(vpair + c + 3) : make_int2(-1, -1);
        const bool a0 = __ldg(vmatch + e0.y) == 0;
        const bool a1 = e1.y >= 0 && __ldg(vmatch + e1.y) == 0;
        const bool a2 = e2.y >= 0 && __ldg(vmatch + e2.y) == 0;
        const bool a3 = e3.y >= 0 && __ldg(vmatch + e3.y) == 0;
        if (a0) { j = e0.x; o = e0.y; return c; }
        if (a1) { j = e1.x; o = e1.y; return c + 1; }
        if (a2) { j = e2.x; o = e2.y; return c + 2; }
        if (a3) { j = e3.x; o = e3.y; return c + 3; }
        if (left <= 4) return end;
        c += 4;
    }
    more = true;
    return end;
}

// a1 for one vertex per lane: T[v] <- the first live entry of v's list at
// or after its cursor. Returns whether v stays active; nb = the edge v newly
// chose (it must count down P[nb]) or -1. All 32 lanes must call it: a lane
// whose walk exceeds its budget is finished by the whole warp, 32 entries
// per step (coalesced list read, one ballot). kPairs: a graph's lists of
// {edge, other endpoint}, liveness read from the endpoints' matched flags,
// records {T, absolute cursor, list end, other endpoint of T}.
template <bool kPairs>
__device__ __forceinline__ bool argmax_vertex(const RoundArgs &a, int r, bool ok, int32_t v, int32_t &nb,
                                              uint32_t &adv) {
    const int lane = threadIdx.x & 31;
    const int32_t *__restrict__ vadj = a.vadj;
    const int2 *__restrict__ vpair = a.vpair;
    const uint8_t *__restrict__ alive = a.alive;
    const uint8_t *__restrict__ vmatch = a.vmatch;
    bool keep = false, walk = false, coop = false;
    nb = -1;
    uint32_t vb = 0, from = 0, end = 0, cn = 0;
    int32_t jj = 0, oo = 0;
    if (ok && r == 1) {
        // every edge is live in round 1: T[v] is the first entry; the record
        // (T, cursor) starts here
        const int32_t f = __ldg(a.firstj + v);
        if (kPairs)
            a.vrec[v] = make_int4(f, (int32_t)(uint32_t)__ldg(a.voff + v), (int32_t)(uint32_t)__ldg(a.voff + v + 1),
                                  __ldg(a.firstnbr + v));
        else
            reinterpret_cast<int2 *>(a.vrec + v)[0] = make_int2(f, 0);
        if (f >= 0) {
            nb = f;
            keep = true;
        }
    } else if (ok) {
        // graphs: a matched vertex keeps its record; its own flag, loaded
        // beside the record, says so
        const bool mine = kPairs && __ldg(vmatch + v) != 0;
        const int4 rec = a.vrec[v];
        if (rec.x >= 0 && !mine) {
            if (kPairs ? __ldg(vmatch + rec.w) == 0 : __ldg(alive + rec.x) != 0) {
                keep = true;  // T[v] still live: unchanged
            } else {
                if (kPairs) {
                    from = (uint32_t)rec.y;
                    end = (uint32_t)rec.z;
                    cn = next_live_pair(vpair, vmatch, from + 1, end, jj, oo, coop);
                } else {
                    vb = (uint32_t)rec.z;
                    end = vb + (uint32_t)rec.w;
                    from = vb + (uint32_t)rec.y;
                    cn = next_live_bounded(vadj, alive, from + 1, end, jj, coop);
                }
                walk = true;
            }
        }
    }
    unsigned cm = __ballot_sync(kFull, coop);
    while (cm) {
        const int src = __ffs(cm) - 1;
        uint32_t p = __shfl_sync(kFull, from, src) + 1 + 4 * kLaneSteps;
        const uint32_t e = __shfl_sync(kFull, end, src);
        uint32_t fpos = e;
        int32_t fj = 0, fo = 0;
        while (p < e) {
            const bool in = (uint32_t)lane < e - p;  // p + lane < e, without overflow
            const uint32_t q = p + (uint32_t)lane;
            unsigned lm;
            int32_t ej, eo = 0;
            if (kPairs) {
                const int2 x = in ? __ldg(vpair + q) : make_int2(-1, -1);
                ej = x.x;
                eo = x.y;
                lm = __ballot_sync(kFull, eo >= 0 && __ldg(vmatch + eo) == 0);
            } else {
                ej = in ? __ldg(vadj + q) : -1;
                lm = __ballot_sync(kFull, ej >= 0 && __ldg(alive + ej) != 0);
            }
            if (lm) {
                const int f = __ffs(lm) - 1;
                fpos = p + (uint32_t)f;
                fj = __shfl_sync(kFull, ej, f);
                if (kPairs) fo = __shfl_sync(kFull, eo, f);
                break;
            }
            if (e - p <= 32) break;  // the list ran out
            p += 32;
        }
        if (lane == src) {
            cn = fpos;
            jj = fj;
            oo = fo;
        }
        cm &= cm - 1;
    }
    if (walk && kPairs) {
        adv += cn - from;
        if (cn < end) {
            a.vrec[v] = make_int4(jj, (int32_t)cn, (int32_t)end, oo);
            nb = jj;
            keep = true;
        } else {
            a.vrec[v] = make_int4(kCurNone, 0, 0, -1);
        }
    } else if (walk) {
        adv += cn - from;
        int2 *st2 = reinterpret_cast<int2 *>(a.vrec + v);
        if (cn < end) {
            st2[0] = make_int2(jj, (int32_t)(cn - vb));
            nb = jj;
            keep = true;
        } else {
            st2[0] = make_int2(kCurNone, 0);
        }
    }
    return keep;
}

// a2 for up to 32 winners, one per lane (j = relabelled edge id, or -1):
// the edge joins M (input numbering, with its round), every vertex of it is
// marked matched, and each vertex emits one kill range: its list from the
// cursor on (the winner's own entry included, which kills the winner). The
// pins of the warp's winners are spread over the lanes, 128 at a time (four
// per lane, their loads in flight together); the items of those pins and
// their entries are reserved with one 64-bit atomic, so the item order and
// the entry offsets ascend together. The reservation counter is one word
// for the whole GPU: one atomic per 128 pins keeps it from serialising the
// step. All 32 lanes must call.
__device__ __forceinline__ void warp_win(const RoundArgs &a, int r, int32_t j, unsigned long long &winpins) {
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    uint32_t len = 0;
    int64_t b = 0;
    int32_t ein = -1;
    if (j >= 0) {
        if (a.graph) {  // d = 2: the pins sit at 2j, 2j + 1
            b = 2 * (int64_t)j;
            len = 2;
        } else {
            b = __ldg(a.eoffj + j);
            len = (uint32_t)(__ldg(a.eoffj + j + 1) - b);
        }
        ein = __ldg(a.order + j);
        a.inM[ein] = 1;
        if (a.wround) a.wround[ein] = r;
        winpins += len;
        if (a.pairs) {
            // graph, fixed order: both endpoints chose j (the countdown
            // reached 0); their matched flags are the whole update - the
            // argmax step reads them, and there is no kill range
            const int2 e = __ldg(reinterpret_cast<const int2 *>(a.pinsj) + j);
            a.vmatch[e.x] = 1;
            a.vmatch[e.y] = 1;
        }
    }
    if (a.pairs) return;
    const uint32_t inc = warp_inclusive_scan(len);
    const uint32_t exc = inc - len;
    const uint32_t total = __shfl_sync(kFull, inc, 31);
    const unsigned lt = lanemask_lt();
    for (uint32_t p0 = 0; p0 < total; p0 += 32 * U) {
        int32_t v[U], jk[U];  // jk: the winner as T[v] names it (j, or its input id when a.t_input)
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t q = p0 + 32 * u + lane;
            // owner of pin q: the largest lane k with exc_k <= q (exc ascends)
            int k = 0;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                const uint32_t e = __shfl_sync(kFull, exc, k + d);
                if (e <= q) k += d;
            }
            jk[u] = __shfl_sync(kFull, a.t_input ? ein : j, k);
            const int64_t bk = __shfl_sync(kFull, b, k);
            const uint32_t ek = __shfl_sync(kFull, exc, k);
            v[u] = q < total ? __ldg(a.pinsj + bk + (q - ek)) : -1;
        }
        uint32_t ibeg[U], ilen[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ibeg[u] = 0;
            ilen[u] = 0;
            if (v[u] >= 0) {
                const int4 rec = a.vrec[v[u]];
                const uint32_t c = (uint32_t)rec.z + (uint32_t)rec.y;
                const uint32_t end = (uint32_t)rec.z + (uint32_t)rec.w;
                // T[v] must be the winner: v chose it, and nothing moves it
                if (rec.x == jk[u] && c < end) {
                    reinterpret_cast<int2 *>(a.vrec + v[u])[0] = make_int2(kCurMatched, 0);
                    ibeg[u] = c;
                    ilen[u] = end - c;
                } else {
                    a.st->fault = 1;
                }
            }
        }
        unsigned has[U];
        uint32_t iinc[U], ibase[U], ebase[U];
        uint32_t nitems = 0, nent = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            has[u] = __ballot_sync(kFull, ilen[u] > 0);
            iinc[u] = warp_inclusive_scan(ilen[u]);
            ibase[u] = nitems;
            ebase[u] = nent;
            nitems += (uint32_t)__popc(has[u]);
            nent += __shfl_sync(kFull, iinc[u], 31);
        }
        unsigned long long old = 0;
        if (lane == 0 && nitems)
            old = atomicAdd(&a.st->kpack, ((unsigned long long)nent << 32) | (unsigned long long)nitems);
        old = __shfl_sync(kFull, old, 0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (ilen[u]) {
                const uint64_t idx = (uint64_t)(uint32_t)old + ibase[u] + (uint32_t)__popc(has[u] & lt);
                const uint32_t eb = (uint32_t)(old >> 32) + ebase[u] + iinc[u] - ilen[u];
                if (idx < a.item_cap) a.items[idx] = KillItem{ibeg[u], eb};
                else a.st->fault = 2;
            }
        }
    }
}

// a1: argmax (cursor advance), proposals, win test, list compaction.
// Warp g owns region g of the active list (the active vertices of one
// vertex range) and compacts it in place into the other list with ballots:
// no barrier and no shared counter inside the loop, so a lane that walks a
// long run of dead entries only holds up its own warp. T[v] is kept as an
// edge id, so the common case - T[v] still live - costs one record read and
// one flag read. At the end each block reserves one slot range for its
// warps' winners and copies them into the contiguous winner list (k_win
// reads the winners' vertex records, which must be complete: that is what
// keeps a2 in its own kernel).
template <bool kPairs>
__global__ void __launch_bounds__(kT, 6) k_argmax(RoundArgs a) {
    __shared__ unsigned long long s_red[kT / 32];
    __shared__ uint32_t s_keep[kT / 32], s_won[kT / 32];
    __shared__ uint32_t s_wbase;
    DevState *st = a.st;
    const int r = st->round;
    const int par = st->parity;
    const int32_t *in = par ? a.list1 : a.list0;
    int32_t *out = par ? a.list0 : a.list1;
    const uint32_t *cnt_in = a.lcnt + (size_t)par * a.nregions;
    uint32_t *cnt_out = a.lcnt + (size_t)(par ^ 1) * a.nregions;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const uint32_t g = blockIdx.x * (kT / 32) + wib;
    uint32_t adv = 0, props = 0;  // one thread's counts stay below kappa < 2^32
    uint32_t kept = 0, won = 0;
    if (g < a.nregions) {
        const uint64_t base = (uint64_t)g * a.region;
        uint32_t count;
        if (r == 1) {
            const int64_t left = a.n - (int64_t)base;
            count = left <= 0 ? 0u : (uint32_t)(left < (int64_t)a.region ? left : (int64_t)a.region);
        } else {
            count = cnt_in[g];
        }
        // from round 2 on the list ids run two groups ahead, and the record
        // of the next group's vertex is requested into L2 while this group
        // walks (the id chain list -> record -> flag -> list is latency-bound
        // once the rounds thin out)
        int32_t vn1 = 0, vn2 = 0;
        if (r > 1) {
            vn1 = lane < count ? in[base + lane] : 0;
            vn2 = 32u + lane < count ? in[base + 32 + lane] : 0;
        }
        for (uint32_t i0 = 0; i0 < count; i0 += 32) {
            const uint32_t i = i0 + lane;
            const bool ok = i < count;
            int32_t v;
            if (r == 1) {
                v = ok ? (int32_t)(base + i) : 0;
            } else {
                v = ok ? vn1 : 0;
                vn1 = vn2;
                if (i + 32 < count) prefetch_l2(a.vrec + vn1);
                vn2 = i + 64 < count ? in[base + i + 64] : 0;
            }
            int32_t nb;
            const bool keep = argmax_vertex<kPairs>(a, r, ok, v, nb, adv);
            bool w = false;
            if (nb >= 0) {
                ++props;
                if (a.p16) {  // a count never goes below 0, so no borrow crosses halves
                    const int sh = (nb & 1) * 16;
                    w = ((atomicSub(&a.P[nb >> 1], 1u << sh) >> sh) & 0xFFFFu) == 1u;
                } else {
                    w = atomicSub(&a.P[nb], 1u) == 1u;
                }
            }
            const unsigned km = __ballot_sync(kFull, keep);
            if (keep) out[base + kept + __popc(km & lt)] = v;
            kept += __popc(km);
            const unsigned wm = __ballot_sync(kFull, w);
            if (w) a.wstage[base + won + __popc(wm & lt)] = nb;
            won += __popc(wm);
        }
        if (lane == 0) cnt_out[g] = kept;
    }
    // a block with nothing to report (most blocks in the late rounds) skips
    // the block-level combining below
    if (!__syncthreads_or(kept != 0 || won != 0 || adv != 0 || props != 0)) return;
    if (lane == 0) {
        s_keep[wib] = kept;
        s_won[wib] = won;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tk = 0, tw = 0;
        for (int w = 0; w < kT / 32; ++w) {
            tk += s_keep[w];
            const uint32_t t = s_won[w];
            s_won[w] = tw;
            tw += t;
        }
        if (tk) atomicAdd(&st->cnt[par ^ 1], tk);
        s_wbase = tw ? atomicAdd(&st->nwin, tw) : 0u;
    }
    __syncthreads();
    if (g < a.nregions)
        for (uint32_t i = lane; i < won; i += 32) {
            const uint64_t idx = (uint64_t)s_wbase + s_won[wib] + i;
            if (idx < a.win_cap) a.win[idx] = a.wstage[(uint64_t)g * a.region + i];
            else st->fault = 2;
        }
    block_add_u64(adv, s_red, &st->adv);
    block_add_u64(props, s_red, &st->proposals);
}

// Statistics of the per-kernel replay only, launched between its timed
// argmax and win kernels: the sum of the degrees of the vertices the argmax
// step kept (the unmatched vertices with a live edge), added to the round's
// counter. The timed match does not run it. The degree comes from the
// vertex record (a graph's record holds the list end).
__global__ void __launch_bounds__(kT) k_kept_degrees(RoundArgs a) {
    __shared__ unsigned long long s_red[kT / 32];
    DevState *st = a.st;
    const int par = st->parity;
    const int32_t *out = par ? a.list0 : a.list1;
    const uint32_t *cnt_out = a.lcnt + (size_t)(par ^ 1) * a.nregions;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)kT + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * kT) >> 5;
    unsigned long long sum = 0;
    for (uint64_t g = warp; g < a.nregions; g += nwarps) {
        const uint32_t c = cnt_out[g];
        for (uint32_t i = lane; i < c; i += 32) {
            const int32_t v = out[g * a.region + i];
            const int4 rec = a.vrec[v];
            if (rec.x < 0) continue;
            sum += a.pairs ? (uint32_t)rec.z - (uint64_t)a.voff[v] : (uint32_t)rec.w;
        }
    }
    block_add_u64(sum, s_red, &st->sdeg);
}

// Statistics of the per-kernel replay only, launched before a round's timed
// kernels: the edges live at the start of the round and the sum of their
// sizes, added to the round's counters. A graph's edge is live while
// neither endpoint is matched (its liveness is read from the matched flags
// in both orders); a hypergraph's live flag is indexed by j in the fixed
// order and by the input id in the re-randomised rounds.
__global__ void __launch_bounds__(kT) k_live_edges(RoundArgs a, int random) {
    __shared__ unsigned long long s_red[kT / 32];
    unsigned long long ne = 0, np = 0;
    for (int64_t j = blockIdx.x * (int64_t)kT + threadIdx.x; j < a.m; j += (int64_t)gridDim.x * kT) {
        bool live;
        int64_t size;
        if (a.pairs) {
            const int2 e = __ldg(reinterpret_cast<const int2 *>(a.pinsj) + j);
            live = a.vmatch[e.x] == 0 && a.vmatch[e.y] == 0;
            size = 2;
        } else {
            live = a.alive[random ? __ldg(a.order + j) : (int32_t)j] != 0;
            size = a.eoffj[j + 1] - a.eoffj[j];
        }
        if (live) {
            ne += 1;
            np += (unsigned long long)size;
        }
    }
    block_add_u64(ne, s_red, &a.st->ledges);
    block_add_u64(np, s_red, &a.st->lpins);
}

// a2: each warp takes 32 winners of the round at a time (warp_win). The
// winners' vertex records were completed by the argmax kernel.
__global__ void __launch_bounds__(kT) k_win(RoundArgs a) {
    __shared__ unsigned long long s_red[kT / 32];
    DevState *st = a.st;
    const uint32_t nw = (uint32_t)min((uint64_t)st->nwin, a.win_cap);
    const int r = st->round;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)kT + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * kT) >> 5;
    if ((uint64_t)blockIdx.x * kT >= nw) return;  // no winner for any warp of this block (uniform)
    unsigned long long winpins = 0;
    for (uint64_t w0 = warp * 32; w0 < nw; w0 += nwarps * 32) {
        const int32_t j = w0 + lane < nw ? a.win[w0 + lane] : -1;
        warp_win(a, r, j, winpins);
    }
    block_add_u64(winpins, s_red, &st->winpins);
}

// Stats row of round r, termination test and next-round decision.
// Returns 1 if another round must run.
__device__ int finish_round(const RoundArgs &a, DevState *st, int r, int64_t active, uint32_t nw,
                            uint32_t next, unsigned long long adv, unsigned long long props,
                            unsigned long long winpins, unsigned long long kills, uint32_t items,
                            unsigned long long live, unsigned long long sdeg, unsigned long long ledges,
                            unsigned long long lpins) {
    write_stats_row(a, r, active, nw, next, adv, props, winpins, kills, items, live, sdeg, ledges, lpins);
    int cont = 0;
    if (st->fault) {
        st->status = HM_ECUDA;
    } else if (nw == 0) {
        // No winner: no edge was live at the start of this round. Vertices
        // still holding a live T[v] would contradict that (a vertex repeated
        // inside an edge can never let the edge reach P = 0).
        st->rounds_done = r - 1;
        if (next > 0) st->status = HM_EINVAL;
    } else {
        st->rounds_done = r;
        if (next > 0) {
            if (r >= a.cap) st->status = HM_ETIMEOUT;
            else cont = 1;
        }
    }
    return cont;
}

// a4 (one thread, after every other block of the kill step has finished):
// records the round, decides whether another round runs, resets the
// per-round counters.
__device__ void round_end(const RoundArgs &a) {
    DevState *st = a.st;
    const int r = st->round, par = st->parity;
    const uint32_t nw = st->nwin, next = st->cnt[par ^ 1];
    const int64_t active = r == 1 ? a.n : (int64_t)st->cnt[par];
    const unsigned long long kp = st->kpack;
    int cont;
    if (a.erounds) {
        // re-randomised round 1, followed by edge rounds: record it; the
        // next round's first pass finds whether any edge is still live and
        // applies the round cap (no winner: no edge was live at all)
        write_stats_row(a, r, active, nw, next, st->adv, st->proposals, st->winpins, kp >> 32, (uint32_t)kp,
                        st->live, st->sdeg, st->ledges, st->lpins);
        cont = 0;
        if (st->fault) st->status = HM_ECUDA;
        else if (nw == 0) st->rounds_done = 0;
        else {
            st->rounds_done = 1;
            cont = 1;
        }
    } else {
        cont = finish_round(a, st, r, active, nw, next, st->adv, st->proposals, st->winpins, kp >> 32,
                            (uint32_t)kp, st->live, st->sdeg, st->ledges, st->lpins);
    }
    st->nwin = 0;
    st->kdone = 0;
    st->adv = st->kills = st->winpins = st->proposals = 0;
    st->live = st->kpack = st->sdeg = 0;
    st->ledges = st->lpins = 0;
    if (cont) {
        st->round = r + 1;
        st->parity = par ^ 1;
        st->cnt[par] = 0;
    } else {
        st->finished = 1;
    }
    if (a.use_cond) cudaGraphSetConditional(a.cond, cont ? 1u : 0u);
}

// a3 + a4: deactivate every entry of every kill range, then end the round.
// The round's ranges are one concatenated sequence of E entries (item i
// starts at offset items[i].ebase); each warp takes an equal slice of it
// (at least kill_chunk entries), finds the item holding its first entry by
// a 32-way search, and walks its slice 128 entries at a time: a window of
// 32 consecutive items sits in the lanes, each entry finds its item in the
// window with five shuffles, and each lane has four entries in flight.
// From round 2 on most targets are already dead (they sit behind the
// cursors of other vertices), and on this GPU a random 1-byte load costs
// less than half of a random 1-byte store, so the flag is read first and
// only live targets are cleared (in round 1 every target is live). A flag
// is cleared by an atomic AND on its 32-bit word with the other three bytes
// kept: a random reduction without a returned value runs at about 1.5x the
// rate of a random 1-byte store here (the flag array is allocated in whole
// words). The block that finishes last (a ticket counter; every other
// block has read the round's state by then) runs round_end.
template <int S>  // the edge id of list entry p is vadj[p * S]
__global__ void __launch_bounds__(kT) k_kill(RoundArgs a) {
    __shared__ int s_last;
    DevState *st = a.st;
    const unsigned long long kp = st->kpack;
    const uint32_t ni = (uint32_t)kp;
    const uint64_t ne = kp >> 32;
    const bool check = st->round > 1;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)kT + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * kT) >> 5;
    // re-randomised rounds: round 1 leaves its working copy of the lists
    // unwritten (every entry is live), so its kill ranges are read from the
    // immutable lists, at the same positions
    const int32_t *__restrict__ vadj =
        (S == 2 && !check) ? reinterpret_cast<const int32_t *>(a.vadjE) : a.vadj;
    uint8_t *__restrict__ alive = a.alive;
    const KillItem *__restrict__ items = a.items;
    if (ni > 0 && ni <= a.item_cap) {
        const uint64_t steps = (ne + 31) / 32;
        uint64_t per = (steps + nwarps - 1) / nwarps;
        const uint64_t least = (uint64_t)(a.kill_chunk + 31) / 32;
        if (per < least) per = least;
        uint64_t q = warp * per * 32;
        const uint64_t q1 = min(ne, q + per * 32);
        if (q < q1) {
            // the item holding entry q: the largest i with items[i].ebase <= q
            uint32_t lo = 0, hi = ni - 1;
            while (lo < hi) {
                const uint32_t stride = (hi - lo) / 32 + 1;
                const uint64_t p = (uint64_t)lo + (uint64_t)lane * stride;
                const bool le = p <= hi && __ldg(&items[p].ebase) <= q;
                const unsigned bm = __ballot_sync(kFull, le);  // lane 0 always set
                lo += (uint32_t)(31 - __clz(bm)) * stride;
                hi = min(hi, lo + stride - 1);
            }
            uint32_t i = lo;
            while (q < q1) {
                const KillItem it = i + lane < ni ? items[i + lane] : KillItem{0u, 0xFFFFFFFFu};
                const uint64_t wend = (uint64_t)i + 32 < ni ? (uint64_t)__ldg(&items[i + 32].ebase) : ne;
                const uint64_t stop = min(wend, q1);
                const uint32_t e1 = __shfl_sync(kFull, it.ebase, 1);
                for (; q < stop; q += 128) {
                    // one item covers all 128 entries: no search
                    const bool one = (uint64_t)e1 >= q + 128;
                    int32_t jj[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint64_t qq = q + 32 * u + lane;
                        int k = 0;
                        if (!one) {
#pragma unroll
                            for (int d = 16; d > 0; d >>= 1) {
                                const uint32_t e = __shfl_sync(kFull, it.ebase, k + d);
                                if ((uint64_t)e <= qq) k += d;
                            }
                        }
                        const uint32_t bg = __shfl_sync(kFull, it.begin, k);
                        const uint32_t eb = __shfl_sync(kFull, it.ebase, k);
                        jj[u] = qq < stop ? __ldg(vadj + (uint64_t)(bg + (uint32_t)(qq - eb)) * S) : -1;
                    }
                    // a stale read can only show 1 for a flag another thread just
                    // cleared (flags only go 1 -> 0 here): then it is written twice
                    bool wr[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) wr[u] = jj[u] >= 0 && (!check || __ldcg(alive + jj[u]) != 0);
                    if (check) {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (wr[u])  // clear the flag byte with a reduction on its word
                                atomicAnd(reinterpret_cast<unsigned int *>(alive) + (jj[u] >> 2),
                                          ~(0xFFu << (8 * (jj[u] & 3))));
                    } else {  // round 1: every target, neighbours in the same word at once
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (wr[u]) alive[jj[u]] = 0;
                    }
                }
                q = stop;
                i += 32;
            }
        }
    } else if (ni > a.item_cap && blockIdx.x == 0 && threadIdx.x == 0) {
        st->fault = 2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&st->kdone, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        round_end(a);
    }
}

// The per-vertex state after a fixed-order match. vmatch (graphs, else
// null): the matched flags, which there stand in for T[v] = kCurMatched;
// order maps T[v] (a relabelled id) to the input id.
__global__ void k_vertex_state(const int4 *vrec, const uint8_t *vmatch, const int32_t *order, int64_t n,
                               int32_t *out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = vmatch && vmatch[v] ? kCurMatched : vrec[v].x;
        out[v] = j >= 0 ? order[j] : (j == kCurMatched ? HM_VERTEX_MATCHED : HM_VERTEX_NONE);
    }
}

// Grid of a grid-stride round kernel: exactly the blocks that fit at once.
template <typename K>
int max_blocks_per_sm(K kernel) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kT, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 4;
    }
    return per_sm;
}

// blocks per SM actually used: the request, capped to what fits (0 = all)
template <typename K>
unsigned grid_of(const Handle *h, K kernel, int want) {
    const int fit = max_blocks_per_sm(kernel);
    const int b = want > 0 && want < fit ? want : fit;
    return (unsigned)std::max(1, h->sm_count * b);
}

// The argmax kernel a handle runs: graphs read liveness from their pair lists.
void (*argmax_kernel(const Handle *h))(RoundArgs) {
    return h->graph ? k_argmax<true> : k_argmax<false>;
}

void launch_kill(const Handle *h, const RoundArgs &a, cudaStream_t s, int kill_stride) {
    if (a.pairs) k_kill<1><<<1, kT, 0, s>>>(a);  // graphs: nothing to kill, one block ends the round
    else if (kill_stride == 2) k_kill<2><<<h->kill_grid, kT, 0, s>>>(a);
    else k_kill<1><<<h->kill_grid, kT, 0, s>>>(a);
}

void launch_win_kill(const Handle *h, const RoundArgs &a, cudaStream_t s, cudaEvent_t *ev, int kill_stride) {
    if (ev) cudaEventRecord(ev[1], s);
    k_win<<<h->win_grid, kT, 0, s>>>(a);
    if (ev) cudaEventRecord(ev[2], s);
    launch_kill(h, a, s, kill_stride);
    if (ev) {  // the round end is part of the kill kernel: its span is empty
        cudaEventRecord(ev[3], s);
        cudaEventRecord(ev[4], s);
    }
}

// One round of the fixed order. ev (or null): events 0-5 of a profiled
// round; the argmax span is ev[0] - ev[5], and the untimed degree count of
// the kept vertices runs between it and the win span (ev[1] - ev[2]).
void launch_round(const Handle *h, const RoundArgs &a, cudaStream_t s, cudaEvent_t *ev) {
    if (ev) cudaEventRecord(ev[0], s);
    if (a.pairs) k_argmax<true><<<h->argmax_grid, kT, 0, s>>>(a);
    else k_argmax<false><<<h->argmax_grid, kT, 0, s>>>(a);
    if (ev) launch_kept_degrees(h, a, s, ev);
    launch_win_kill(h, a, s, ev, 1);
}


unsigned init_grid(const Handle *h) {
    return grid_for((uint64_t)std::max<int64_t>(h->m, 1), kT, h->sm_count, 16);
}

void capture_init(Handle *h, cudaStream_t s, void *ctx) {
    k_init<<<init_grid(h), kT, 0, s>>>(*static_cast<const RoundArgs *>(ctx));
}

void capture_round(Handle *h, cudaStream_t s, void *ctx) {
    launch_round(h, *static_cast<const RoundArgs *>(ctx), s, nullptr);
}

hm_status add_match_to_graph_impl(Handle *h, cudaGraph_t g) {
    cudaError_t e;
    cudaGraphConditionalHandle cond;
    if ((e = cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphConditionalHandleCreate");
    RoundArgs a = round_args(h);
    a.cond = cond;
    a.use_cond = 1;
    cudaGraphNode_t init_node = nullptr;
    hm_status st = capture_chain(h, g, capture_init, &a, &init_node);
    if (st != HM_OK) return st;
    return add_while_loop(h, g, init_node, cond, capture_round, &a);
}

hm_status build_graph(Handle *h) {
    cudaError_t e;
    if (h->exec) {
        cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
    struct G {
        cudaGraph_t g;
        ~G() { cudaGraphDestroy(g); }
    } guard{g};
    hm_status st = add_match_to_graph_impl(h, g);
    if (st != HM_OK) return st;
    if ((e = cudaGraphInstantiate(&h->exec, g, 0)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphInstantiate");
    h->graph_cap = h->cap;
    h->graph_cfg = h->cfg;
    return HM_OK;
}

}  // namespace

void launch_win_kill_end(const Handle *h, const RoundArgs &a, cudaStream_t s, cudaEvent_t *ev, int kill_stride) {
    launch_win_kill(h, a, s, ev, kill_stride);
}

void launch_live_edges(const Handle *h, const RoundArgs &a, cudaStream_t s, int random) {
    k_live_edges<<<grid_for((uint64_t)std::max<int64_t>(h->m, 1), kT, h->sm_count, 8), kT, 0, s>>>(a, random);
}

void launch_kept_degrees(const Handle *h, const RoundArgs &a, cudaStream_t s, cudaEvent_t *ev) {
    cudaEventRecord(ev[5], s);  // the end of the argmax span
    k_kept_degrees<<<grid_for((uint64_t)h->nregions * 32, kT, h->sm_count, 8), kT, 0, s>>>(a);
}

hm_status capture_chain(Handle *h, cudaGraph_t g, void (*capture)(Handle *, cudaStream_t, void *), void *ctx,
                        cudaGraphNode_t *tail) {
    cudaError_t e;
    if (!h->cap_stream) {
        e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    }
    size_t before = 0;
    if ((e = cudaGraphGetNodes(g, nullptr, &before)) != cudaSuccess) return cuda_fail(e, "graph nodes");
    std::vector<cudaGraphNode_t> old(before);
    if (before && (e = cudaGraphGetNodes(g, old.data(), &before)) != cudaSuccess)
        return cuda_fail(e, "graph nodes");
    std::sort(old.begin(), old.end());
    // captured with no dependencies: the chain is a new root of g
    if ((e = cudaStreamBeginCaptureToGraph(h->cap_stream, g, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "begin capture");
    capture(h, h->cap_stream, ctx);
    cudaGraph_t out = nullptr;
    if ((e = cudaStreamEndCapture(h->cap_stream, &out)) != cudaSuccess) return cuda_fail(e, "end capture");
    size_t nn = 0;
    if ((e = cudaGraphGetNodes(g, nullptr, &nn)) != cudaSuccess) return cuda_fail(e, "graph nodes");
    std::vector<cudaGraphNode_t> nodes(nn);
    if ((e = cudaGraphGetNodes(g, nodes.data(), &nn)) != cudaSuccess) return cuda_fail(e, "graph nodes");
    *tail = nullptr;
    int tails = 0;
    for (cudaGraphNode_t x : nodes) {
        if (std::binary_search(old.begin(), old.end(), x)) continue;
        size_t nout = 0;
        cudaGraphNodeGetDependentNodes(x, nullptr, nullptr, &nout);
        if (nout == 0) {
            *tail = x;
            ++tails;
        }
    }
    if (tails != 1) return cuda_fail(cudaErrorUnknown, "captured chain has no single end node");
    return HM_OK;
}

hm_status add_while_loop(Handle *h, cudaGraph_t g, cudaGraphNode_t after, cudaGraphConditionalHandle cond,
                         void (*body)(Handle *, cudaStream_t, void *), void *ctx) {
    cudaError_t e;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if ((e = cudaGraphAddNode(&wnode, g, &after, nullptr, 1, &cp)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphAddNode (while)");
    cudaGraph_t bg = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(h->cap_stream, bg, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "begin capture (loop body)");
    body(h, h->cap_stream, ctx);
    cudaGraph_t out = nullptr;
    if ((e = cudaStreamEndCapture(h->cap_stream, &out)) != cudaSuccess)
        return cuda_fail(e, "end capture (loop body)");
    return HM_OK;
}

RoundArgs round_args(const Handle *h) {
    RoundArgs a{};
    a.st = h->st;
    a.voff = h->voff;
    a.vadj = h->vadj;
    a.eoffj = h->eoffj;
    a.pinsj = h->pinsj;
    a.order = h->order;
    a.alive = h->alive;
    a.P = h->P;
    a.P0 = h->P0;
    a.vrec = h->vrec;
    a.firstj = h->firstj;
    a.pairs = h->graph ? 1 : 0;
    a.vpair = h->vpair;
    a.firstnbr = h->firstnbr;
    a.vmatch = h->vmatch;
    a.list0 = h->list0;
    a.list1 = h->list1;
    a.lcnt = h->lcnt;
    a.wstage = h->wstage;
    a.nregions = h->nregions;
    a.region = h->region;
    a.win = h->win;
    a.items = h->items;
    a.inM = h->inM;
    a.stats = h->stats;
    a.n = h->n;
    a.m = h->m;
    a.cap = h->cap;
    a.p16 = h->p16 ? 1 : 0;
    a.graph = h->graph ? 1 : 0;
    a.item_cap = h->item_cap;
    a.wround = h->wround;
    a.kill_chunk = h->cfg.kill_chunk;
    a.win_cap = h->win_cap;
    a.use_cond = 0;
    return a;
}

hm_status alloc_round_state(Handle *h, cudaStream_t s) {
    const uint64_t n = (uint64_t)h->n, m = (uint64_t)h->m;
    h->win_cap = std::min(n, m) + 1;
    h->item_cap = n + 1;  // one kill range per newly matched vertex
    hm_status st;
    if ((st = dalloc(&h->alive, (m + 3) / 4 * 4, s, "alive")) != HM_OK) return st;  // whole words
    if ((st = dalloc(&h->P, m, s, "P")) != HM_OK) return st;
    if ((st = dalloc(&h->P0, h->p16 ? (m + 1) / 2 : m, s, "initial P")) != HM_OK) return st;
    if (!h->vrec) {  // normally built by hm_create
        set_error("vertex records missing");
        return HM_EINVAL;
    }
    // list regions: sized for the largest argmax grid any launch config can use
    h->regions_cap = (uint32_t)(h->sm_count * max_blocks_per_sm(argmax_kernel(h)) * (kT / 32));
    h->list_cap = n + 32 * (uint64_t)h->regions_cap + 32;
    if ((st = dalloc(&h->list0, h->list_cap, s, "active list")) != HM_OK) return st;
    if ((st = dalloc(&h->list1, h->list_cap, s, "active list")) != HM_OK) return st;
    if ((st = dalloc(&h->wstage, h->list_cap, s, "winner staging")) != HM_OK) return st;
    if ((st = dalloc(&h->lcnt, 2 * (uint64_t)h->regions_cap, s, "region lengths")) != HM_OK) return st;
    if (h->edge_rounds && (st = dalloc(&h->wround, m, s, "win rounds")) != HM_OK) return st;
    if ((st = dalloc(&h->win, h->win_cap, s, "winners")) != HM_OK) return st;
    if ((st = dalloc(&h->items, h->item_cap, s, "kill items")) != HM_OK) return st;
    if ((st = dalloc(&h->inM, m, s, "result mask")) != HM_OK) return st;
    if (h->graph && (st = dalloc(&h->vmatch, n, s, "matched flags")) != HM_OK) return st;
    if ((st = apply_config(h, h->cfg)) != HM_OK) return st;
    if (m) {
        RoundArgs a = round_args(h);
        k_p0<<<grid_for(m, kT, h->sm_count, 16), kT, 0, s>>>(a, h->P0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "initial P");
    }
    if ((st = dalloc(&h->stats, (uint64_t)kStatRounds * HM_STATS_COLS, s, "round stats")) != HM_OK) return st;
    if ((st = dalloc(&h->st, 1, s, "loop state")) != HM_OK) return st;
    if ((st = dalloc(&h->res_idx, m, s, "result ids")) != HM_OK) return st;
    if ((st = dalloc(&h->res_w, m, s, "result weights")) != HM_OK) return st;
    if ((st = dalloc(&h->res_part, compact_scratch_elems(m) + 1, s, "result scratch")) != HM_OK) return st;
    if ((st = dalloc(&h->res_bucket, 256, s, "result weight buckets")) != HM_OK) return st;
    cudaError_t e = cudaMemsetAsync(h->stats, 0, (size_t)kStatRounds * HM_STATS_COLS * sizeof(int64_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "stats reset");
    h->h_st = new (std::nothrow) DevState();
    if (!h->h_st) {
        set_error("out of host memory");
        return HM_ENOMEM;
    }
    return HM_OK;
}

hm_status apply_config(Handle *h, const LaunchConfig &c) {
    if (c.kill_chunk < kMinKillChunk || c.kill_chunk > (1 << 20) || c.argmax_bpsm < 0 || c.win_bpsm < 0 ||
        c.kill_bpsm < 0) {
        set_error("launch config out of range");
        return HM_EINVAL;
    }
    h->cfg = c;
    h->argmax_grid = grid_of(h, argmax_kernel(h), c.argmax_bpsm);
    h->win_grid = grid_of(h, k_win, c.win_bpsm);
    h->kill_grid = grid_of(h, k_kill<1>, c.kill_bpsm);
    h->nregions = h->argmax_grid * (kT / 32);
    if (h->nregions > h->regions_cap) h->nregions = h->regions_cap;
    const uint64_t n = (uint64_t)h->n;
    h->region = (uint32_t)((((n + h->nregions - 1) / h->nregions) + 31) / 32 * 32);
    if (h->region == 0) h->region = 32;
    return HM_OK;
}

hm_status add_match_to_graph(Handle *h, cudaGraph_t g) { return add_match_to_graph_impl(h, g); }

hm_status launch_match_graph(Handle *h, cudaStream_t s) {
    if (!h->exec || h->graph_cap != h->cap || !(h->graph_cfg == h->cfg)) {
        hm_status st = build_graph(h);
        if (st != HM_OK) return st;
    }
    cudaError_t e = cudaGraphLaunch(h->exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return HM_OK;
}

hm_status profile_match(Handle *h, cudaStream_t s, double *ms, int64_t *launches, double *round_ms,
                        int32_t max_rounds) {
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
    RoundArgs a = round_args(h);
    float t = 0;
    cudaEventRecord(ev[5], s);
    k_init<<<init_grid(h), kT, 0, s>>>(a);
    cudaEventRecord(ev[0], s);
    cudaError_t e = cudaEventSynchronize(ev[0]);
    if (e != cudaSuccess) return cuda_fail(e, "profile init");
    cudaEventElapsedTime(&t, ev[5], ev[0]);
    ms[HM_K_INIT] += t;
    launches[HM_K_INIT] += 1;
    for (int32_t r = 0;; ++r) {
        launch_live_edges(h, a, s, 0);  // untimed: before the round's first event
        launch_round(h, a, s, ev);
        cudaMemcpyAsync(h->h_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "profile round");
        for (int k = 0; k < 4; ++k) {
            cudaEventElapsedTime(&t, ev[k], k == 0 ? ev[5] : ev[k + 1]);
            ms[HM_K_ARGMAX + k] += t;
            launches[HM_K_ARGMAX + k] += k == 3 ? 0 : 1;  // the round end is part of the kill kernel
            if (r < max_rounds) round_ms[(int64_t)r * 4 + k] = t;
        }
        if (h->h_st->finished) break;
    }
    cudaEventRecord(h->done, s);
    return HM_OK;
}

// Median CUDA-event time of `reps` graph launches of h's match under config c.
static hm_status time_config(Handle *h, cudaStream_t s, const LaunchConfig &c, int reps, double *ms) {
    hm_status st = apply_config(h, c);
    if (st != HM_OK) return st;
    if ((st = launch_match_graph(h, s)) != HM_OK) return st;  // rebuild + warm-up
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<float> t;
    for (int r = 0; r < reps && st == HM_OK; ++r) {
        cudaEventRecord(e0, s);
        st = launch_match_graph(h, s);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) st = cuda_fail(e, "autotune");
        float x = 0;
        cudaEventElapsedTime(&x, e0, e1);
        t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HM_OK) return st;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return HM_OK;
}

hm_status autotune(Handle *h, cudaStream_t s, LaunchConfig *best, double *best_ms) {
    LaunchConfig cur = h->cfg;
    double cur_ms = 0;
    hm_status st = time_config(h, s, cur, 3, &cur_ms);
    if (st != HM_OK) return st;
    auto consider = [&](LaunchConfig c) -> hm_status {
        if (c == cur) return HM_OK;
        double ms = 0;
        hm_status r = time_config(h, s, c, 3, &ms);
        if (r != HM_OK) return r;
        if (ms < cur_ms) {
            cur = c;
            cur_ms = ms;
        }
        return HM_OK;
    };
    const int fit_arg = max_blocks_per_sm(argmax_kernel(h));
    for (int pass = 0; pass < 2 && st == HM_OK; ++pass) {
        for (int chunk : {64, 128, 256, 512, 1024}) {
            LaunchConfig c = cur;
            c.kill_chunk = chunk;
            if ((st = consider(c)) != HM_OK) return st;
        }
        for (int b = fit_arg; b >= std::max(1, fit_arg - 3); --b) {
            LaunchConfig c = cur;
            c.argmax_bpsm = b == fit_arg ? 0 : b;
            if ((st = consider(c)) != HM_OK) return st;
        }
        for (int b : {0, 4, 2}) {
            LaunchConfig c = cur;
            c.win_bpsm = b;
            if ((st = consider(c)) != HM_OK) return st;
        }
        for (int b : {0, 4, 2}) {
            LaunchConfig c = cur;
            c.kill_bpsm = b;
            if ((st = consider(c)) != HM_OK) return st;
        }
    }
    if ((st = apply_config(h, cur)) != HM_OK) return st;
    *best = cur;
    *best_ms = cur_ms;
    return HM_OK;
}

cudaError_t launch_vertex_state(const Handle *h, int32_t *out_dev, cudaStream_t s) {
    if (h->last_random) return launch_rand_vertex_state(h, out_dev, s);
    const int4 *vrec = h->vrec;
    const uint8_t *vmatch = h->vmatch;  // graphs (both orders): the matched flags
    k_vertex_state<<<grid_for((uint64_t)h->n, kT, h->sm_count, 16), kT, 0, s>>>(vrec, vmatch, h->order, h->n,
                                                                               out_dev);
    return cudaGetLastError();
}

// Stream-ordered frees on the handle's own stream: cudaFree would wait for
// the whole device, stalling every other stream (other handles, requests).
void free_handle_buffers(Handle *h) {
    free_rand_buffers(h);
    void *bufs[] = {h->voff, h->vadj, h->eoffj, h->pinsj, h->order, h->weights, h->alive, h->P, h->P0,
                    h->vrec, h->firstj, h->vpair, h->firstnbr, h->vmatch, h->list0, h->list1, h->lcnt, h->wstage, h->wround, h->win,
                    h->items, h->inM, h->stats, h->st, h->res_idx, h->res_w, h->res_part, h->res_bucket};
    cudaStream_t s = h->cap_stream;
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, s);
    if (s) cudaStreamSynchronize(s);
    delete h->h_st;
    h->h_st = nullptr;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->done) cudaEventDestroy(h->done);
}

}  // namespace hm
