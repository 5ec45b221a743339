// create.cu - builds a handle's device structures from the edge CSR.
//
//  1. validate the input (Sec. 2.1: edges are non-empty vertex sets, weights
//     are positive reals);
//  2. fix the strict order on edges and relabel edges by decreasing priority
//     (j = 0 is the best edge): a stable radix sort of the complemented
//     32-bit priority over edges taken in increasing id, so equal priorities
//     keep the smaller id first;
//  3. copy the pins into j order (E_id/E_p of Sec. 4.1);
//  4. build the vertex CSR (V_id/V_p of Sec. 4.1) by a stable radix sort of
//     the (vertex, j) pairs by vertex: every vertex's list comes out in
//     ascending j, i.e. decreasing priority, which turns the per-vertex argmax
//     of every round (Alg. 1 / Alg. 3) into a forward-only cursor. A vertex
//     repeated inside an edge shows up as two equal neighbours in that list.
#include "hm_internal.cuh"

#include <algorithm>
#include <cstdio>

namespace hm {
namespace {

constexpr int kT = 256;

enum : uint32_t { kErrEdgeRange = 1u, kErrPin = 2u, kErrWeight = 4u, kErrDup = 8u };

struct CreateErr {
    uint32_t flags;
    uint32_t pad;
    unsigned long long first[4];  // first offending index per error kind
    unsigned long long max_size;  // largest edge size
};

__device__ __forceinline__ void report(CreateErr *err, uint32_t kind, int bit, unsigned long long idx) {
    atomicOr(&err->flags, kind);
    atomicMin(&err->first[bit], idx);
}

__device__ __forceinline__ void check_pin(int32_t p, int64_t n, uint64_t i, CreateErr *err) {
    if (p < 0 || (int64_t)p >= n) report(err, kErrPin, 1, i);
}

// Sec. 2.1: every edge is a non-empty set, weights are positive. Also
// finds the largest edge size (it decides the width of the P counters).
// Pins are read 16 bytes at a time when the array is 16-byte aligned.
__global__ void k_validate(const int64_t *__restrict__ eoff, const int32_t *__restrict__ pins,
                           const float *__restrict__ w, int64_t n, int64_t m, uint64_t kappa,
                           CreateErr *err) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long mx = 0;
    for (uint64_t i = tid; i < (uint64_t)m; i += nth) {
        const int64_t sz = eoff[i + 1] - eoff[i];
        if (sz <= 0) report(err, kErrEdgeRange, 0, i);
        else if ((unsigned long long)sz > mx) mx = (unsigned long long)sz;
        if (w) {
            const uint32_t b = __float_as_uint(w[i]);
            // finite and > 0: sign clear, not zero, exponent below all-ones
            if (b == 0u || b >= 0x7F800000u) report(err, kErrWeight, 2, i);
        }
    }
    uint64_t done = 0;
    if ((reinterpret_cast<uintptr_t>(pins) & 15u) == 0) {
        const uint64_t n4 = kappa / 4;
        const int4 *p4 = reinterpret_cast<const int4 *>(pins);
        for (uint64_t q = tid; q < n4; q += nth) {
            const int4 x = __ldg(p4 + q);
            check_pin(x.x, n, 4 * q, err);
            check_pin(x.y, n, 4 * q + 1, err);
            check_pin(x.z, n, 4 * q + 2, err);
            check_pin(x.w, n, 4 * q + 3, err);
        }
        done = 4 * n4;
    }
    for (uint64_t i = done + tid; i < kappa; i += nth) check_pin(__ldg(pins + i), n, i, err);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, d);
        if (y > mx) mx = y;
    }
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(&err->max_size, mx);
}

// Sort key = complemented priority (ascending sort = decreasing priority).
// Positive finite floats order like their bit patterns. For a union of
// independent instances (inst_ebase != nullptr: first edge of each of the
// ninst instances) the hash priority uses the edge's id inside its own
// instance, so every instance is ordered exactly as it would be alone.
__global__ void k_priority(const float *__restrict__ w, uint32_t salt, int64_t m,
                           const int64_t *__restrict__ inst_ebase, int32_t ninst,
                           uint32_t *__restrict__ key, uint32_t *__restrict__ val) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t local = e;
        if (!w && inst_ebase) {
            int lo = 0, hi = ninst - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (inst_ebase[mid] <= e) lo = mid; else hi = mid - 1;
            }
            local = e - inst_ebase[lo];
        }
        const uint32_t prio = w ? __float_as_uint(w[e]) : fmix32((uint32_t)local ^ salt);
        key[e] = ~prio;
        val[e] = (uint32_t)e;
    }
}

// Size and first input pin of every edge, in j order.
__global__ void k_sizes_j(const int64_t *__restrict__ eoff, const uint32_t *__restrict__ order,
                          int64_t m, int64_t *__restrict__ szj, int64_t *__restrict__ srcj) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = order[j];
        const int64_t b = eoff[e];
        szj[j] = eoff[e + 1] - b;
        srcj[j] = b;
    }
}

// Pins of input edge order[j] -> pinsj[eoffj[j] ..]; the same slots of
// jval receive j. Output-driven: a block fills kRelTile consecutive output
// slots, loads the offsets of exactly the edges covering them (first[t] is
// the edge containing the tile's first slot) and where their pins start in
// the input (srcj), locates each slot's edge by binary search in shared
// memory, and writes both outputs coalesced whatever the edge sizes. One
// tile per block: the GPU keeps many tiles' dependent loads in flight.
constexpr int kRelTile = kRelabelTile;

// first[t] = the edge that contains output slot t*kRelTile.
__global__ void k_tile_first(const int64_t *__restrict__ eoffj, int64_t m, uint64_t ntiles,
                             int32_t *__restrict__ first) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t b = (uint64_t)eoffj[j], e = (uint64_t)eoffj[j + 1];
        for (uint64_t t = (b + kRelTile - 1) / kRelTile; t * kRelTile < e && t < ntiles; ++t)
            first[t] = (int32_t)j;
    }
}

__global__ void __launch_bounds__(kT) k_relabel(const int32_t *__restrict__ pins, const int64_t *__restrict__ srcj,
                                               const int64_t *__restrict__ eoffj, const int32_t *__restrict__ first,
                                               int64_t m, uint64_t kappa, uint64_t ntiles,
                                               int32_t *__restrict__ pinsj, uint32_t *__restrict__ jval) {
    __shared__ int64_t s_off[kRelTile + 1];  // eoffj of the tile's edges
    __shared__ int64_t s_src[kRelTile];      // their first input pin
    const uint64_t t = blockIdx.x;
    if (t >= ntiles) return;
    const uint64_t p0 = t * kRelTile;
    const uint64_t p1 = p0 + kRelTile < kappa ? p0 + kRelTile : kappa;
    const int64_t j0 = first[t];
    const int64_t j1 = t + 1 < ntiles ? first[t + 1] : m - 1;  // last edge touching the tile
    const int ne = (int)(j1 - j0 + 1);                          // <= kRelTile + 1
    for (int k = threadIdx.x; k <= ne && k <= kRelTile; k += kT) {
        s_off[k] = eoffj[j0 + k];
        if (k < ne && k < kRelTile) s_src[k] = srcj[j0 + k];
    }
    __syncthreads();
    const int hi0 = (ne < kRelTile ? ne : kRelTile) - 1;
    for (uint64_t p = p0 + threadIdx.x; p < p1; p += kT) {
        int lo = 0, hi = hi0;  // last k with s_off[k] <= p
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((uint64_t)s_off[mid] <= p) lo = mid; else hi = mid - 1;
        }
        pinsj[p] = pins[s_src[lo] + (int64_t)(p - (uint64_t)s_off[lo])];
        jval[p] = (uint32_t)(j0 + lo);
    }
}

// Input-driven relabel of the pin tiles [t0, t1) (tiles of kRelTile
// consecutive INPUT pins, first[t] = the input edge holding the tile's
// first pin): a block loads the input offsets of the tile's edges and, per
// edge, its relabelled id j and the first slot of its pins in j order, then
// writes every pin to its slot. A block reads only its own tile, so the
// tiles can run as soon as their pins have arrived. Pins outside [0, n) are
// reported (and written; the build stops before anything indexes by them).
__global__ void __launch_bounds__(kT) k_relabel_in(const int32_t *__restrict__ pins, const int64_t *__restrict__ eoff,
                                                  const int32_t *__restrict__ jof,
                                                  const int64_t *__restrict__ eoffj,
                                                  const int32_t *__restrict__ first, int64_t m, int64_t n,
                                                  uint64_t kappa, uint64_t ntiles, uint64_t t0,
                                                  int32_t *__restrict__ pinsj, uint32_t *__restrict__ jval,
                                                  CreateErr *err) {
    __shared__ int64_t s_off[kRelTile + 1];  // input offsets of the tile's edges
    __shared__ int64_t s_dst[kRelTile];      // their first slot in j order
    __shared__ int32_t s_j[kRelTile];        // their relabelled ids
    const uint64_t t = t0 + blockIdx.x;
    if (t >= ntiles) return;
    const uint64_t p0 = t * kRelTile;
    const uint64_t p1 = p0 + kRelTile < kappa ? p0 + kRelTile : kappa;
    const int64_t e0 = first[t];
    const int64_t e1 = t + 1 < ntiles ? first[t + 1] : m - 1;  // last edge touching the tile
    const int ne = (int)(e1 - e0 + 1);                          // <= kRelTile + 1
    for (int k = threadIdx.x; k <= ne && k <= kRelTile; k += kT) {
        s_off[k] = eoff[e0 + k];
        if (k < ne && k < kRelTile) {
            const int32_t j = __ldg(jof + e0 + k);
            s_j[k] = j;
            s_dst[k] = __ldg(eoffj + j);
        }
    }
    __syncthreads();
    const int hi0 = (ne < kRelTile ? ne : kRelTile) - 1;
    for (uint64_t p = p0 + threadIdx.x; p < p1; p += kT) {
        int lo = 0, hi = hi0;  // last k with s_off[k] <= p
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((uint64_t)s_off[mid] <= p) lo = mid; else hi = mid - 1;
        }
        const int32_t v = pins[p];
        if (v < 0 || (int64_t)v >= n) report(err, kErrPin, 1, p);
        const int64_t slot = s_dst[lo] + (int64_t)(p - (uint64_t)s_off[lo]);
        pinsj[slot] = v;
        jval[slot] = (uint32_t)s_j[lo];
    }
}

// jof[order[j]] = j: the relabelled id of every input edge.
__global__ void k_inverse(const uint32_t *__restrict__ order, int64_t m, int32_t *__restrict__ jof) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        jof[order[j]] = (int32_t)j;
}

// d = 2: edge j's pins are the pair of input edge order[j]; eoffj[j] = 2j.
__global__ void k_relabel_pairs(const int32_t *__restrict__ pins, const uint32_t *__restrict__ order, int64_t m,
                                int64_t *__restrict__ eoffj, int32_t *__restrict__ pinsj, uint32_t *__restrict__ jval) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= m;
         j += (int64_t)gridDim.x * blockDim.x) {
        eoffj[j] = 2 * j;
        if (j == m) continue;
        const int64_t e = order[j];
        const int32_t a = __ldg(pins + 2 * e), b = __ldg(pins + 2 * e + 1);
        reinterpret_cast<int2 *>(pinsj)[j] = make_int2(a, b);
        reinterpret_cast<uint2 *>(jval)[j] = make_uint2((uint32_t)j, (uint32_t)j);
    }
}

// voff from the vertex-sorted pin list: position i starts the segments of
// the vertices (sv[i-1], sv[i]] (degree-0 vertices get empty segments).
// firstj[v] = the first entry of v's list (or -2 for degree 0). Also flags a
// vertex repeated inside one edge (equal (v, j) neighbours). Four positions
// per thread, read 16 bytes at a time.
__device__ __forceinline__ void voff_at(uint64_t i, uint32_t prev_v, uint32_t v, uint32_t prev_j, uint32_t j,
                                        uint64_t kappa, int64_t n, int64_t *__restrict__ voff,
                                        int32_t *__restrict__ firstj, CreateErr *err) {
    const int64_t lo = i == 0 ? 0 : (int64_t)prev_v + 1;
    const int64_t hi = i == kappa ? n : (int64_t)v;
    for (int64_t x = lo; x <= hi; ++x) {
        voff[x] = (int64_t)i;
        if (x < n) firstj[x] = (x == hi && i < kappa) ? (int32_t)j : -2;
    }
    if (i > 0 && i < kappa && v == prev_v && j == prev_j) report(err, kErrDup, 3, i);
}

__global__ void k_voff(const uint32_t *__restrict__ sv, const uint32_t *__restrict__ vadj,
                       uint64_t kappa, int64_t n, int64_t *__restrict__ voff,
                       int32_t *__restrict__ firstj, CreateErr *err) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n4 = kappa / 4;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(sv);
    const uint4 *a4 = reinterpret_cast<const uint4 *>(vadj);
    for (uint64_t q = tid; q < n4; q += nth) {
        const uint4 v = __ldg(s4 + q), j = __ldg(a4 + q);
        const uint32_t pv = q ? __ldg(sv + 4 * q - 1) : 0u, pj = q ? __ldg(vadj + 4 * q - 1) : 0u;
        voff_at(4 * q, pv, v.x, pj, j.x, kappa, n, voff, firstj, err);
        voff_at(4 * q + 1, v.x, v.y, j.x, j.y, kappa, n, voff, firstj, err);
        voff_at(4 * q + 2, v.y, v.z, j.y, j.z, kappa, n, voff, firstj, err);
        voff_at(4 * q + 3, v.z, v.w, j.z, j.w, kappa, n, voff, firstj, err);
    }
    for (uint64_t i = 4 * n4 + tid; i <= kappa; i += nth) {
        const uint32_t pv = i ? sv[i - 1] : 0u, pj = i ? vadj[i - 1] : 0u;
        const uint32_t v = i < kappa ? sv[i] : 0u, j = i < kappa ? vadj[i] : 0u;
        voff_at(i, pv, v, pj, j, kappa, n, voff, firstj, err);
    }
}

// Constant half of the per-vertex record: list start and degree (the
// mutable half, T[v] and its cursor, is reset by every match). Graphs keep
// {T[v], cursor, list end, other endpoint of T[v]}, all rewritten by round 1.
__global__ void k_vrec_meta(const int64_t *__restrict__ voff, int64_t n, int graph, int4 *__restrict__ vrec,
                            int32_t *__restrict__ firstnbr) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = voff[v], e = voff[v + 1];
        if (graph) {
            vrec[v] = make_int4(-2, (int32_t)(uint32_t)b, (int32_t)(uint32_t)e, -1);
            if (e == b) firstnbr[v] = -1;
        } else {
            vrec[v] = make_int4(-2, 0, (int32_t)(uint32_t)b, (int32_t)(uint32_t)(e - b));
        }
    }
}

// Graphs: each list entry with the other endpoint of its edge (vertex key[p]
// owns entry p, edge vadj[p] has pins pinsj[2j], pinsj[2j + 1]), and that
// endpoint for every list's first entry.
__global__ void k_pairs_nbr(const uint32_t *__restrict__ key, const int32_t *__restrict__ vadj,
                            const int32_t *__restrict__ pinsj, uint64_t kappa, int2 *__restrict__ vpair,
                            int32_t *__restrict__ firstnbr) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < kappa;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = key[p];
        const int32_t j = vadj[p];
        const int2 e = __ldg(reinterpret_cast<const int2 *>(pinsj) + j);
        const int32_t o = (uint32_t)e.x == v ? e.y : e.x;
        vpair[p] = make_int2(j, o);
        if (p == 0 || key[p - 1] != v) firstnbr[v] = o;
    }
}

template <typename T>
void dfree(T *&p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
}

int bit_width(uint64_t x) {
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

}  // namespace

// Frees every registered temporary (stream-ordered) when it goes out of scope.
struct Temps {
    cudaStream_t s;
    void *p[16] = {};
    int k = 0;
    explicit Temps(cudaStream_t st) : s(st) {}
    template <typename T>
    hm_status get(T **out, uint64_t count, const char *what) {
        hm_status st = dalloc(out, count, s, what);
        if (st == HM_OK) p[k++] = *out;
        return st;
    }
    template <typename T>
    void drop(T *&q) {
        for (int i = 0; i < k; ++i)
            if (p[i] == q) {
                cudaFreeAsync(p[i], s);
                p[i] = nullptr;
            }
        q = nullptr;
    }
    ~Temps() {
        for (int i = 0; i < k; ++i)
            if (p[i]) cudaFreeAsync(p[i], s);
    }
};

hm_status create_structures(Handle *h, const int64_t *eoff, const int32_t *pins,
                            const float *weights, cudaStream_t s, const int64_t *inst_ebase,
                            int32_t ninst, const PinChunks *feed) {
    const int64_t n = h->n, m = h->m;
    const uint64_t kappa = h->kappa;
    struct Events {
        cudaEvent_t e[5] = {};
        ~Events() {
            for (auto &x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    for (auto &e : ev.e)
        if (cudaEventCreate(&e) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaEventCreate");

    Temps tmp(s);
    hm_status st;
    const uint64_t big = std::max<uint64_t>((uint64_t)m, kappa);
    const unsigned gbig = grid_for(big, kT, h->sm_count, 16);
    const unsigned gm = grid_for((uint64_t)m, kT, h->sm_count, 16);

    CreateErr *derr = nullptr;
    if ((st = tmp.get(&derr, 1, "error word")) != HM_OK) return st;
    CreateErr init{};
    init.first[0] = init.first[1] = init.first[2] = init.first[3] = ~0ull;
    CreateErr herr{};
    cudaEventRecord(ev.e[0], s);
    cudaError_t ce = cudaMemcpyAsync(derr, &init, sizeof init, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "error word upload");

    // 1. validation (the pins later, when they are still arriving)
    k_validate<<<gbig, kT, 0, s>>>(eoff, feed ? nullptr : pins, h->weighted ? weights : nullptr, n, m,
                                   feed ? 0 : kappa, derr);
    cudaMemcpyAsync(&herr, derr, sizeof herr, cudaMemcpyDeviceToHost, s);
    ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_fail(ce, "validation");
    if (herr.flags) {
        char buf[200];
        if (herr.flags & kErrEdgeRange)
            snprintf(buf, sizeof buf,
                     "eoff is not strictly increasing at edge %llu (empty or decreasing edge)",
                     herr.first[0]);
        else if (herr.flags & kErrPin)
            snprintf(buf, sizeof buf, "pin at position %llu is outside [0, n)", herr.first[1]);
        else
            snprintf(buf, sizeof buf, "weight of edge %llu is not finite and > 0", herr.first[2]);
        set_error(buf);
        return HM_EINVAL;
    }
    h->p16 = herr.max_size <= 0xFFFFull;
    // sizes are >= 1 (validated), so kappa = 2m with none above 2 means all are 2
    h->graph = m > 0 && herr.max_size == 2 && kappa == 2 * (uint64_t)m;
    cudaEventRecord(ev.e[1], s);

    // 2. order on edges: stable sort of ~priority over edges in id order
    uint32_t *key = nullptr, *val = nullptr, *tk = nullptr, *tv = nullptr, *sk = nullptr,
             *order_u = nullptr, *rscratch = nullptr;
    if ((st = tmp.get(&key, big, "sort keys")) != HM_OK ||
        (st = tmp.get(&val, big, "sort values")) != HM_OK ||
        (st = tmp.get(&tk, big, "sort keys (alt)")) != HM_OK ||
        (st = tmp.get(&tv, big, "sort values (alt)")) != HM_OK ||
        (st = tmp.get(&sk, (uint64_t)m, "sorted priorities")) != HM_OK ||
        (st = tmp.get(&rscratch, radix_scratch_elems(big), "sort scratch")) != HM_OK ||
        (st = dalloc(&order_u, (uint64_t)m, s, "order")) != HM_OK)
        return st;
    h->order = (int32_t *)order_u;  // owned by the handle from here on
    const uint32_t salt = (uint32_t)splitmix64_first(h->seed);
    k_priority<<<gm, kT, 0, s>>>(h->weighted ? weights : nullptr, salt, m, inst_ebase, ninst, key, val);
    ce = radix_sort_pairs(key, val, sk, order_u, tk, tv, (uint64_t)m, 32, rscratch, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "priority sort");
    tmp.drop(sk);
    cudaEventRecord(ev.e[2], s);

    // 3. edge CSR in j order
    if ((st = dalloc(&h->eoffj, (uint64_t)m + 1, s, "eoffj")) != HM_OK ||
        (st = dalloc(&h->pinsj, kappa, s, "pinsj")) != HM_OK)
        return st;
    if (feed && h->graph) {
        // d = 2: an edge holds only two pins, so relabelling as the chunks
        // arrive would cost two random reads per pair; gather the pairs once
        // every chunk is in, after checking the pins
        for (int c = 0; c < feed->chunks; ++c) cudaStreamWaitEvent(s, feed->ev[c], 0);
        if (kappa) k_validate<<<gbig, kT, 0, s>>>(eoff, pins, nullptr, n, 0, kappa, derr);
        cudaMemcpyAsync(&herr, derr, sizeof herr, cudaMemcpyDeviceToHost, s);
        ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return cuda_fail(ce, "pin validation");
        if (herr.flags & kErrPin) {
            char buf[200];
            snprintf(buf, sizeof buf, "pin at position %llu is outside [0, n)", herr.first[1]);
            set_error(buf);
            return HM_EINVAL;
        }
        k_relabel_pairs<<<gm, kT, 0, s>>>(pins, order_u, m, h->eoffj, h->pinsj, val);
    } else if (feed) {
        // edge offsets in j order, the inverse order, the input tiles' first
        // edges; then every chunk of pins is relabelled once it has arrived
        {
            int64_t *szj = nullptr, *srcj = nullptr, *i64scratch = nullptr;
            if ((st = tmp.get(&szj, (uint64_t)m, "edge sizes")) != HM_OK ||
                (st = tmp.get(&srcj, (uint64_t)m, "edge sources")) != HM_OK ||
                (st = tmp.get(&i64scratch, scan_scratch_elems((uint64_t)m), "scan scratch")) != HM_OK)
                return st;
            k_sizes_j<<<gm, kT, 0, s>>>(eoff, order_u, m, szj, srcj);
            ce = exclusive_scan_i64(szj, h->eoffj, (uint64_t)m, h->eoffj + m, i64scratch, s);
            if (ce != cudaSuccess) return cuda_fail(ce, "edge offsets");
            tmp.drop(szj);
            tmp.drop(srcj);
            tmp.drop(i64scratch);
        }
        const uint64_t ntiles = (kappa + kRelTile - 1) / kRelTile;
        int32_t *jof = nullptr, *first = nullptr;
        if ((st = tmp.get(&jof, (uint64_t)m, "inverse order")) != HM_OK ||
            (st = tmp.get(&first, ntiles, "relabel tiles")) != HM_OK)
            return st;
        k_inverse<<<gm, kT, 0, s>>>(order_u, m, jof);
        k_tile_first<<<gm, kT, 0, s>>>(eoff, m, ntiles, first);
        for (int c = 0; c < feed->chunks; ++c) {
            cudaStreamWaitEvent(s, feed->ev[c], 0);
            const uint64_t ta = feed->begin[c] / kRelTile;
            const uint64_t tb = (feed->begin[c + 1] + kRelTile - 1) / kRelTile;
            if (tb > ta)
                k_relabel_in<<<(unsigned)(tb - ta), kT, 0, s>>>(pins, eoff, jof, h->eoffj, first, m, n, kappa,
                                                                 ntiles, ta, h->pinsj, val, derr);
        }
        tmp.drop(jof);
        tmp.drop(first);
        // the pins must be valid before the vertex CSR indexes by them
        cudaMemcpyAsync(&herr, derr, sizeof herr, cudaMemcpyDeviceToHost, s);
        ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return cuda_fail(ce, "relabel");
        if (herr.flags & kErrPin) {
            char buf[200];
            snprintf(buf, sizeof buf, "pin at position %llu is outside [0, n)", herr.first[1]);
            set_error(buf);
            return HM_EINVAL;
        }
    } else if (h->graph) {
        // d = 2: offsets 2j, each edge's pair gathered in one 8-byte load;
        // val receives j for both pin slots (pinsj and val: 8-byte aligned)
        k_relabel_pairs<<<gm, kT, 0, s>>>(pins, order_u, m, h->eoffj, h->pinsj, val);
    } else {
        int64_t *szj = nullptr, *srcj = nullptr, *i64scratch = nullptr;
        if ((st = tmp.get(&szj, (uint64_t)m, "edge sizes")) != HM_OK ||
            (st = tmp.get(&srcj, (uint64_t)m, "edge sources")) != HM_OK ||
            (st = tmp.get(&i64scratch, scan_scratch_elems((uint64_t)m), "scan scratch")) != HM_OK)
            return st;
        k_sizes_j<<<gm, kT, 0, s>>>(eoff, order_u, m, szj, srcj);
        ce = exclusive_scan_i64(szj, h->eoffj, (uint64_t)m, h->eoffj + m, i64scratch, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "edge offsets");
        tmp.drop(szj);
        tmp.drop(i64scratch);
        // val receives j for every pin slot; the relabelled pins double as
        // the keys of the vertex sort
        const uint64_t ntiles = (kappa + kRelTile - 1) / kRelTile;
        int32_t *first = nullptr;
        if ((st = tmp.get(&first, ntiles, "relabel tiles")) != HM_OK) return st;
        k_tile_first<<<gm, kT, 0, s>>>(h->eoffj, m, ntiles, first);
        if (ntiles > 0)
            k_relabel<<<(unsigned)ntiles, kT, 0, s>>>(pins, srcj, h->eoffj, first, m, kappa, ntiles, h->pinsj, val);
        tmp.drop(first);
        tmp.drop(srcj);
    }
    cudaEventRecord(ev.e[3], s);

    // 4. vertex CSR: stable sort of (v, j) by v; keys land in `key`, values in vadj
    if ((st = dalloc(&h->vadj, kappa, s, "vadj")) != HM_OK ||
        (st = dalloc(&h->voff, (uint64_t)n + 1, s, "voff")) != HM_OK ||
        (st = dalloc(&h->firstj, (uint64_t)n, s, "first entries")) != HM_OK ||
        (st = dalloc(&h->vrec, (uint64_t)n, s, "vertex records")) != HM_OK)
        return st;
    if (h->graph && ((st = dalloc(&h->vpair, kappa, s, "list pairs")) != HM_OK ||
                     (st = dalloc(&h->firstnbr, (uint64_t)n, s, "first neighbours")) != HM_OK))
        return st;
    const int vbits = bit_width(n > 0 ? (uint64_t)(n - 1) : 0);
    ce = radix_sort_pairs((const uint32_t *)h->pinsj, val, key, (uint32_t *)h->vadj, tk, tv, kappa,
                          vbits, rscratch, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "vertex sort");
    k_voff<<<grid_for(kappa + 1, kT, h->sm_count, 16), kT, 0, s>>>(key, (const uint32_t *)h->vadj,
                                                                  kappa, n, h->voff, h->firstj, derr);
    if (h->graph && kappa)
        k_pairs_nbr<<<grid_for(kappa, kT, h->sm_count, 16), kT, 0, s>>>(key, h->vadj, h->pinsj, kappa, h->vpair,
                                                                       h->firstnbr);
    k_vrec_meta<<<grid_for((uint64_t)n, kT, h->sm_count, 16), kT, 0, s>>>(h->voff, n, h->graph ? 1 : 0, h->vrec,
                                                                         h->firstnbr);
    cudaEventRecord(ev.e[4], s);
    cudaMemcpyAsync(&herr, derr, sizeof herr, cudaMemcpyDeviceToHost, s);
    ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_fail(ce, "vertex CSR");
    if (herr.flags & kErrDup) {
        char buf[160];
        snprintf(buf, sizeof buf,
                 "duplicate pin: a vertex appears twice in one edge (vertex-sorted position %llu)",
                 herr.first[3]);
        set_error(buf);
        return HM_EINVAL;
    }
    float ms = 0;
    for (int i = 0; i < 4; ++i) {
        cudaEventElapsedTime(&ms, ev.e[i], ev.e[i + 1]);
        h->create_ms[i] = ms;
    }
    cudaEventElapsedTime(&ms, ev.e[0], ev.e[4]);
    h->create_ms[4] = ms;

    // weights in input numbering, for the result weight
    if (h->weighted) {
        if ((st = dalloc(&h->weights, (uint64_t)m, s, "weights")) != HM_OK) return st;
        ce = cudaMemcpyAsync(h->weights, weights, (size_t)m * sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "weights copy");
    }
    return HM_OK;
}

}  // namespace hm
