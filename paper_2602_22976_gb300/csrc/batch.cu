// batch.cu - many independent hypergraphs matched by one graph launch.
//
// Instances are grouped into size classes (by kappa, factors of four). Each
// class becomes one handle over the disjoint union of its instances: vertex
// and edge ids are offset per instance, so no two instances share a vertex
// and the round loop of Sec. 3.1 runs on all of them at once without any
// interaction. Hash priorities use instance-local edge ids and weight ties
// keep the smaller local id first, so every instance gets exactly the
// matching and round count it would get alone; an instance's round count is
// the round in which its last edge joined the matching.
//
// All classes' loops are independent branches of one CUDA graph, so classes
// in their latency-bound last rounds overlap the work of others. Each class
// has its own launch shape, optionally picked by the autotuner.
//
// A class of small instances (every instance below kSmallClassPins pins) is
// not run as a union round loop: a persistent kernel of one-block workers
// takes its instances one at a time from a counter and matches each alone,
// every round inside the block (the rounds of Sec. 3.1 written edge by edge:
// every live edge folds its key into its vertices' slots with a 64-bit
// atomicMax, edges holding the slot at all their vertices win, edges with a
// matched vertex die), on the instance's part of the union's input arrays.
// It writes the union's result mask and per-edge rounds, so the results are
// read the same way for every class. The union handle is still built (its
// validation and weights serve), but its round loop is not launched.
#include "hm_internal.cuh"
#include "exact_sum.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

namespace hm {
namespace {

constexpr int kBT = 256;

struct Member {            // one instance inside its class's union
    int64_t eidx;          // index of its eoff[0] in the caller's eoff array
    int64_t pbase;         // first pin in the caller's pins array
    int64_t wbase;         // first weight in the caller's weights array
    int64_t ub, upb, vb;   // first union edge, union pin, union vertex
    int64_t nv;            // its vertex count: local pins must be in [0, nv)
};

// One instance of a small class: its first union edge (its edges' offsets
// are eoff_u[ub .. ub + m], absolute union pin positions), its first union
// vertex, and its sizes.
struct SmallInst {
    int64_t ub, vb;
    int32_t n, m;
};

constexpr int64_t kSmallClassPins = 1 << 16;          // a class is small when every instance is below this
constexpr size_t kSmallScratchBytes = size_t(2) << 20;  // and one worker's working memory fits this
constexpr int kSmallThreads = 1024;

struct BatchClass {
    std::vector<int32_t> inst;  // member instances, ascending
    std::vector<Member> mem;
    Handle *h = nullptr;
    // small classes: the union's input arrays (kept), the instance table,
    // the workers' working memory
    bool small = false;
    int64_t *eoff_u = nullptr;
    int32_t *pins_u = nullptr;
    SmallInst *si = nullptr;
    unsigned char *scratch = nullptr;
    size_t scratch_per = 0;
    unsigned grid = 0;
};

struct Batch {
    int32_t count = 0;
    int device = 0;
    bool weighted = true;
    std::vector<int64_t> n, m, kappa;
    std::vector<int32_t> cls_of;
    std::vector<BatchClass> cls;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    cudaStream_t last_stream = nullptr;
    bool matched = false;
};

// kappa of every instance: its last offset
// first and last offset of every instance: out[2i] = eoff[first], out[2i+1] = eoff[last]
__global__ void k_last_offsets(const int64_t *__restrict__ eoff, const int64_t *__restrict__ last_idx,
                               const int64_t *__restrict__ m, int32_t count, int64_t *__restrict__ out) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        out[2 * i] = eoff[last_idx[i] - m[i]];
        out[2 * i + 1] = eoff[last_idx[i]];
    }
}

__device__ __forceinline__ int member_of(const int64_t *base, int nmem, int64_t x) {
    int lo = 0, hi = nmem - 1;  // last member with base <= x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// union edge offsets and weights (thread per union edge, plus the final offset)
__global__ void k_union_edges(const int64_t *__restrict__ eoff, const float *__restrict__ w,
                              const Member *__restrict__ mem, const int64_t *__restrict__ ubase, int nmem,
                              int64_t m_u, uint64_t kappa_u, int64_t *__restrict__ eoff_u,
                              float *__restrict__ w_u) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e <= m_u;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e == m_u) {
            eoff_u[m_u] = (int64_t)kappa_u;
            continue;
        }
        const Member mb = mem[member_of(ubase, nmem, e)];
        const int64_t le = e - mb.ub;
        eoff_u[e] = mb.upb + eoff[mb.eidx + le];
        if (w) w_u[e] = w[mb.wbase + le];
    }
}

// union pins (thread per union pin). A pin outside its own instance's
// [0, n) becomes -1, which the union's validation rejects: offset into the
// union it would otherwise land on another instance's vertex.
__global__ void k_union_pins(const int32_t *__restrict__ pins, const Member *__restrict__ mem,
                             const int64_t *__restrict__ pbase_u, int nmem, uint64_t kappa_u,
                             int32_t *__restrict__ pins_u) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < kappa_u;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const Member mb = mem[member_of(pbase_u, nmem, (int64_t)p)];
        const int64_t lp = pins[mb.pbase + ((int64_t)p - mb.upb)];
        pins_u[p] = (lp < 0 || lp >= mb.nv) ? -1 : (int32_t)(lp + mb.vb);
    }
}

// Small classes: resets the instance counter and the class's status.
__global__ void k_small_init(DevState *st) {
    st->nwin = 0;
    st->status = HM_OK;
    st->fault = 0;
    st->finished = 1;
}

__host__ __device__ __forceinline__ size_t small_align(size_t x) { return (x + 255) & ~size_t(255); }

// The key of an instance's edge e (instance-local id): weight bits, then the
// smaller id first; unweighted, the seeded fmix32 priority of the local id
// (the order hm_create gives the instance alone).
__device__ __forceinline__ unsigned long long small_key(const float *w, uint32_t salt, int32_t e) {
    if (w) return ((unsigned long long)__float_as_uint(w[e]) << 32) | (0xFFFFFFFFull - (uint32_t)e);
    return (0x3F800000ull << 32) | fmix32((uint32_t)e ^ salt);
}

// Small classes: one-block workers, each matching whole instances taken from
// a counter (st->nwin), every round inside the block. Working memory of a
// worker: best (uint64[n]), matched (uint8[n]), alive (uint8[m]).
__global__ void __launch_bounds__(kSmallThreads, 1)
k_small_batch(const SmallInst *__restrict__ si, int32_t count, const int64_t *__restrict__ eoff_u,
              const int32_t *__restrict__ pins_u, const float *__restrict__ w_u, uint32_t salt,
              uint8_t *__restrict__ inM, int32_t *__restrict__ wround, unsigned char *__restrict__ scratch,
              size_t per, DevState *st) {
    __shared__ int32_t s_i;
    unsigned char *my = scratch + (size_t)blockIdx.x * per;
    const int t = threadIdx.x;
    for (;;) {
        if (t == 0) s_i = (int32_t)atomicAdd(&st->nwin, 1u);
        __syncthreads();
        const int32_t i = s_i;
        __syncthreads();  // every thread has read s_i before it is rewritten
        if (i >= count) break;  // uniform
        const SmallInst q = si[i];
        const int64_t *eo = eoff_u + q.ub;
        const float *w = w_u ? w_u + q.ub : nullptr;
        unsigned long long *best = reinterpret_cast<unsigned long long *>(my);
        uint8_t *matched = my + small_align((size_t)q.n * 8);
        uint8_t *alive = matched + small_align((size_t)q.n);
        for (int32_t e = t; e < q.m; e += kSmallThreads) {
            alive[e] = 1;
            inM[q.ub + e] = 0;
        }
        for (int32_t v = t; v < q.n; v += kSmallThreads) matched[v] = 0;
        __syncthreads();
        int32_t rounds = 0;
        for (;;) {
            for (int32_t v = t; v < q.n; v += kSmallThreads) best[v] = 0ull;
            __syncthreads();
            int any = 0;
            for (int32_t e = t; e < q.m; e += kSmallThreads) {
                if (!alive[e]) continue;
                any = 1;
                const unsigned long long k = small_key(w, salt, e);
                for (int64_t p = eo[e]; p < eo[e + 1]; ++p) atomicMax(&best[pins_u[p] - q.vb], k);
            }
            if (!__syncthreads_or(any)) break;
            if (rounds >= q.m) {  // every round has a winner: never reached for valid input
                if (t == 0) st->status = HM_ECUDA;
                break;
            }
            ++rounds;
            for (int32_t e = t; e < q.m; e += kSmallThreads) {
                if (!alive[e]) continue;
                const unsigned long long k = small_key(w, salt, e);
                bool all = true;
                for (int64_t p = eo[e]; p < eo[e + 1] && all; ++p) all = best[pins_u[p] - q.vb] == k;
                if (all) {  // winners are vertex-disjoint: these writes never collide
                    inM[q.ub + e] = 1;
                    wround[q.ub + e] = rounds;
                    alive[e] = 0;
                    for (int64_t p = eo[e]; p < eo[e + 1]; ++p) matched[pins_u[p] - q.vb] = 1;
                }
            }
            __syncthreads();
            for (int32_t e = t; e < q.m; e += kSmallThreads) {
                if (!alive[e]) continue;
                for (int64_t p = eo[e]; p < eo[e + 1]; ++p)
                    if (matched[pins_u[p] - q.vb]) {
                        alive[e] = 0;
                        break;
                    }
            }
            __syncthreads();
        }
        __syncthreads();  // the block's working memory is reused by the next instance
    }
}

__global__ void k_gather_rounds(const int32_t *__restrict__ idx, const int32_t *__restrict__ wround,
                                const uint32_t *__restrict__ count, int32_t *__restrict__ out) {
    const uint32_t c = *count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x)
        out[i] = wround[idx[i]];
}

hm_status bad(const char *msg) {
    set_error(msg);
    return HM_EINVAL;
}

void free_batch(Batch *b) {
    for (auto &c : b->cls) {
        if (c.h) {
            if (c.h->done) cudaEventSynchronize(c.h->done);
            if (c.h->cap_stream) cudaStreamSynchronize(c.h->cap_stream);
        }
        for (void *p : {(void *)c.eoff_u, (void *)c.pins_u, (void *)c.si, (void *)c.scratch})
            if (p) cudaFree(p);
        if (c.h) {
            free_handle_buffers(c.h);
            delete c.h;
        }
    }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->done) cudaEventDestroy(b->done);
    delete b;
}

template <typename T>
hm_status upload(T **dst, const std::vector<T> &src, cudaStream_t s) {
    cudaError_t e = cudaMallocAsync((void **)dst, std::max<size_t>(1, src.size()) * sizeof(T), s);
    if (e == cudaSuccess && !src.empty())
        e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch upload");
    return HM_OK;
}

// Builds the handle of one class from the caller's concatenated arrays.
hm_status build_class(Batch *b, BatchClass &c, const int64_t *eoff, const int32_t *pins, const float *w,
                      uint64_t seed, int sm_count, cudaStream_t s) {
    const int nmem = (int)c.inst.size();
    int64_t n_u = 0, m_u = 0, k_u = 0;
    std::vector<int64_t> ubase(nmem), pbase(nmem);
    for (int k = 0; k < nmem; ++k) {
        Member &mb = c.mem[k];
        const int32_t i = c.inst[k];
        mb.ub = m_u;
        mb.upb = k_u;
        mb.vb = n_u;
        ubase[k] = m_u;
        pbase[k] = k_u;
        n_u += b->n[i];
        m_u += b->m[i];
        k_u += b->kappa[i];
    }
    if (n_u > INT32_MAX || m_u > INT32_MAX || (uint64_t)k_u > 0xFFFFFFFFull)
        return bad("a size class of the batch exceeds 2^31-1 vertices or edges or 2^32-1 pins");
    {
        int64_t maxk = 0, maxn = 0, maxm = 0;
        for (int k = 0; k < nmem; ++k) {
            const int32_t i = c.inst[k];
            maxk = std::max(maxk, b->kappa[i]);
            maxn = std::max(maxn, b->n[i]);
            maxm = std::max(maxm, b->m[i]);
        }
        c.scratch_per = small_align((size_t)maxn * 8) + small_align((size_t)maxn) + small_align((size_t)maxm);
        c.small = maxk < kSmallClassPins && c.scratch_per <= kSmallScratchBytes;
    }
    Member *d_mem = nullptr;
    int64_t *d_ub = nullptr, *d_pb = nullptr, *eoff_u = nullptr;
    int32_t *pins_u = nullptr;
    float *w_u = nullptr;
    hm_status st = upload(&d_mem, c.mem, s);
    if (st == HM_OK) st = upload(&d_ub, ubase, s);
    if (st == HM_OK) st = upload(&d_pb, pbase, s);
    cudaError_t e = cudaSuccess;
    if (st == HM_OK) e = cudaMallocAsync((void **)&eoff_u, (size_t)(m_u + 1) * 8, s);
    if (st == HM_OK && e == cudaSuccess) e = cudaMallocAsync((void **)&pins_u, (size_t)std::max<int64_t>(1, k_u) * 4, s);
    if (st == HM_OK && e == cudaSuccess && b->weighted)
        e = cudaMallocAsync((void **)&w_u, (size_t)std::max<int64_t>(1, m_u) * 4, s);
    if (st == HM_OK && e != cudaSuccess) st = cuda_fail(e, "batch union buffers");
    if (st == HM_OK) {
        k_union_edges<<<grid_for((uint64_t)m_u + 1, kBT, sm_count, 8), kBT, 0, s>>>(
            eoff, b->weighted ? w : nullptr, d_mem, d_ub, nmem, m_u, (uint64_t)k_u, eoff_u, w_u);
        k_union_pins<<<grid_for((uint64_t)k_u, kBT, sm_count, 8), kBT, 0, s>>>(pins, d_mem, d_pb, nmem,
                                                                              (uint64_t)k_u, pins_u);
        if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(e, "batch union build");
    }
    if (st == HM_OK) {
        Handle *h = new (std::nothrow) Handle();
        if (h) h->edge_rounds = true;  // an instance's round count is the round of its last winner
        if (!h) {
            st = HM_ENOMEM;
        } else {
            c.h = h;
            h->n = n_u;
            h->m = m_u;
            h->kappa = (uint64_t)k_u;
            h->weighted = b->weighted;
            h->seed = seed;
            h->cap = m_u + 1;
            h->device = b->device;
            h->sm_count = sm_count;
            if ((e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
                st = cuda_fail(e, "cudaStreamCreate");
            if (st == HM_OK)
                st = create_structures(h, eoff_u, pins_u, w_u, s, b->weighted ? nullptr : d_ub, nmem);
            if (st == HM_OK) st = alloc_round_state(h, s);
            if (st == HM_OK && (e = cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming)) != cudaSuccess)
                st = cuda_fail(e, "cudaEventCreate");
        }
    }
    if (st == HM_OK && c.small) {
        // the workers read the union's input arrays: keep them (they live as
        // long as the batch), with the instance table and working memory
        std::vector<SmallInst> si(nmem);
        for (int k = 0; k < nmem; ++k) {
            const int32_t i = c.inst[k];
            si[k] = SmallInst{c.mem[k].ub, c.mem[k].vb, (int32_t)b->n[i], (int32_t)b->m[i]};
        }
        int per_sm = 0;  // resident workers per SM
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small_batch, kSmallThreads, 0) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        c.grid = (unsigned)std::min<int64_t>(nmem, (int64_t)sm_count * per_sm);
        if ((e = cudaMalloc((void **)&c.si, si.size() * sizeof(SmallInst))) != cudaSuccess ||
            (e = cudaMemcpyAsync(c.si, si.data(), si.size() * sizeof(SmallInst), cudaMemcpyHostToDevice, s)) !=
                cudaSuccess ||
            (e = cudaMalloc((void **)&c.scratch, std::max<size_t>(1, c.scratch_per * c.grid))) != cudaSuccess ||
            (e = cudaMalloc((void **)&c.eoff_u, (size_t)(m_u + 1) * 8)) != cudaSuccess ||
            (e = cudaMalloc((void **)&c.pins_u, (size_t)std::max<int64_t>(1, k_u) * 4)) != cudaSuccess ||
            (e = cudaMemcpyAsync(c.eoff_u, eoff_u, (size_t)(m_u + 1) * 8, cudaMemcpyDeviceToDevice, s)) !=
                cudaSuccess ||
            (k_u > 0 && (e = cudaMemcpyAsync(c.pins_u, pins_u, (size_t)k_u * 4, cudaMemcpyDeviceToDevice, s)) !=
                            cudaSuccess))
            st = cuda_fail(e, "batch small class");
    }
    if (d_mem) cudaFreeAsync(d_mem, s);
    if (d_ub) cudaFreeAsync(d_ub, s);
    if (d_pb) cudaFreeAsync(d_pb, s);
    if (eoff_u) cudaFreeAsync(eoff_u, s);
    if (pins_u) cudaFreeAsync(pins_u, s);
    if (w_u) cudaFreeAsync(w_u, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess && st == HM_OK) st = cuda_fail(e, "batch class");
    return st;
}

// A small class's branch of the batch graph: counter reset, then the workers.
void capture_small(Handle *h, cudaStream_t s, void *ctx) {
    const BatchClass &c = *static_cast<const BatchClass *>(ctx);
    k_small_init<<<1, 1, 0, s>>>(h->st);
    k_small_batch<<<c.grid, kSmallThreads, 0, s>>>(c.si, (int32_t)c.inst.size(), c.eoff_u, c.pins_u,
                                                    h->weighted ? h->weights : nullptr,
                                                    (uint32_t)splitmix64_first(h->seed), h->inM, h->wround,
                                                    c.scratch, c.scratch_per, h->st);
}

hm_status build_batch_graph(Batch *b) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
    hm_status st = HM_OK;
    for (auto &c : b->cls) {
        if (st != HM_OK) break;
        if (c.small) {
            cudaGraphNode_t tail = nullptr;
            st = capture_chain(c.h, g, capture_small, &c, &tail);
        } else {
            st = add_match_to_graph(c.h, g);
        }
    }
    if (st == HM_OK) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        if ((e = cudaGraphInstantiate(&b->exec, g, 0)) != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate");
    }
    cudaGraphDestroy(g);
    return st;
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" {

hm_status hm_batch_create(hm_batch **out, int32_t count, const int64_t *n, const int64_t *m,
                          const int64_t *eoff, const int32_t *pins, const float *weights, uint64_t seed,
                          uint32_t flags, void *cuda_stream) {
    if (!out) return bad("out is NULL");
    *out = nullptr;
    if (count < 1) return bad("count must be >= 1");
    if (!n || !m) return bad("n and m (host arrays) must not be NULL");
    if (flags & ~(HM_UNWEIGHTED | HM_BORROW_INPUT | HM_VALIDATE | HM_AUTOTUNE | HM_ONE_CLASS))
        return bad("unknown flag bits");
    if (!eoff) return bad("eoff is NULL");
    const bool weighted = !(flags & HM_UNWEIGHTED);
    int64_t sum_m = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (n[i] < 0 || m[i] < 0 || n[i] > INT32_MAX || m[i] > INT32_MAX)
            return bad("every n[i], m[i] must be in [0, 2^31-1]");
        if (m[i] > 0 && n[i] == 0) return bad("an instance has edges but no vertices");
        sum_m += m[i];
    }
    if (weighted && sum_m > 0 && !weights) return bad("weights is NULL without HM_UNWEIGHTED");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Batch *b = new (std::nothrow) Batch();
    if (!b) return HM_ENOMEM;
    b->count = count;
    b->weighted = weighted;
    b->n.assign(n, n + count);
    b->m.assign(m, m + count);
    b->kappa.assign(count, 0);
    cudaError_t e = cudaGetDevice(&b->device);
    int sm_count = 0;
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, b->device);
    // kappa of every instance (one read of all last offsets)
    std::vector<int64_t> eidx(count), last(count);
    int64_t ei = 0;
    for (int32_t i = 0; i < count; ++i) {
        eidx[i] = ei;
        last[i] = ei + m[i];
        ei += m[i] + 1;
    }
    int64_t *d_last = nullptr, *d_m = nullptr, *d_kappa = nullptr;
    std::vector<int64_t> ends(2 * (size_t)count);
    hm_status st = upload(&d_last, last, s);
    if (st == HM_OK) st = upload(&d_m, b->m, s);
    if (st == HM_OK && (e = cudaMallocAsync((void **)&d_kappa, (size_t)count * 16, s)) != cudaSuccess)
        st = cuda_fail(e, "batch kappa");
    if (st == HM_OK) {
        k_last_offsets<<<grid_for((uint64_t)count, kBT, sm_count, 8), kBT, 0, s>>>(eoff, d_last, d_m, count, d_kappa);
        if ((e = cudaMemcpyAsync(ends.data(), d_kappa, (size_t)count * 16, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            st = cuda_fail(e, "batch kappa");
    }
    for (int32_t i = 0; i < count && st == HM_OK; ++i) {
        if (ends[2 * (size_t)i] != 0) {
            char buf[96];
            snprintf(buf, sizeof buf, "instance %d: eoff[0] must be 0", (int)i);
            st = bad(buf);
        }
        b->kappa[i] = ends[2 * (size_t)i + 1];
    }
    if (d_last) cudaFreeAsync(d_last, s);
    if (d_m) cudaFreeAsync(d_m, s);
    if (d_kappa) cudaFreeAsync(d_kappa, s);
    if (st != HM_OK) {
        free_batch(b);
        return st;
    }
    // size classes: floor(log4(kappa)), instance bases in the caller's arrays
    int64_t pb = 0, wb = 0;
    std::vector<Member> mem(count);
    int maxc = 0;
    b->cls_of.assign(count, 0);
    for (int32_t i = 0; i < count; ++i) {
        if (b->kappa[i] < m[i] || (uint64_t)b->kappa[i] > 0xFFFFFFFFull) {
            free_batch(b);
            return bad("an instance's eoff[m] is below m or above 2^32-1");
        }
        mem[i].eidx = eidx[i];
        mem[i].pbase = pb;
        mem[i].wbase = wb;
        mem[i].nv = n[i];
        pb += b->kappa[i];
        wb += m[i];
        int cl = 0;
        if (!(flags & HM_ONE_CLASS))
            for (int64_t k = b->kappa[i]; k >= 4; k >>= 2) ++cl;
        b->cls_of[i] = cl;
        maxc = std::max(maxc, cl);
    }
    if (pb > 0 && !pins) {
        free_batch(b);
        return bad("pins is NULL");
    }
    std::vector<int> remap(maxc + 1, -1);
    for (int32_t i = 0; i < count; ++i) {
        int &r = remap[b->cls_of[i]];
        if (r < 0) {
            r = (int)b->cls.size();
            b->cls.emplace_back();
        }
    }
    for (int32_t i = 0; i < count; ++i) {
        const int c = remap[b->cls_of[i]];
        b->cls_of[i] = c;
        b->cls[c].inst.push_back(i);
        b->cls[c].mem.push_back(mem[i]);
    }
    for (auto &c : b->cls) {
        st = build_class(b, c, eoff, pins, weights, seed, sm_count, s);
        if (st != HM_OK) {
            free_batch(b);
            return st;
        }
        if ((flags & HM_AUTOTUNE) && !c.small) {  // a small class's workers have no launch shape to tune
            LaunchConfig best;
            double ms = 0;
            if ((st = autotune(c.h, s, &best, &ms)) != HM_OK) {
                free_batch(b);
                return st;
            }
        }
    }
    if ((st = build_batch_graph(b)) != HM_OK ||
        ((e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess &&
         (st = cuda_fail(e, "cudaEventCreate")) != HM_OK)) {
        free_batch(b);
        return st;
    }
    *out = reinterpret_cast<hm_batch *>(b);
    return HM_OK;
}

hm_status hm_batch_match(hm_batch *bb, void *cuda_stream) {
    Batch *b = reinterpret_cast<Batch *>(bb);
    if (!b) return bad("batch is NULL");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (b->matched && s != b->last_stream && cudaEventQuery(b->done) == cudaErrorNotReady) {
        set_error("a match of this batch is still running on another stream");
        return HM_EBUSY;
    }
    cudaGetLastError();
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->done, s);
    if (e != cudaSuccess) return cuda_fail(e, "hm_batch_match");
    for (auto &c : b->cls) {  // the class handles' results are read after this event
        cudaEventRecord(c.h->done, s);
        c.h->matched_once = true;
        c.h->last_stream = s;
    }
    b->last_stream = s;
    b->matched = true;
    return HM_OK;
}

hm_status hm_batch_result(hm_batch *bb, int32_t *edges_out, int64_t *counts_out, int32_t *rounds_out,
                          double *weights_out) {
    Batch *b = reinterpret_cast<Batch *>(bb);
    if (!b) return bad("batch is NULL");
    if (!b->matched) return bad("no match has been run on this batch");
    cudaError_t e = cudaEventSynchronize(b->done);
    if (e != cudaSuccess) return cuda_fail(e, "waiting for the batch");
    std::vector<int64_t> cnt(b->count, 0);
    std::vector<int32_t> rnd(b->count, 0);
    std::vector<ExactSum> wsum(b->weighted ? b->count : 0);
    std::vector<std::vector<int32_t>> per(b->count);
    hm_status worst = HM_OK;
    for (auto &c : b->cls) {
        Handle *h = c.h;
        cudaStream_t s = h->cap_stream;
        if ((e = cudaMemcpy(h->h_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "batch loop state");
        if (h->h_st->status != HM_OK && worst == HM_OK) {
            worst = h->h_st->status == HM_ETIMEOUT ? HM_ETIMEOUT
                  : h->h_st->status == HM_EINVAL   ? HM_EINVAL
                                                   : HM_ECUDA;
            set_error("a size class of the batch did not finish cleanly");
        }
        const uint64_t m = (uint64_t)h->m;
        uint32_t count = 0;
        int32_t *d_rnd = nullptr;
        e = compact_flags(h->inM, m, h->weighted ? h->weights : nullptr, h->res_idx, h->res_w, h->res_part, s);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_rnd, std::max<uint64_t>(1, m) * 4, s);
        if (e == cudaSuccess) {
            const uint32_t *dcount = h->res_part + compact_scratch_elems(m);
            k_gather_rounds<<<grid_for(m, kBT, h->sm_count, 8), kBT, 0, s>>>(h->res_idx, h->wround, dcount, d_rnd);
            e = cudaMemcpyAsync(&count, dcount, sizeof count, cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        std::vector<int32_t> idx(count), rr(count);
        std::vector<float> ww(h->weighted ? count : 0);
        if (e == cudaSuccess && count) {
            e = cudaMemcpy(idx.data(), h->res_idx, (size_t)count * 4, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(rr.data(), d_rnd, (size_t)count * 4, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && h->weighted)
                e = cudaMemcpy(ww.data(), h->res_w, (size_t)count * 4, cudaMemcpyDeviceToHost);
        }
        if (d_rnd) cudaFreeAsync(d_rnd, s);
        if (e != cudaSuccess) return cuda_fail(e, "batch result");
        // global ids ascend and members ascend by first edge: walk both
        size_t k = 0;
        for (uint32_t t = 0; t < count; ++t) {
            const int64_t g = idx[t];
            while (k + 1 < c.mem.size() && c.mem[k + 1].ub <= g) ++k;
            const int32_t i = c.inst[k];
            per[i].push_back((int32_t)(g - c.mem[k].ub));
            cnt[i] += 1;
            rnd[i] = std::max(rnd[i], rr[t]);
            if (h->weighted) wsum[i].add(ww[t]);
        }
    }
    int64_t off = 0;
    for (int32_t i = 0; i < b->count; ++i) {
        if (edges_out && cnt[i]) memcpy(edges_out + off, per[i].data(), (size_t)cnt[i] * 4);
        off += cnt[i];
        if (counts_out) counts_out[i] = cnt[i];
        if (rounds_out) rounds_out[i] = rnd[i];
        if (weights_out) weights_out[i] = b->weighted ? wsum[i].value() : (double)cnt[i];
    }
    return worst;
}

hm_status hm_batch_info(hm_batch *bb, int32_t *nclasses_out, int32_t *class_of, int32_t *configs) {
    Batch *b = reinterpret_cast<Batch *>(bb);
    if (!b) return bad("batch is NULL");
    if (nclasses_out) *nclasses_out = (int32_t)b->cls.size();
    if (class_of)
        for (int32_t i = 0; i < b->count; ++i) class_of[i] = b->cls_of[i];
    if (configs)
        for (size_t c = 0; c < b->cls.size(); ++c) {
            const LaunchConfig &x = b->cls[c].h->cfg;
            configs[4 * c + 0] = x.kill_chunk;
            configs[4 * c + 1] = x.argmax_bpsm;
            configs[4 * c + 2] = x.win_bpsm;
            configs[4 * c + 3] = x.kill_bpsm;
        }
    return HM_OK;
}

void hm_batch_destroy(hm_batch *bb) {
    Batch *b = reinterpret_cast<Batch *>(bb);
    if (!b) return;
    if (b->done) cudaEventSynchronize(b->done);
    free_batch(b);
}

}  // extern "C"
