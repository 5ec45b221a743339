// noalloc.cu - hm_match_noalloc: the whole matching of a small hypergraph in
// one kernel launch, without allocating any memory.
//
// Who needs this: code that is not allowed to allocate device memory at the
// moment it wants a matching. Examples are a host framework that owns every
// byte of device memory through its own arena and forbids other allocators,
// and latency-bound loops that cannot pay for cudaMalloc's implicit
// synchronisation and page mapping. Such callers pass their inputs and
// outputs; everything else this entry point needs lives in a fixed,
// file-scope device array that the library declares once.
//
// The kernel is one thread block that runs the rounds directly on the edge
// CSR: each round clears best[v], every live edge folds its key into the
// best[] of its vertices with a 64-bit atomicMax on the packed key
// (weight bits << 32 | tie-break), edges whose key is the best at all their
// vertices join the matching and mark their vertices, and live edges that
// touch a marked vertex are deactivated. The order on edges is the same
// strict order as hm_match's, so the result is the same matching and round
// count.
//
// hm_solve_host runs the same kernel for small inputs (solve_small below),
// on working memory from the stream's pool, after k_check_small has checked
// the input the way hm_create does.
#include "hm_internal.cuh"
#include "exact_sum.cuh"

#include <algorithm>
#include <climits>
#include <cstdio>
#include <mutex>

namespace hm {
namespace {

// Size of the static scratch array. Every GPU that loads libhm.so keeps
// these bytes reserved until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB

// The scratch array. Host code must not use this symbol as a device address:
// in host code it names a host-side stand-in. Its device address is obtained
// with cudaGetSymbolAddress, once per device, below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// best: uint64[n], matched: uint8[n], alive: uint8[m]
inline size_t scratch_bytes(int64_t n, int64_t m) {
    return align256((size_t)n * 8) + align256((size_t)n) + align256((size_t)m);
}

// Packed key: larger wins. Weighted: weight bits, then smaller id first.
// Unweighted: bits of 1.0f, then the seeded fmix32 priority (the helpers
// hm_create's order uses, so both paths order edges identically).
__device__ __forceinline__ unsigned long long na_key(const float *w, uint32_t salt, int64_t e) {
    if (w) return ((unsigned long long)__float_as_uint(w[e]) << 32) | (0xFFFFFFFFull - (uint32_t)e);
    return (0x3F800000ull << 32) | fmix32((uint32_t)e ^ salt);
}

constexpr int kNaThreads = 1024;

// Error kinds of the checking form, in the order hm_create reports them.
enum : int32_t { kNaRange = 1, kNaPin = 2, kNaWeight = 4, kNaRepeat = 8 };

// Input checks of hm_solve_host's small inputs (every edge at most
// kSmallMaxSize pins), on a grid of kCkThreads-thread blocks: edge ranges,
// pins, weights, and no vertex twice in one edge. first[k] receives the
// first offending index (edge, or pin position) of error kind bit k; the
// caller sets all four to ~0 beforehand. A repeat in a short edge is found
// by one thread comparing all pairs; a longer edge is taken by a warp, which
// inserts its pins into the warp's own open-addressing table of kNaSlots
// slots in shared memory (never more than half full). An edge's pins are
// only read once its own range lies inside [0, kappa).
constexpr int kCkThreads = 256;
constexpr int kNaSlots = 512;
constexpr uint32_t kNaEmpty = 0xFFFFFFFFu;
static_assert(2 * kSmallMaxSize <= kNaSlots, "a warp's table must stay at most half full");

__global__ void __launch_bounds__(kCkThreads)
k_check_small(const int64_t *__restrict__ eoff, const int32_t *__restrict__ pins, const float *__restrict__ w,
              int64_t n, int64_t m, int64_t kappa, unsigned long long *__restrict__ first) {
    __shared__ uint32_t s_tab[kCkThreads / 32][kNaSlots];
    const int64_t tid = blockIdx.x * (int64_t)kCkThreads + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * kCkThreads;
    if (tid == 0 && eoff[0] != 0) atomicMin(&first[0], 0ull);
    for (int64_t e = tid; e < m; e += nth) {
        if (eoff[e + 1] <= eoff[e]) atomicMin(&first[0], (unsigned long long)e);
        if (w) {
            const uint32_t b = __float_as_uint(w[e]);
            if (b == 0u || b >= 0x7F800000u) atomicMin(&first[2], (unsigned long long)e);
        }
    }
    for (int64_t i = tid; i < kappa; i += nth) {
        const int32_t p = pins[i];
        if (p < 0 || (int64_t)p >= n) atomicMin(&first[1], (unsigned long long)i);
    }
    for (int64_t e = tid; e < m; e += nth) {
        const int64_t b = eoff[e], en = eoff[e + 1];
        if (b < 0 || en > kappa || en <= b || en - b > 16) continue;
        for (int64_t i = b; i < en; ++i) {
            const int32_t p = pins[i];
            for (int64_t j = i + 1; j < en; ++j)
                if (pins[j] == p) atomicMin(&first[3], (unsigned long long)e);
        }
    }
    const int lane = threadIdx.x & 31;
    uint32_t *tab = s_tab[threadIdx.x >> 5];
    for (int k = lane; k < kNaSlots; k += 32) tab[k] = kNaEmpty;
    __syncwarp();
    for (int64_t e = tid >> 5; e < m; e += nth >> 5) {  // uniform in the warp
        const int64_t b = eoff[e], en = eoff[e + 1];
        if (b < 0 || en > kappa || en - b <= 16 || en - b > kSmallMaxSize) continue;
        bool dup = false;
        for (int64_t i = b + lane; i < en; i += 32) {
            const uint32_t v = (uint32_t)pins[i];
            uint32_t h = (v * 2654435761u) >> 23;  // 9 bits (Knuth's multiplicative hash)
            for (int probe = 0; probe < kNaSlots; ++probe) {
                const uint32_t prev = atomicCAS(&tab[h], kNaEmpty, v);
                if (prev == kNaEmpty) break;  // v is in the table now
                if (prev == v) {              // v was there already: a repeat
                    dup = true;
                    break;
                }
                h = (h + 1) & (kNaSlots - 1);
            }
        }
        __syncwarp();
        if (__any_sync(0xffffffffu, dup) && lane == 0) atomicMin(&first[3], (unsigned long long)e);
        for (int k = lane; k < kNaSlots; k += 32) tab[k] = kNaEmpty;  // clear for the next edge
        __syncwarp();
    }
}

// result[0] = rounds that started with a live edge, result[1] = hm_status
// (HM_OK, or HM_EINVAL for an invalid edge range, pin or weight).
// first (hm_solve_host's small inputs): k_check_small has checked the input;
// if it found an error, result[2] and result[3] receive the kinds found
// (kNa* bits) and the first offending index of the most important one, and
// nothing runs. Otherwise (null: hm_match_noalloc) the kernel checks ranges,
// pins and weights itself.
__global__ void __launch_bounds__(kNaThreads, 1)
k_match_noalloc(const int64_t *__restrict__ eoff, const int32_t *__restrict__ pins,
                const float *__restrict__ w, uint32_t salt, int64_t n, int64_t m,
                uint8_t *__restrict__ in_matching, int32_t *__restrict__ result,
                unsigned char *__restrict__ scratch, const unsigned long long *__restrict__ first) {
    unsigned long long *best = reinterpret_cast<unsigned long long *>(scratch);
    uint8_t *matched = scratch + align256((size_t)n * 8);
    uint8_t *alive = matched + align256((size_t)n);
    const int t = threadIdx.x;

    if (first) {
        int32_t bits = 0, at = -1;
        for (int k = 3; k >= 0; --k)
            if (first[k] != ~0ull) {
                bits |= 1 << k;
                at = (int32_t)first[k];
            }
        if (bits) {
            if (t == 0) result[0] = 0, result[1] = HM_EINVAL, result[2] = bits, result[3] = at;
            return;
        }
    } else {
        // validation of the edge ranges and weights (Sec. 2.1), then of the
        // pins; pins are only read once the ranges are known to be sound
        int bad = (t == 0 && eoff[0] != 0);
        for (int64_t e = t; e < m; e += kNaThreads) {
            if (eoff[e + 1] <= eoff[e]) bad = 1;
            if (w) {
                const uint32_t b = __float_as_uint(w[e]);
                if (b == 0u || b >= 0x7F800000u) bad = 1;
            }
        }
        if (__syncthreads_or(bad)) {
            if (t == 0) result[0] = 0, result[1] = HM_EINVAL;
            return;
        }
        const int64_t kappa = eoff[m];
        for (int64_t i = t; i < kappa; i += kNaThreads) {
            const int32_t p = pins[i];
            if (p < 0 || (int64_t)p >= n) bad = 1;
        }
        if (__syncthreads_or(bad)) {
            if (t == 0) result[0] = 0, result[1] = HM_EINVAL;
            return;
        }
    }

    // every call starts from a clean state: the array keeps the last call's bytes
    for (int64_t e = t; e < m; e += kNaThreads) {
        alive[e] = 1;
        in_matching[e] = 0;
    }
    for (int64_t v = t; v < n; v += kNaThreads) matched[v] = 0;
    __syncthreads();

    int32_t rounds = 0;
    for (;;) {
        for (int64_t v = t; v < n; v += kNaThreads) best[v] = 0ull;
        __syncthreads();
        int any = 0;
        for (int64_t e = t; e < m; e += kNaThreads) {
            if (!alive[e]) continue;
            any = 1;
            const unsigned long long k = na_key(w, salt, e);
            for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i) atomicMax(&best[pins[i]], k);
        }
        if (!__syncthreads_or(any) || rounds > m) break;  // rounds <= m for valid input
        ++rounds;
        for (int64_t e = t; e < m; e += kNaThreads) {
            if (!alive[e]) continue;
            const unsigned long long k = na_key(w, salt, e);
            bool all = true;
            for (int64_t i = eoff[e]; i < eoff[e + 1] && all; ++i) all = best[pins[i]] == k;
            if (all) {  // winners are vertex-disjoint: these writes never collide
                in_matching[e] = 1;
                alive[e] = 0;
                for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i) matched[pins[i]] = 1;
            }
        }
        __syncthreads();
        for (int64_t e = t; e < m; e += kNaThreads) {
            if (!alive[e]) continue;
            for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i)
                if (matched[pins[i]]) {
                    alive[e] = 0;
                    break;
                }
        }
        __syncthreads();
    }
    if (t == 0) {
        result[0] = rounds;
        result[1] = HM_OK;
        if (first) result[2] = 0, result[3] = -1;
    }
}

// Memory of the current device (or managed memory): the kernel is launched
// on the current device, and memory of another GPU would fault there.
bool on_device(const void *p) { return usable_device_pointer(p); }

}  // namespace

// hm_solve_host's path for small inputs: one block runs the whole matching
// (launch and synchronisation costs dominate hm_create + hm_match there).
// Its working memory comes from the stream's pool, so concurrent calls
// (the server's workers) never share it. The result is compacted and its
// weight summed on the device as hm_result does; one synchronisation.
hm_status solve_small(int64_t n, int64_t m, uint64_t kappa, const int64_t *eoff, const int32_t *pins,
                      const float *weights, uint64_t seed, bool weighted, int32_t *edges_out,
                      int64_t *count_out, int32_t *rounds_out, double *weight_out, cudaStream_t s) {
    int dev = 0, sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += align256(bytes ? bytes : 1);
        return at;
    };
    const size_t a_eoff = take((size_t)(m + 1) * 8), a_pins = take((size_t)kappa * 4),
                 a_w = take(weighted ? (size_t)m * 4 : 0), a_scr = take(scratch_bytes(n, m)), a_inm = take((size_t)m),
                 a_res = take(4 * sizeof(int32_t)), a_idx = take((size_t)m * 4),
                 a_part = take((compact_scratch_elems((uint64_t)m) + 1) * 4),
                 a_bkt = take(kExpBuckets * sizeof(unsigned long long)),
                 a_first = take(4 * sizeof(unsigned long long));
    unsigned char *buf = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&buf, off, s);
    if (e != cudaSuccess) return cuda_fail(e, "hm_solve_host: allocation");
    struct Free {
        unsigned char *p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } guard{buf, s};
    int64_t *d_eoff = reinterpret_cast<int64_t *>(buf + a_eoff);
    int32_t *d_pins = reinterpret_cast<int32_t *>(buf + a_pins);
    float *d_w = weighted ? reinterpret_cast<float *>(buf + a_w) : nullptr;
    uint8_t *d_inm = buf + a_inm;
    int32_t *d_res = reinterpret_cast<int32_t *>(buf + a_res);
    int32_t *d_idx = reinterpret_cast<int32_t *>(buf + a_idx);
    uint32_t *d_part = reinterpret_cast<uint32_t *>(buf + a_part);
    unsigned long long *d_bkt = reinterpret_cast<unsigned long long *>(buf + a_bkt);
    e = cudaMemcpyAsync(d_eoff, eoff, (size_t)(m + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && kappa)
        e = cudaMemcpyAsync(d_pins, pins, (size_t)kappa * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && weighted && m)
        e = cudaMemcpyAsync(d_w, weights, (size_t)m * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "hm_solve_host: upload");
    const uint32_t salt = (uint32_t)splitmix64_first(seed);
    unsigned long long *d_first = reinterpret_cast<unsigned long long *>(buf + a_first);
    e = cudaMemsetAsync(d_first, 0xFF, 4 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "hm_solve_host: check state");
    const uint64_t work = std::max<uint64_t>((uint64_t)m, kappa);
    const unsigned grid = (unsigned)std::min<uint64_t>((work + 4 * kCkThreads - 1) / (4 * kCkThreads),
                                                       (uint64_t)(2 * std::max(sm, 1)));
    k_check_small<<<grid ? grid : 1, kCkThreads, 0, s>>>(d_eoff, d_pins, d_w, n, m, (int64_t)kappa, d_first);
    k_match_noalloc<<<1, kNaThreads, 0, s>>>(d_eoff, d_pins, d_w, salt, n, m, d_inm, d_res, buf + a_scr, d_first);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = compact_flags(d_inm, (uint64_t)m, nullptr, d_idx, nullptr, d_part, s);
    const bool wsum = weight_out && weighted;
    if (e == cudaSuccess && wsum) e = weight_buckets(d_inm, d_w, (uint64_t)m, d_bkt, sm, s);
    int32_t res[4] = {};
    uint32_t count = 0;
    uint64_t bucket[kExpBuckets];
    if (e == cudaSuccess) e = cudaMemcpyAsync(res, d_res, sizeof res, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&count, d_part + compact_scratch_elems((uint64_t)m), sizeof count,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && wsum) e = cudaMemcpyAsync(bucket, d_bkt, sizeof bucket, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "hm_solve_host: small-input match");
    if (res[1] != HM_OK) {
        char msg[200];
        const unsigned long long at = (unsigned long long)(uint32_t)res[3];
        if (res[2] & kNaRange)
            snprintf(msg, sizeof msg, "eoff is not strictly increasing at edge %llu (empty or decreasing edge)", at);
        else if (res[2] & kNaPin)
            snprintf(msg, sizeof msg, "pin at position %llu is outside [0, n)", at);
        else if (res[2] & kNaWeight)
            snprintf(msg, sizeof msg, "weight of edge %llu is not finite and > 0", at);
        else
            snprintf(msg, sizeof msg, "duplicate pin: a vertex appears twice in one edge (edge %llu)", at);
        set_error(msg);
        return HM_EINVAL;
    }
    if (edges_out && count) {
        e = cudaMemcpyAsync(edges_out, d_idx, (size_t)count * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "hm_solve_host: result copy");
    }
    if (count_out) *count_out = count;
    if (rounds_out) *rounds_out = res[0];
    if (weight_out) *weight_out = wsum ? exact_sum_value(bucket) : (double)count;
    return HM_OK;
}

}  // namespace hm

using namespace hm;

extern "C" hm_status hm_match_noalloc(int64_t n, int64_t m, const int64_t *eoff, const int32_t *pins,
                                      const float *weights, uint64_t seed, uint32_t flags,
                                      uint8_t *in_matching, int32_t *result, void *cuda_stream) {
    if (flags & ~(HM_UNWEIGHTED | HM_BORROW_INPUT | HM_VALIDATE)) {
        set_error("unknown flag bits");
        return HM_EINVAL;
    }
    if (n < 0 || m < 0 || n > INT32_MAX || m > INT32_MAX) {
        set_error("n and m must be in [0, 2^31-1]");
        return HM_EINVAL;
    }
    const size_t need = scratch_bytes(n, m);
    if (need > kNoAllocScratchBytes) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "hm_match_noalloc: n=%lld, m=%lld needs %zu bytes of scratch (9*n + m, each part "
                 "rounded up to 256); the fixed scratch array holds %zu bytes",
                 (long long)n, (long long)m, need, kNoAllocScratchBytes);
        set_error(buf);
        return HM_EINVAL;
    }
    const bool weighted = !(flags & HM_UNWEIGHTED);
    if (!eoff || !result || (m > 0 && (!pins || !in_matching)) || (m > 0 && weighted && !weights)) {
        set_error("hm_match_noalloc: NULL input or output pointer");
        return HM_EINVAL;
    }
    if (!on_device(eoff) || !on_device(result) || (m > 0 && (!on_device(pins) || !on_device(in_matching))) ||
        (m > 0 && weighted && !on_device(weights))) {
        set_error("hm_match_noalloc: inputs and outputs must be device memory of the current device");
        return HM_EINVAL;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "hm_match_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("hm_match_noalloc: device index out of range");
        return HM_EINVAL;
    }
    void *scratch = nullptr;
    {
        // One-time set-up per device, with that device current: the device
        // address of the scratch array.
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "hm_match_noalloc: cudaGetSymbolAddress");
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    const uint32_t salt = (uint32_t)splitmix64_first(seed);
    // a launch error is read back below: clear one that an earlier call of
    // the caller left behind, so it is not reported as this launch's
    cudaGetLastError();
    k_match_noalloc<<<1, kNaThreads, 0, (cudaStream_t)cuda_stream>>>(
        eoff, pins, weighted ? weights : nullptr, salt, n, m, in_matching, result,
        static_cast<unsigned char *>(scratch), nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "hm_match_noalloc: launch");
    return HM_OK;
}
