// noalloc.cu - hm_match_noalloc: the whole matching of a small hypergraph in
// one kernel launch, without allocating any memory.
//
// Who needs this: code that is not allowed to allocate device memory at the
// moment it wants a matching. Examples are a caller in the middle of
// capturing a CUDA graph on its stream (cudaMalloc is not a capturable call
// and invalidates the capture), a host framework that owns every byte of
// device memory through its own arena and forbids other allocators, and
// latency-bound loops that cannot pay for cudaMalloc's implicit
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
#include "hm_internal.cuh"

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

__device__ __forceinline__ uint32_t na_fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

__host__ __device__ inline uint64_t na_splitmix64_first(uint64_t x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

// Packed key: larger wins. Weighted: weight bits, then smaller id first.
// Unweighted: bits of 1.0f, then the seeded fmix32 priority.
__device__ __forceinline__ unsigned long long na_key(const float *w, uint32_t salt, int64_t e) {
    if (w) return ((unsigned long long)__float_as_uint(w[e]) << 32) | (0xFFFFFFFFull - (uint32_t)e);
    return (0x3F800000ull << 32) | na_fmix32((uint32_t)e ^ salt);
}

constexpr int kNaThreads = 1024;

// result[0] = rounds that started with a live edge, result[1] = hm_status
// (HM_OK, or HM_EINVAL for an invalid edge range, pin or weight).
__global__ void __launch_bounds__(kNaThreads, 1)
k_match_noalloc(const int64_t *__restrict__ eoff, const int32_t *__restrict__ pins,
                const float *__restrict__ w, uint32_t salt, int64_t n, int64_t m,
                uint8_t *__restrict__ in_matching, int32_t *__restrict__ result,
                unsigned char *__restrict__ scratch) {
    unsigned long long *best = reinterpret_cast<unsigned long long *>(scratch);
    uint8_t *matched = scratch + align256((size_t)n * 8);
    uint8_t *alive = matched + align256((size_t)n);
    const int t = threadIdx.x;

    // validation of the edge ranges and weights (Sec. 2.1), then of the pins;
    // pins are only read once the ranges are known to be sound
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
    if (t == 0) result[0] = rounds, result[1] = HM_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
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
        set_error("hm_match_noalloc: inputs and outputs must be device memory");
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
    const uint32_t salt = (uint32_t)na_splitmix64_first(seed);
    k_match_noalloc<<<1, kNaThreads, 0, (cudaStream_t)cuda_stream>>>(
        eoff, pins, weighted ? weights : nullptr, salt, n, m, in_matching, result,
        static_cast<unsigned char *>(scratch));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "hm_match_noalloc: launch");
    return HM_OK;
}
