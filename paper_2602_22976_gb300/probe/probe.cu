// probe.cu - libhmprobe.so, a measurement tool of the benchmark (not part of
// the matching library): the rate of random single-element accesses of this
// GPU into an array of a given size.
//
// The round kernels are bound by such accesses (1-byte live flags, 4-byte
// counters and cursors gathered or scattered at random), not by streaming
// bandwidth, so a copy-bandwidth roofline alone says little about them.
// bench.py reports these rates next to the HBM roofline.
//
// int hmprobe_random_access(uint64_t array_bytes, uint64_t ops,
//                           double *gops_out, void *cuda_stream)
//   Runs `ops` accesses of each kind (below) at pseudo-random indices of a
//   device scratch array of `array_bytes` bytes (1 KiB .. 4 GiB, allocated
//   and freed here, stream-ordered) and writes the best of two timed runs
//   after a warm-up run, in 1e9 accesses per second, to HOST
//   double[kProbeCount]. Waits for completion. Returns 0, or 1 (bad
//   argument), 2 (out of device memory), 3 (a CUDA call failed); the
//   message is in hmprobe_last_error().
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

namespace {

enum { kStore1 = 0, kLoad1 = 1, kLoad4 = 2, kRed4 = 3, kAtomic4 = 4, kProbeCount = 5 };

thread_local char g_msg[200] = "";

// index of the i-th access: a 64-bit mix of i, reduced to the array
__device__ __forceinline__ uint32_t probe_index(uint64_t x, uint32_t size) {
    x ^= x >> 33;
    x *= 0xFF51AFD7ED558CCDULL;
    x ^= x >> 33;
    x *= 0xC4CEB9FE1A85EC53ULL;
    x ^= x >> 33;
    return (uint32_t)(x % size);
}

template <int MODE>
__global__ void __launch_bounds__(256) k_probe(uint8_t *a8, uint32_t *a32, uint32_t size, uint64_t ops,
                                               unsigned long long *sink) {
    unsigned long long acc = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < ops;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t idx = probe_index(i, size);
        if (MODE == kStore1) a8[idx] = 0;
        else if (MODE == kLoad1) acc += __ldcg(a8 + idx);
        else if (MODE == kLoad4) acc += __ldcg(a32 + idx);
        else if (MODE == kRed4) atomicSub(a32 + idx, 1u);
        else acc += atomicSub(a32 + idx, 1u);
    }
    if (acc == 0x5EEDULL) *sink = acc;  // keeps the loads alive
}

int fail(int code, const char *what, cudaError_t e = cudaSuccess) {
    if (e != cudaSuccess) snprintf(g_msg, sizeof g_msg, "%s: %s", what, cudaGetErrorString(e));
    else snprintf(g_msg, sizeof g_msg, "%s", what);
    return code;
}

}  // namespace

extern "C" const char *hmprobe_last_error(void) { return g_msg; }

extern "C" int hmprobe_random_access(uint64_t array_bytes, uint64_t ops, double *gops_out, void *cuda_stream) {
    g_msg[0] = 0;
    if (!gops_out) return fail(1, "gops_out is NULL");
    if (array_bytes < 1024 || array_bytes > (uint64_t)1 << 32 || ops == 0)
        return fail(1, "array_bytes must be in [1 KiB, 4 GiB] and ops > 0");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint8_t *buf = nullptr;
    unsigned long long *sink = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&buf, array_bytes, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&sink, sizeof *sink, s);
    if (e != cudaSuccess) {
        if (buf) cudaFreeAsync(buf, s);
        cudaGetLastError();
        return fail(2, "out of device memory");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const unsigned grid = (unsigned)(sms * 8);
    const uint32_t n8 = (uint32_t)(array_bytes > 0xFFFFFFFFull ? 0xFFFFFFFFull : array_bytes);
    const uint32_t n32 = (uint32_t)(array_bytes / 4);
    for (int mode = 0; mode < kProbeCount && e == cudaSuccess; ++mode) {
        float best = 0.f;
        for (int rep = 0; rep < 3; ++rep) {  // the first run warms the array into L2 where it fits
            e = cudaMemsetAsync(buf, 1, array_bytes, s);
            if (e != cudaSuccess) break;
            cudaEventRecord(e0, s);
            const uint32_t sz = (mode == kStore1 || mode == kLoad1) ? n8 : n32;
            uint32_t *b32 = reinterpret_cast<uint32_t *>(buf);
            switch (mode) {
            case kStore1: k_probe<kStore1><<<grid, 256, 0, s>>>(buf, b32, sz, ops, sink); break;
            case kLoad1: k_probe<kLoad1><<<grid, 256, 0, s>>>(buf, b32, sz, ops, sink); break;
            case kLoad4: k_probe<kLoad4><<<grid, 256, 0, s>>>(buf, b32, sz, ops, sink); break;
            case kRed4: k_probe<kRed4><<<grid, 256, 0, s>>>(buf, b32, sz, ops, sink); break;
            default: k_probe<kAtomic4><<<grid, 256, 0, s>>>(buf, b32, sz, ops, sink); break;
            }
            cudaEventRecord(e1, s);
            e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const float g = (float)ops / ms / 1e6f;
            if (rep > 0 && g > best) best = g;
        }
        gops_out[mode] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(buf, s);
    cudaFreeAsync(sink, s);
    if (e != cudaSuccess) return fail(3, "probe", e);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(3, "probe", e);
    return 0;
}
