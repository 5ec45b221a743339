// probe.cu - hm_probe_random_access: measures this GPU's rate of random
// single-element accesses into an array of a given size.
//
// The round kernels are bound by such accesses (1-byte live flags, 4-byte
// counters and cursors gathered or scattered at random), not by streaming
// bandwidth, so a copy-bandwidth roofline alone says little about them.
// The benchmark reports these rates next to the HBM roofline.
#include "hm_internal.cuh"

namespace hm {
namespace {

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
        if (MODE == HM_PROBE_STORE1) a8[idx] = 0;
        else if (MODE == HM_PROBE_LOAD1) acc += __ldcg(a8 + idx);
        else if (MODE == HM_PROBE_LOAD4) acc += __ldcg(a32 + idx);
        else if (MODE == HM_PROBE_RED4) atomicSub(a32 + idx, 1u);
        else acc += atomicSub(a32 + idx, 1u);
    }
    if (acc == 0x5EEDULL) *sink = acc;  // keeps the loads alive
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" hm_status hm_probe_random_access(uint64_t array_bytes, uint64_t ops, double *gops_out,
                                            void *cuda_stream) {
    if (!gops_out) {
        set_error("gops_out is NULL");
        return HM_EINVAL;
    }
    if (array_bytes < 1024 || array_bytes > (uint64_t)1 << 32 || ops == 0) {
        set_error("hm_probe_random_access: array_bytes must be in [1 KiB, 4 GiB] and ops > 0");
        return HM_EINVAL;
    }
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
        set_error("hm_probe_random_access: out of device memory");
        return HM_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const unsigned grid = (unsigned)(sms * 8);
    const uint32_t n8 = (uint32_t)(array_bytes > 0xFFFFFFFFull ? 0xFFFFFFFFull : array_bytes);
    const uint32_t n32 = (uint32_t)(array_bytes / 4);
    for (int mode = 0; mode < HM_PROBE_COUNT && e == cudaSuccess; ++mode) {
        float best = 0.f;
        for (int rep = 0; rep < 3; ++rep) {  // first run warms the array into L2 where it fits
            e = cudaMemsetAsync(buf, 1, array_bytes, s);
            if (e != cudaSuccess) break;
            cudaEventRecord(e0, s);
            const uint32_t sz = (mode == HM_PROBE_STORE1 || mode == HM_PROBE_LOAD1) ? n8 : n32;
            uint32_t *b32 = reinterpret_cast<uint32_t *>(buf);
            switch (mode) {
            case HM_PROBE_STORE1: k_probe<HM_PROBE_STORE1><<<grid, 256, 0, s>>>(buf, b32, sz, ops, sink); break;
            case HM_PROBE_LOAD1: k_probe<HM_PROBE_LOAD1><<<grid, 256, 0, s>>>(buf, b32, sz, ops, sink); break;
            case HM_PROBE_LOAD4: k_probe<HM_PROBE_LOAD4><<<grid, 256, 0, s>>>(buf, b32, sz, ops, sink); break;
            case HM_PROBE_RED4: k_probe<HM_PROBE_RED4><<<grid, 256, 0, s>>>(buf, b32, sz, ops, sink); break;
            default: k_probe<HM_PROBE_ATOMIC4><<<grid, 256, 0, s>>>(buf, b32, sz, ops, sink); break;
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
    if (e != cudaSuccess) return cuda_fail(e, "hm_probe_random_access");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "hm_probe_random_access");
    return HM_OK;
}
