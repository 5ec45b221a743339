// prims.cu - device-wide primitives used while building a handle and when
// reading results: exclusive scan, stable LSD radix sort of 32-bit key/value
// pairs, and stable flag compaction. None of this runs inside the round loop.
#include "hm_internal.cuh"

namespace hm {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // 4096 elements per block
constexpr int kWarps = kThreads / 32;
static_assert(kThreads == 256, "histogram and scatter kernels use one thread per digit");

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

// Exclusive scan of one value per thread over the block; *total gets the sum.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T x, T *total) {
    __shared__ T warp_sum[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_inclusive_scan(x);
    if (lane == 31) warp_sum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kWarps ? warp_sum[lane] : T(0);
        T wi = warp_inclusive_scan(w);
        if (lane < kWarps) warp_sum[lane] = wi - w;
        if (lane == kWarps - 1) *total = wi;
    }
    __syncthreads();
    T r = warp_sum[warp] + inc - x;
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ scan

template <typename T>
__global__ void __launch_bounds__(kThreads) scan_reduce_k(const T *in, uint64_t n, T *part) {
    const uint64_t base = (uint64_t)blockIdx.x * kTile + (uint64_t)threadIdx.x * kItems;
    T s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k)
        if (base + k < n) s += in[base + k];
    __shared__ T tot;
    block_exclusive_scan<T>(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Single block: exclusive scan of part[0..nb) in place; grand total -> *total.
template <typename T>
__global__ void __launch_bounds__(kThreads) scan_part_k(T *part, uint64_t nb, T *total) {
    __shared__ T tot;
    T carry = 0;
    for (uint64_t b0 = 0; b0 < nb; b0 += (uint64_t)kThreads * kItems) {
        const uint64_t base = b0 + (uint64_t)threadIdx.x * kItems;
        T v[kItems];
        T s = 0;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            v[k] = base + k < nb ? part[base + k] : T(0);
            s += v[k];
        }
        T ex = block_exclusive_scan<T>(s, &tot);
        T run = carry + ex;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            if (base + k < nb) part[base + k] = run;
            run += v[k];
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) scan_down_k(const T *in, T *out, uint64_t n, const T *part) {
    const uint64_t base = (uint64_t)blockIdx.x * kTile + (uint64_t)threadIdx.x * kItems;
    T v[kItems];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        v[k] = base + k < n ? in[base + k] : T(0);
        s += v[k];
    }
    __shared__ T tot;
    T run = block_exclusive_scan<T>(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

template <typename T>
cudaError_t exclusive_scan_t(const T *in, T *out, uint64_t n, T *total, T *scratch, cudaStream_t s) {
    if (n == 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(T), s);
        return cudaSuccess;
    }
    const uint64_t nb = (n + kTile - 1) / kTile;
    scan_reduce_k<T><<<(unsigned)nb, kThreads, 0, s>>>(in, n, scratch);
    scan_part_k<T><<<1, kThreads, 0, s>>>(scratch, nb, total);
    scan_down_k<T><<<(unsigned)nb, kThreads, 0, s>>>(in, out, n, scratch);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ radix sort

__global__ void __launch_bounds__(kThreads) rs_hist_k(const uint32_t *keys, uint64_t n, int shift,
                                                      uint32_t *hist, uint32_t ntiles) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;  // kThreads == 256
    __syncthreads();
    const uint64_t tbase = (uint64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int k = 0; k < kItems; ++k) {
        uint64_t i = tbase + (uint64_t)k * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one tile. Warp w owns the contiguous sub-tile
// [w*512, (w+1)*512) and walks it 32 elements at a time; lanes with equal
// digits are ranked with __match_any_sync, so equal keys keep input order
// inside the warp, and warps are ordered by a per-digit prefix over warps.
// The tile is first rearranged in shared memory into digit order, then
// written out by consecutive threads, so each run of equal digits becomes
// one coalesced segment of the output.
__global__ void __launch_bounds__(kThreads) rs_scatter_k(const uint32_t *kin, const uint32_t *vin,
                                                         uint32_t *kout, uint32_t *vout, uint64_t n,
                                                         int shift, const uint32_t *offs,
                                                         uint32_t ntiles) {
    constexpr int kSub = 32 * kItems;
    __shared__ uint32_t wcnt[kWarps][256];
    __shared__ uint32_t dstart[256];  // first tile-local slot of each digit
    __shared__ uint32_t goff[256];    // global position of each digit's run from this tile
    __shared__ uint32_t skey[kTile], sval[kTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < kWarps * 256; d += kThreads) (&wcnt[0][0])[d] = 0;
    goff[threadIdx.x] = offs[(uint64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();
    const uint64_t tbase = (uint64_t)blockIdx.x * kTile;
    const uint32_t tcount = (uint32_t)(n - tbase < (uint64_t)kTile ? n - tbase : (uint64_t)kTile);
    const unsigned lt = (1u << lane) - 1u;
    uint32_t key[kItems], val[kItems], rank[kItems];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const uint32_t li = (uint32_t)warp * kSub + it * 32 + lane;
        const bool ok = li < tcount;
        key[it] = ok ? kin[tbase + li] : 0u;
        val[it] = ok ? vin[tbase + li] : 0u;
        const uint32_t d = ok ? ((key[it] >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t base = d < 256u ? wcnt[warp][d] : 0u;
        rank[it] = base + __popc(peers & lt);
        __syncwarp();
        if (d < 256u && (peers & lt) == 0u) wcnt[warp][d] = base + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        // per digit: prefix over warps; per tile: prefix over digits
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t t = wcnt[w][d];
            wcnt[w][d] = run;
            run += t;
        }
        __shared__ uint32_t tot;
        dstart[d] = block_exclusive_scan<uint32_t>(run, &tot);
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const uint32_t li = (uint32_t)warp * kSub + it * 32 + lane;
        if (li < tcount) {
            const uint32_t d = (key[it] >> shift) & 255u;
            const uint32_t slot = dstart[d] + wcnt[warp][d] + rank[it];
            skey[slot] = key[it];
            sval[slot] = val[it];
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tcount; i += kThreads) {
        const uint32_t k = skey[i];
        const uint32_t d = (k >> shift) & 255u;
        const uint64_t pos = (uint64_t)goff[d] + (i - dstart[d]);
        kout[pos] = k;
        vout[pos] = sval[i];
    }
}

// ------------------------------------------------------------------ compaction

__global__ void __launch_bounds__(kThreads) cmp_count_k(const uint8_t *f, uint64_t n, uint32_t *part) {
    const uint64_t base = (uint64_t)blockIdx.x * kTile + (uint64_t)threadIdx.x * kItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k)
        if (base + k < n) s += f[base + k] != 0;
    __shared__ uint32_t tot;
    block_exclusive_scan<uint32_t>(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) cmp_write_k(const uint8_t *f, uint64_t n, const uint32_t *part,
                                                        const float *w, int32_t *idx, float *wout) {
    const uint64_t base = (uint64_t)blockIdx.x * kTile + (uint64_t)threadIdx.x * kItems;
    uint32_t s = 0;
    uint8_t fl[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        fl[k] = base + k < n ? f[base + k] : 0;
        s += fl[k] != 0;
    }
    __shared__ uint32_t tot;
    uint32_t run = block_exclusive_scan<uint32_t>(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (fl[k]) {
            idx[run] = (int32_t)(base + k);
            if (w) wout[run] = w[base + k];
            ++run;
        }
    }
}

}  // namespace

size_t scan_scratch_elems(uint64_t n) { return (size_t)((n + kTile - 1) / kTile) + 1; }

cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *total,
                               uint32_t *scratch, cudaStream_t s) {
    return exclusive_scan_t<uint32_t>(in, out, n, total, scratch, s);
}

cudaError_t exclusive_scan_i64(const int64_t *in, int64_t *out, uint64_t n, int64_t *total,
                               int64_t *scratch, cudaStream_t s) {
    return exclusive_scan_t<int64_t>(in, out, n, total, scratch, s);
}

size_t radix_scratch_elems(uint64_t n) {
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    const uint64_t hist = 256 * (ntiles ? ntiles : 1);
    return (size_t)(hist + scan_scratch_elems(hist));
}

cudaError_t radix_sort_pairs(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *keys_out,
                             uint32_t *vals_out, uint32_t *tmp_k, uint32_t *tmp_v, uint64_t n,
                             int end_bit, uint32_t *scratch, cudaStream_t s) {
    const int passes = (end_bit + 7) / 8;
    if (n == 0) return cudaSuccess;
    if (passes == 0) {
        cudaError_t e = cudaMemcpyAsync(keys_out, keys_in, n * 4, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(vals_out, vals_in, n * 4, cudaMemcpyDeviceToDevice, s);
    }
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    uint32_t *hist = scratch;
    uint32_t *scan_tmp = scratch + 256 * ntiles;
    const uint32_t *ck = keys_in, *cv = vals_in;
    for (int p = 0; p < passes; ++p) {
        // The last pass must land in *_out: alternate backwards from it.
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t *nk = to_out ? keys_out : tmp_k;
        uint32_t *nv = to_out ? vals_out : tmp_v;
        const int shift = 8 * p;
        rs_hist_k<<<(unsigned)ntiles, kThreads, 0, s>>>(ck, n, shift, hist, (uint32_t)ntiles);
        cudaError_t e = exclusive_scan_u32(hist, hist, 256 * ntiles, nullptr, scan_tmp, s);
        if (e != cudaSuccess) return e;
        rs_scatter_k<<<(unsigned)ntiles, kThreads, 0, s>>>(ck, cv, nk, nv, n, shift, hist,
                                                           (uint32_t)ntiles);
        ck = nk;
        cv = nv;
    }
    return cudaGetLastError();
}

size_t compact_scratch_elems(uint64_t n) { return scan_scratch_elems(n); }

cudaError_t compact_flags(const uint8_t *flags, uint64_t n, const float *w, int32_t *idx_out,
                          float *w_out, uint32_t *part, cudaStream_t s) {
    const uint64_t nb = (n + kTile - 1) / kTile;
    uint32_t *count = part + compact_scratch_elems(n);
    if (n == 0) return cudaMemsetAsync(count, 0, sizeof(uint32_t), s);
    cmp_count_k<<<(unsigned)nb, kThreads, 0, s>>>(flags, n, part);
    scan_part_k<uint32_t><<<1, kThreads, 0, s>>>(part, nb, count);
    cmp_write_k<<<(unsigned)nb, kThreads, 0, s>>>(flags, n, part, w, idx_out, w_out);
    return cudaGetLastError();
}

}  // namespace hm
