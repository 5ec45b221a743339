// prims.cu - device-wide primitives used while building a handle and when
// reading results: exclusive scan, stable LSD radix sort of 32-bit key/value
// pairs, and stable flag compaction. None of this runs inside the round loop.
#include "hm_internal.cuh"

namespace hm {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // 2048 elements per block (scan, compaction)
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
// LSD radix sort of 32-bit keys with 32-bit values, 8-bit digits. A pass:
//  1. rs_hist_k: every tile of kRTile keys counts its digits into one
//     256-entry row of a tile-major histogram (a coalesced 1 KB write);
//  2. rs_scan_{a,b,c}_k: the histogram becomes the output offset of every
//     (tile, digit) run - digits in order, and inside a digit the tiles in
//     order, which is what makes the pass stable - with every access a
//     coalesced row of 256 words (a: per-digit sums over blocks of
//     kScanTiles tiles; b: one block scans those sums and the digit totals;
//     c: running offsets inside each block of tiles);
//  3. rs_scatter_k: every tile ranks its keys (stable inside the tile),
//     regroups them by digit in shared memory and writes each digit's run
//     to its offset with consecutive threads.
constexpr int kRI = 16;                 // keys per thread
constexpr int kRTile = kThreads * kRI;  // 4096 keys per tile
constexpr int kScanTiles = 256;         // tiles per block of the offset scan

__global__ void __launch_bounds__(kThreads) rs_hist_k(const uint32_t *__restrict__ keys, uint64_t n, int shift,
                                                      uint32_t *__restrict__ hist) {
    __shared__ uint32_t cnt[kWarps][256];  // one sub-histogram per warp: fewer same-address atomics
    for (int d = threadIdx.x; d < kWarps * 256; d += kThreads) (&cnt[0][0])[d] = 0;
    __syncthreads();
    uint32_t *mine = cnt[threadIdx.x >> 5];
    const uint64_t tbase = (uint64_t)blockIdx.x * kRTile;
    if (tbase + kRTile <= n) {  // full tile: 16-byte loads
        const uint4 *k4 = reinterpret_cast<const uint4 *>(keys + tbase);
#pragma unroll
        for (int k = 0; k < kRI / 4; ++k) {
            const uint4 x = __ldg(k4 + k * kThreads + threadIdx.x);
            atomicAdd(&mine[(x.x >> shift) & 255u], 1u);
            atomicAdd(&mine[(x.y >> shift) & 255u], 1u);
            atomicAdd(&mine[(x.z >> shift) & 255u], 1u);
            atomicAdd(&mine[(x.w >> shift) & 255u], 1u);
        }
    } else {
        for (int k = 0; k < kRI; ++k) {
            const uint64_t i = tbase + (uint64_t)k * kThreads + threadIdx.x;
            if (i < n) atomicAdd(&mine[(__ldg(keys + i) >> shift) & 255u], 1u);
        }
    }
    __syncthreads();
    uint32_t sum = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) sum += cnt[w][threadIdx.x];
    hist[(uint64_t)blockIdx.x * 256 + threadIdx.x] = sum;
}

// part[b][d] = sum of hist[t][d] over the tiles t of block b.
__global__ void __launch_bounds__(kThreads) rs_scan_a_k(const uint32_t *__restrict__ hist, uint64_t ntiles,
                                                        uint32_t *__restrict__ part) {
    const uint64_t t0 = (uint64_t)blockIdx.x * kScanTiles;
    const uint64_t t1 = t0 + kScanTiles < ntiles ? t0 + kScanTiles : ntiles;
    uint32_t s = 0;
#pragma unroll 8
    for (uint64_t t = t0; t < t1; ++t) s += hist[t * 256 + threadIdx.x];
    part[(uint64_t)blockIdx.x * 256 + threadIdx.x] = s;
}

// One block: part[b][d] <- (keys of digits < d) + (keys of digit d in blocks < b).
__global__ void __launch_bounds__(kThreads) rs_scan_b_k(uint32_t *part, uint64_t nb) {
    const int d = threadIdx.x;
    uint32_t run = 0;
    for (uint64_t b0 = 0; b0 < nb; b0 += 8) {
        uint32_t x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = b0 + k < nb ? part[(b0 + k) * 256 + d] : 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (b0 + k < nb) part[(b0 + k) * 256 + d] = run;
            run += x[k];
        }
    }
    __shared__ uint32_t tot;
    const uint32_t base = block_exclusive_scan<uint32_t>(run, &tot);
    for (uint64_t b = 0; b < nb; ++b) part[b * 256 + d] += base;
}

// hist[t][d] <- output offset of the run of digit d from tile t.
__global__ void __launch_bounds__(kThreads) rs_scan_c_k(uint32_t *hist, uint64_t ntiles, const uint32_t *part) {
    const uint64_t t0 = (uint64_t)blockIdx.x * kScanTiles;
    const uint64_t t1 = t0 + kScanTiles < ntiles ? t0 + kScanTiles : ntiles;
    const int d = threadIdx.x;
    uint32_t run = part[(uint64_t)blockIdx.x * 256 + d];
    for (uint64_t t = t0; t < t1; t += 8) {
        uint32_t x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = t + k < t1 ? hist[(t + k) * 256 + d] : 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (t + k < t1) hist[(t + k) * 256 + d] = run;
            run += x[k];
        }
    }
}

// Stable scatter of one tile. Warp w owns the contiguous sub-tile
// [w*512, (w+1)*512) and walks it 32 keys at a time; lanes with equal
// digits are ranked with __match_any_sync, so equal keys keep input order
// inside the warp, and warps are ordered by a per-digit prefix over warps.
// The tile is first rearranged in shared memory into digit order, then
// written out by consecutive threads, so each run of equal digits becomes
// one coalesced segment of the output.
__global__ void __launch_bounds__(kThreads, 3) rs_scatter_k(const uint32_t *__restrict__ kin,
                                                         const uint32_t *__restrict__ vin,
                                                         uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                         uint64_t n, int shift, const uint32_t *__restrict__ offs) {
    constexpr int kSub = 32 * kRI;
    __shared__ uint32_t wcnt[kWarps][256];
    __shared__ uint32_t dstart[256];  // first tile-local slot of each digit
    __shared__ uint32_t goff[256];    // global position of each digit's run from this tile
    __shared__ uint32_t skey[kRTile], sval[kRTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < kWarps * 256; d += kThreads) (&wcnt[0][0])[d] = 0;
    goff[threadIdx.x] = offs[(uint64_t)blockIdx.x * 256 + threadIdx.x];
    __syncthreads();
    const uint64_t tbase = (uint64_t)blockIdx.x * kRTile;
    const uint32_t tcount = (uint32_t)(n - tbase < (uint64_t)kRTile ? n - tbase : (uint64_t)kRTile);
    const unsigned lt = (1u << lane) - 1u;
    uint32_t key[kRI], val[kRI], rank[kRI];
#pragma unroll
    for (int it = 0; it < kRI; ++it) {
        const uint32_t li = (uint32_t)warp * kSub + it * 32 + lane;
        const bool ok = li < tcount;
        key[it] = ok ? __ldg(kin + tbase + li) : 0u;
        val[it] = ok ? __ldg(vin + tbase + li) : 0u;
    }
#pragma unroll
    for (int it = 0; it < kRI; ++it) {
        const uint32_t li = (uint32_t)warp * kSub + it * 32 + lane;
        const uint32_t d = li < tcount ? ((key[it] >> shift) & 255u) : 256u;
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
    for (int it = 0; it < kRI; ++it) {
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

// Per exponent field E, the sum of the integer significands of the weights
// of the flagged entries (see exact_sum.cuh): block totals in shared memory,
// one global atomic per block and bucket.
__global__ void __launch_bounds__(kThreads) wsum_k(const uint8_t *__restrict__ f, const float *__restrict__ w,
                                                   uint64_t n, unsigned long long *__restrict__ bucket) {
    __shared__ unsigned long long sb[256];
    sb[threadIdx.x] = 0;  // kThreads == 256
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)kThreads + threadIdx.x; i < n; i += (uint64_t)gridDim.x * kThreads) {
        if (f[i]) {
            const uint32_t u = __float_as_uint(w[i]);
            const uint32_t E = (u >> 23) & 255u, fr = u & 0x7FFFFFu;
            atomicAdd(&sb[E], (unsigned long long)(E ? (fr | 0x800000u) : fr));
        }
    }
    __syncthreads();
    if (sb[threadIdx.x]) atomicAdd(&bucket[threadIdx.x], sb[threadIdx.x]);
}

}  // namespace

cudaError_t weight_buckets(const uint8_t *flags, const float *w, uint64_t n, unsigned long long *bucket,
                           int sm_count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bucket, 0, 256 * sizeof(unsigned long long), s);
    if (e != cudaSuccess || n == 0) return e;
    wsum_k<<<grid_for(n, kThreads, sm_count, 8), kThreads, 0, s>>>(flags, w, n, bucket);
    return cudaGetLastError();
}

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
    const uint64_t ntiles = (n + kRTile - 1) / kRTile;
    const uint64_t nb = (ntiles + kScanTiles - 1) / kScanTiles;
    return (size_t)(256 * ((ntiles ? ntiles : 1) + (nb ? nb : 1)));
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
    const uint64_t ntiles = (n + kRTile - 1) / kRTile;
    const uint64_t nb = (ntiles + kScanTiles - 1) / kScanTiles;
    uint32_t *hist = scratch;                  // [ntiles][256]
    uint32_t *part = scratch + 256 * ntiles;   // [nb][256]
    const uint32_t *ck = keys_in, *cv = vals_in;
    for (int p = 0; p < passes; ++p) {
        // The last pass must land in *_out: alternate backwards from it.
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t *nk = to_out ? keys_out : tmp_k;
        uint32_t *nv = to_out ? vals_out : tmp_v;
        const int shift = 8 * p;
        rs_hist_k<<<(unsigned)ntiles, kThreads, 0, s>>>(ck, n, shift, hist);
        rs_scan_a_k<<<(unsigned)nb, kThreads, 0, s>>>(hist, ntiles, part);
        rs_scan_b_k<<<1, kThreads, 0, s>>>(part, nb);
        rs_scan_c_k<<<(unsigned)nb, kThreads, 0, s>>>(hist, ntiles, part);
        rs_scatter_k<<<(unsigned)ntiles, kThreads, 0, s>>>(ck, cv, nk, nv, n, shift, hist);
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
