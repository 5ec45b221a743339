// api.cu - the extern "C" entry points declared in include/hm.h.
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

bool usable_device_pointer(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    if (at.type != cudaMemoryTypeDevice) return false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.device == dev;
}

namespace {
thread_local std::string g_err;

bool device_pointer(const void *p) { return usable_device_pointer(p); }

hm_status einval(const char *msg) {
    g_err = msg;
    return HM_EINVAL;
}

hm_status check_device(const Handle *h) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != h->device) return einval("the current CUDA device is not the handle's device");
    return HM_OK;
}

// Waits for the last match and copies the loop state to the host.
hm_status wait_state(Handle *h) {
    if (!h->matched_once) return einval("no match has been run on this handle");
    cudaError_t e = cudaEventSynchronize(h->done);
    if (e != cudaSuccess) return cuda_fail(e, "waiting for the match");
    e = cudaMemcpy(h->h_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the loop state");
    return HM_OK;
}

hm_status loop_status(const Handle *h) {
    switch (h->h_st->status) {
    case HM_OK:
        return HM_OK;
    case HM_ETIMEOUT:
        g_err = "round cap reached before the loop finished";
        return HM_ETIMEOUT;
    case HM_EINVAL:
        g_err = "duplicate pin: a round found no winner while vertices still had live edges";
        return HM_EINVAL;
    default: {
        char buf[120];
        snprintf(buf, sizeof buf, "internal consistency check failed in the round loop (code %d)",
                 h->h_st->fault);
        g_err = buf;
        return HM_ECUDA;
    }
    }
}

void raise_pool_threshold(int dev);

// Builds a handle from checked arguments (device inputs; see create_structures
// for feed).
hm_status create_handle(hm_handle **out, int64_t n, int64_t m, uint64_t kappa, const int64_t *eoff,
                        const int32_t *pins, const float *weights, uint64_t seed, bool weighted, cudaStream_t s,
                        const PinChunks *feed) {
    Handle *h = new (std::nothrow) Handle();
    if (!h) return HM_ENOMEM;
    h->n = n;
    h->m = m;
    h->kappa = kappa;
    h->weighted = weighted;
    h->seed = seed;
    h->cap = m + 1;
    cudaError_t e;
    if ((e = cudaGetDevice(&h->device)) != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaGetDevice");
    }
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    raise_pool_threshold(h->device);
    hm_status st = HM_OK;
    if ((e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        st = cuda_fail(e, "cudaStreamCreate");
    if (st == HM_OK) st = create_structures(h, eoff, pins, weights, s, nullptr, 0, feed);
    if (st == HM_OK) st = alloc_round_state(h, s);
    if (st == HM_OK) {
        if ((e = cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming)) != cudaSuccess)
            st = cuda_fail(e, "cudaEventCreate");
    }
    if (st == HM_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(e, "hm_create");
    if (st != HM_OK) {
        cudaStreamSynchronize(s);
        hm_destroy(reinterpret_cast<hm_handle *>(h));
        return st;
    }
    *out = reinterpret_cast<hm_handle *>(h);
    return HM_OK;
}

void raise_pool_threshold(int dev) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
}
}  // namespace

void set_error(const std::string &msg) { g_err = msg; }

hm_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    cudaGetLastError();
    return HM_ECUDA;
}

}  // namespace hm

using namespace hm;

extern "C" {

const char *hm_last_error(void) { return g_err.c_str(); }

void hm_destroy(hm_handle *hh) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return;
    if (h->done) cudaEventSynchronize(h->done);
    if (h->cap_stream) cudaStreamSynchronize(h->cap_stream);
    free_handle_buffers(h);
    delete h;
}

hm_status hm_create(hm_handle **out, int64_t n, int64_t m, const int64_t *eoff, const int32_t *pins,
                    const float *weights, uint64_t seed, uint32_t flags, void *cuda_stream) {
    if (!out) return einval("out is NULL");
    *out = nullptr;
    if (flags & ~(HM_UNWEIGHTED | HM_BORROW_INPUT | HM_VALIDATE)) return einval("unknown flag bits");
    if (n < 0 || n > INT32_MAX) return einval("n must be in [0, 2^31-1]");
    if (m < 0 || m > INT32_MAX) return einval("m must be in [0, 2^31-1]");
    const bool weighted = !(flags & HM_UNWEIGHTED);
    if (!eoff) return einval("eoff is NULL");
    if (!device_pointer(eoff)) return einval("eoff must be device memory");
    if (m > 0 && weighted) {
        if (!weights) return einval("weights is NULL without HM_UNWEIGHTED");
        if (!device_pointer(weights)) return einval("weights must be device memory");
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int64_t ends[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(&ends[0], eoff, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&ends[1], eoff + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "reading eoff[0], eoff[m]");
    if (ends[0] != 0) return einval("eoff[0] must be 0");
    if (ends[1] < m) return einval("eoff[m] < m: some edge is empty or eoff decreases");
    if ((uint64_t)ends[1] > 0xFFFFFFFFull) return einval("kappa = eoff[m] must be <= 2^32-1");
    if (ends[1] > 0) {
        if (!pins) return einval("pins is NULL");
        if (!device_pointer(pins)) return einval("pins must be device memory");
    }
    if (m > 0 && n == 0) return einval("edges need vertices: n == 0 with m > 0");
    return create_handle(out, n, m, (uint64_t)ends[1], eoff, pins, weights, seed, weighted, s, nullptr);
}

hm_status hm_set_round_cap(hm_handle *hh, int64_t cap) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return einval("handle is NULL");
    if (cap < 1) return einval("round cap must be >= 1");
    h->cap = cap;
    return HM_OK;
}

hm_status hm_set_noise(hm_handle *hh, float amplitude) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return einval("handle is NULL");
    if (!(amplitude >= 0.f) || std::isinf(amplitude)) return einval("noise amplitude must be finite and >= 0");
    h->noise = amplitude;
    return HM_OK;
}

static hm_status busy_check(Handle *h, cudaStream_t s) {
    if (h->matched_once && s != h->last_stream && cudaEventQuery(h->done) == cudaErrorNotReady)
        return HM_EBUSY;
    cudaGetLastError();
    return HM_OK;
}

hm_status hm_match(hm_handle *hh, void *cuda_stream) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return einval("handle is NULL");
    hm_status st = check_device(h);
    if (st != HM_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (busy_check(h, s) != HM_OK) {
        g_err = "a match of this handle is still running on another stream";
        return HM_EBUSY;
    }
    st = h->noise > 0.f ? launch_match_graph_rand(h, s) : launch_match_graph(h, s);
    if (st != HM_OK) return st;
    h->last_random = h->noise > 0.f;
    cudaError_t e = cudaEventRecord(h->done, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    h->last_stream = s;
    h->matched_once = true;
    return HM_OK;
}

hm_status hm_profile_match(hm_handle *hh, void *cuda_stream, double *ms_out, int64_t *launches_out,
                           double *round_ms_out, int32_t max_rounds) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return einval("handle is NULL");
    if (!ms_out || !launches_out) return einval("output pointer is NULL");
    hm_status st = check_device(h);
    if (st != HM_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (busy_check(h, s) != HM_OK) {
        g_err = "a match of this handle is still running on another stream";
        return HM_EBUSY;
    }
    if (!round_ms_out) max_rounds = 0;
    if (max_rounds < 0) return einval("max_rounds < 0");
    st = h->noise > 0.f ? profile_match_rand(h, s, ms_out, launches_out, round_ms_out, max_rounds)
                        : profile_match(h, s, ms_out, launches_out, round_ms_out, max_rounds);
    h->last_random = h->noise > 0.f;
    h->last_stream = s;
    h->matched_once = true;
    return st;
}

hm_status hm_launch_config(hm_handle *hh, const int32_t *set, int32_t *get) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return einval("handle is NULL");
    if (set) {
        LaunchConfig c;
        c.kill_chunk = set[0];
        c.argmax_bpsm = set[1];
        c.win_bpsm = set[2];
        c.kill_bpsm = set[3];
        hm_status st = apply_config(h, c);
        if (st != HM_OK) return st;
    }
    if (get) {
        get[0] = h->cfg.kill_chunk;
        get[1] = h->cfg.argmax_bpsm;
        get[2] = h->cfg.win_bpsm;
        get[3] = h->cfg.kill_bpsm;
    }
    return HM_OK;
}

hm_status hm_autotune(hm_handle *hh, void *cuda_stream, int32_t *config_out, double *ms_out) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return einval("handle is NULL");
    hm_status st = check_device(h);
    if (st != HM_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (busy_check(h, s) != HM_OK) {
        g_err = "a match of this handle is still running on another stream";
        return HM_EBUSY;
    }
    LaunchConfig best;
    double ms = 0;
    st = autotune(h, s, &best, &ms);
    if (st != HM_OK) return st;
    h->last_random = false;
    cudaEventRecord(h->done, s);
    h->last_stream = s;
    h->matched_once = true;
    if (config_out) {
        config_out[0] = best.kill_chunk;
        config_out[1] = best.argmax_bpsm;
        config_out[2] = best.win_bpsm;
        config_out[3] = best.kill_bpsm;
    }
    if (ms_out) *ms_out = ms;
    return HM_OK;
}

hm_status hm_result(hm_handle *hh, int32_t *edges_out, int64_t *count_out, int32_t *rounds_out,
                    double *weight_out) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return einval("handle is NULL");
    hm_status st = wait_state(h);
    if (st != HM_OK) return st;
    cudaStream_t s = h->cap_stream;
    const uint64_t m = (uint64_t)h->m;
    cudaError_t e = compact_flags(h->inM, m, nullptr, h->res_idx, nullptr, h->res_part, s);
    const bool wsum = weight_out && h->weighted;
    if (e == cudaSuccess && wsum) e = weight_buckets(h->inM, h->weights, m, h->res_bucket, h->sm_count, s);
    uint32_t count = 0;
    uint64_t bucket[kExpBuckets];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&count, h->res_part + compact_scratch_elems(m), sizeof count,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && wsum) e = cudaMemcpyAsync(bucket, h->res_bucket, sizeof bucket, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "result compaction");
    if (edges_out && count)
        if ((e = cudaMemcpy(edges_out, h->res_idx, (size_t)count * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "result copy");
    if (weight_out) *weight_out = wsum ? exact_sum_value(bucket) : (double)count;
    if (count_out) *count_out = count;
    if (rounds_out) *rounds_out = h->h_st->rounds_done;
    return loop_status(h);
}

hm_status hm_result_device(hm_handle *hh, uint8_t *in_matching, void *cuda_stream) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return einval("handle is NULL");
    if (!in_matching) return einval("in_matching is NULL");
    if (!h->matched_once) return einval("no match has been run on this handle");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaStreamWaitEvent(s, h->done, 0);
    if (e == cudaSuccess && h->m)
        e = cudaMemcpyAsync(in_matching, h->inM, (size_t)h->m, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "hm_result_device");
    return HM_OK;
}

hm_status hm_round_stats(hm_handle *hh, int64_t *stats, int32_t max_rounds, int32_t *rows_out) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return einval("handle is NULL");
    if (!stats || !rows_out || max_rounds < 0) return einval("bad output arguments");
    hm_status st = wait_state(h);
    if (st != HM_OK) return st;
    int32_t rows = h->h_st->round;
    if (rows > kStatRounds) rows = kStatRounds;
    if (rows > max_rounds) rows = max_rounds;
    if (rows > 0) {
        cudaError_t e = cudaMemcpy(stats, h->stats, (size_t)rows * HM_STATS_COLS * sizeof(int64_t),
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "hm_round_stats");
    }
    *rows_out = rows;
    return HM_OK;
}

hm_status hm_vertex_state(hm_handle *hh, int32_t *best_edge_out) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return einval("handle is NULL");
    if (!best_edge_out) return einval("best_edge_out is NULL");
    hm_status st = wait_state(h);
    if (st != HM_OK) return st;
    if (h->n == 0) return HM_OK;
    cudaStream_t s = h->cap_stream;
    int32_t *d = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&d, (size_t)h->n * 4, s);
    if (e != cudaSuccess) return cuda_fail(e, "hm_vertex_state alloc");
    e = launch_vertex_state(h, d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(best_edge_out, d, (size_t)h->n * 4, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "hm_vertex_state");
    if (e2 != cudaSuccess) return cuda_fail(e2, "hm_vertex_state");
    return HM_OK;
}

hm_status hm_create_ms(hm_handle *hh, double *ms_out) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return einval("handle is NULL");
    if (!ms_out) return einval("ms_out is NULL");
    memcpy(ms_out, h->create_ms, sizeof h->create_ms);
    return HM_OK;
}

hm_status hm_solve_host(int64_t n, int64_t m, const int64_t *eoff, const int32_t *pins,
                        const float *weights, uint64_t seed, uint32_t flags, int32_t *edges_out,
                        int64_t *count_out, int32_t *rounds_out, double *weight_out, void *cuda_stream) {
    if (n < 0 || m < 0 || m > INT32_MAX || n > INT32_MAX) return einval("n, m must be in [0, 2^31-1]");
    if (!eoff) return einval("eoff is NULL");
    const bool weighted = !(flags & HM_UNWEIGHTED);
    if (m > 0 && weighted && !weights) return einval("weights is NULL without HM_UNWEIGHTED");
    const int64_t kappa = eoff[m];
    if (eoff[0] != 0 || kappa < 0 || (uint64_t)kappa > 0xFFFFFFFFull)
        return einval("eoff[0] must be 0 and eoff[m] in [0, 2^32-1]");
    if (kappa > 0 && !pins) return einval("pins is NULL");
    if (flags & ~(HM_UNWEIGHTED | HM_BORROW_INPUT | HM_VALIDATE)) return einval("unknown flag bits");
    if (kappa < m) return einval("eoff[m] < m: some edge is empty or eoff decreases");
    if (m > 0 && n == 0) return einval("edges need vertices: n == 0 with m > 0");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaGetDevice(&dev);
    raise_pool_threshold(dev);
    if (m == 0) {
        if (count_out) *count_out = 0;
        if (rounds_out) *rounds_out = 0;
        if (weight_out) *weight_out = 0.0;
        return HM_OK;
    }
    // Small inputs: one thread block runs the whole matching (a handle's
    // build, graph and their synchronisations cost more than the matching
    // there). Its repeated-vertex check compares pairs within an edge, so
    // it takes inputs whose edges are at most kSmallMaxSize pins.
    if ((uint64_t)kappa <= kSmallPins) {
        int64_t widest = 0;
        for (int64_t e = 0; e < m; ++e) widest = std::max(widest, eoff[e + 1] - eoff[e]);
        if (widest <= kSmallMaxSize)
            return solve_small(n, m, (uint64_t)kappa, eoff, pins, weights, seed, weighted, edges_out, count_out,
                               rounds_out, weight_out, s);
    }
    // The offsets and weights go first on the caller's stream: the edge phase
    // of the build (their validation, the order, the edge offsets) needs only
    // them and runs while the pins still cross the host link, in chunks, on a
    // second stream; each chunk is relabelled as soon as it has arrived.
    // Below 4M pins (16 MB, under 0.1 ms on the link) the overlap saves less
    // than the stream and events cost: the pins follow on the caller's stream
    // and the build reads them from the device like hm_create.
    constexpr int kChunks = 8;
    const bool chunked = kappa >= (int64_t)1 << 22;
    int64_t *d_eoff = nullptr;
    int32_t *d_pins = nullptr;
    float *d_w = nullptr;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_ew = nullptr, ev_pins[kChunks] = {};
    uint64_t begin[kChunks + 1];
    for (int c = 0; c <= kChunks; ++c) {  // chunk starts on relabel-tile boundaries
        const uint64_t x = (uint64_t)kappa * (uint64_t)c / kChunks;
        begin[c] = c == kChunks ? (uint64_t)kappa : x / kRelabelTile * kRelabelTile;
    }
    cudaError_t e = cudaSuccess;
    if (chunked) {
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_ew, cudaEventDisableTiming);
        for (int c = 0; c < kChunks && e == cudaSuccess; ++c)
            e = cudaEventCreateWithFlags(&ev_pins[c], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_eoff, (size_t)(m + 1) * 8, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_pins, (size_t)(kappa > 0 ? kappa : 1) * 4, s);
    if (e == cudaSuccess && weighted) e = cudaMallocAsync((void **)&d_w, (size_t)(m > 0 ? m : 1) * 4, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_eoff, eoff, (size_t)(m + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && weighted && m > 0)
        e = cudaMemcpyAsync(d_w, weights, (size_t)m * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !chunked && kappa > 0)
        e = cudaMemcpyAsync(d_pins, pins, (size_t)kappa * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && chunked) e = cudaEventRecord(ev_ew, s);
    if (e == cudaSuccess && chunked) e = cudaStreamWaitEvent(cs, ev_ew, 0);
    for (int c = 0; c < kChunks && e == cudaSuccess && chunked; ++c) {
        if (begin[c + 1] > begin[c])
            e = cudaMemcpyAsync(d_pins + begin[c], pins + begin[c], (size_t)(begin[c + 1] - begin[c]) * 4,
                                cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev_pins[c], cs);
    }
    hm_status st = HM_OK;
    if (e != cudaSuccess) st = cuda_fail(e, "hm_solve_host upload");
    hm_handle *h = nullptr;
    if (st == HM_OK) {
        const PinChunks feed{kChunks, begin, ev_pins};
        st = create_handle(&h, n, m, (uint64_t)kappa, d_eoff, d_pins, d_w, seed, weighted, s,
                           chunked ? &feed : nullptr);
    }
    // the inputs are no longer needed once the handle is built; every copy
    // issued on the copy stream has finished before they are freed (on an
    // early failure too), and the caller may reuse its pins at once
    if (cs) cudaStreamSynchronize(cs);
    if (d_eoff) cudaFreeAsync(d_eoff, s);
    if (d_pins) cudaFreeAsync(d_pins, s);
    if (d_w) cudaFreeAsync(d_w, s);
    if (cs) cudaStreamDestroy(cs);
    if (ev_ew) cudaEventDestroy(ev_ew);
    for (auto &x : ev_pins)
        if (x) cudaEventDestroy(x);
    if (st == HM_OK) st = hm_match(h, cuda_stream);
    if (st == HM_OK) st = hm_result(h, edges_out, count_out, rounds_out, weight_out);
    if (h) {
        std::string keep = g_err;
        hm_destroy(h);
        g_err = keep;
    }
    return st;
}

}  // extern "C"
