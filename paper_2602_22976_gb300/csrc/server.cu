// server.cu - hm_server: a request loop in front of the matcher with
// continuous batching (no counterpart in the paper; serves the paper's
// setting of hypergraphs arriving inside a larger computation, Sec. 5.1).
//
// Requests (host edge CSR) enter a FIFO queue. `slots` worker threads, each
// with its own CUDA stream, admit work as soon as a slot is free and its
// estimated device footprint fits under the HBM budget. A free worker takes
// the queue head and every compatible request queued right behind it (up
// to kGroupMax requests and kGroupPins pins, within the budget): a lone
// request runs the public single-instance path (upload, hm_create,
// hm_match, hm_result); a group runs as one batch (one upload into
// concatenated buffers, hm_batch_create with all instances in one union,
// one graph launch, hm_batch_result), so under load the per-request setup
// is paid once per group. Requests that arrive while others are on the GPU
// are admitted as slots and memory free up, and their kernels run
// concurrently with the others'. Batched instances are disjoint inside the
// union, so every request gets exactly the result it gets alone.
#include "hm_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

namespace hm {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    int64_t n = 0, m = 0;
    uint64_t kappa = 0;
    const int64_t *eoff = nullptr;
    const int32_t *pins = nullptr;
    const float *w = nullptr;
    uint64_t seed = 0;
    uint32_t flags = 0;
    uint64_t bytes = 0;  // admission estimate
    Clock::time_point t_submit, t_start, t_done;
    bool done = false;
    hm_status status = HM_OK;
    std::string err;
    std::vector<int32_t> edges;
    int64_t count = 0;
    int32_t rounds = 0;
    double weight = 0;
};

struct Server {
    int device = 0;
    int slots = 0;
    uint64_t budget = 0;
    uint64_t reserved = 0, peak_reserved = 0;
    int64_t inflight = 0, peak_inflight = 0, done_count = 0;
    int64_t groups = 0, peak_group = 0;  // units of work started, largest group
    int64_t next_ticket = 1;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<int64_t, std::shared_ptr<Request>> live;  // submitted, not yet collected
    std::vector<std::thread> workers;
};

constexpr size_t kGroupMax = 256;              // requests per group
constexpr uint64_t kGroupPins = 64ull << 20;   // pins per group

// Device bytes one request may hold at its peak (hm_create temporaries plus
// the handle and the uploaded input), with slack for allocator rounding.
uint64_t footprint(int64_t n, int64_t m, uint64_t kappa) {
    return 36 * kappa + 64 * (uint64_t)m + 72 * (uint64_t)n + (16ull << 20);
}

// Requests that can share one batch: the same flags, and for unweighted
// input the same seed (its hash priorities depend on the seed; the
// weighted order depends on the weights and local edge ids only).
bool compatible(const Request &a, const Request &b) {
    if (a.flags != b.flags) return false;
    return !(a.flags & HM_UNWEIGHTED) || a.seed == b.seed;
}

void solve_alone(Request &r, cudaStream_t s) {
    r.edges.resize((size_t)std::max<int64_t>(r.m, 1));
    r.status = hm_solve_host(r.n, r.m, r.eoff, r.pins, r.w, r.seed, r.flags, r.edges.data(), &r.count, &r.rounds,
                             &r.weight, s);
    if (r.status != HM_OK) r.err = hm_last_error();
    r.edges.resize(r.status == HM_OK ? (size_t)r.count : 0);
}

// A group as one batch. If anything fails (an invalid request among them,
// say), every request of the group runs alone, so each reports its own
// status.
void solve_group(std::vector<std::shared_ptr<Request>> &g, cudaStream_t s) {
    const int32_t cnt = (int32_t)g.size();
    std::vector<int64_t> n(cnt), m(cnt);
    uint64_t E = 0, K = 0, M = 0;
    for (int32_t i = 0; i < cnt; ++i) {
        n[i] = g[i]->n;
        m[i] = g[i]->m;
        E += (uint64_t)g[i]->m + 1;
        K += g[i]->kappa;
        M += (uint64_t)g[i]->m;
    }
    const bool weighted = !(g[0]->flags & HM_UNWEIGHTED);
    int64_t *d_eoff = nullptr;
    int32_t *d_pins = nullptr;
    float *d_w = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&d_eoff, E * 8, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_pins, std::max<uint64_t>(K, 1) * 4, s);
    if (e == cudaSuccess && weighted) e = cudaMallocAsync((void **)&d_w, std::max<uint64_t>(M, 1) * 4, s);
    uint64_t eo = 0, po = 0, wo = 0;
    for (int32_t i = 0; i < cnt && e == cudaSuccess; ++i) {
        const Request &r = *g[i];
        e = cudaMemcpyAsync(d_eoff + eo, r.eoff, ((size_t)r.m + 1) * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && r.kappa)
            e = cudaMemcpyAsync(d_pins + po, r.pins, (size_t)r.kappa * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && weighted && r.m)
            e = cudaMemcpyAsync(d_w + wo, r.w, (size_t)r.m * 4, cudaMemcpyHostToDevice, s);
        eo += (uint64_t)r.m + 1;
        po += r.kappa;
        wo += (uint64_t)r.m;
    }
    hm_status st = e == cudaSuccess ? HM_OK : HM_ECUDA;
    if (e != cudaSuccess) cudaGetLastError();
    hm_batch *b = nullptr;
    if (st == HM_OK)
        st = hm_batch_create(&b, cnt, n.data(), m.data(), d_eoff, d_pins, d_w, g[0]->seed,
                             g[0]->flags | HM_ONE_CLASS, s);
    if (d_eoff) cudaFreeAsync(d_eoff, s);
    if (d_pins) cudaFreeAsync(d_pins, s);
    if (d_w) cudaFreeAsync(d_w, s);
    std::vector<int32_t> edges((size_t)std::max<uint64_t>(M, 1));
    std::vector<int64_t> counts(cnt, 0);
    std::vector<int32_t> rounds(cnt, 0);
    std::vector<double> weights(cnt, 0.0);
    if (st == HM_OK) st = hm_batch_match(b, s);
    if (st == HM_OK) st = hm_batch_result(b, edges.data(), counts.data(), rounds.data(), weights.data());
    hm_batch_destroy(b);
    if (st != HM_OK) {
        for (auto &r : g) solve_alone(*r, s);
        return;
    }
    size_t off = 0;
    for (int32_t i = 0; i < cnt; ++i) {
        Request &r = *g[i];
        r.edges.assign(edges.begin() + (ptrdiff_t)off, edges.begin() + (ptrdiff_t)(off + (size_t)counts[i]));
        off += (size_t)counts[i];
        r.count = counts[i];
        r.rounds = rounds[i];
        r.weight = weights[i];
        r.status = HM_OK;
    }
}

void worker(Server *S) {
    cudaSetDevice(S->device);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (;;) {
        std::vector<std::shared_ptr<Request>> g;
        uint64_t bytes = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                return S->stop || (!S->queue.empty() && S->reserved + S->queue.front()->bytes <= S->budget);
            });
            if (S->stop) break;
            g.push_back(S->queue.front());
            S->queue.pop_front();
            bytes = g[0]->bytes;
            uint64_t pins = g[0]->kappa;
            // the compatible requests queued right behind the head (FIFO order kept)
            while (!S->queue.empty() && g.size() < kGroupMax) {
                const std::shared_ptr<Request> &q = S->queue.front();
                if (!compatible(*g[0], *q) || pins + q->kappa > kGroupPins ||
                    S->reserved + bytes + q->bytes > S->budget)
                    break;
                bytes += q->bytes;
                pins += q->kappa;
                g.push_back(q);
                S->queue.pop_front();
            }
            S->reserved += bytes;
            S->peak_reserved = std::max(S->peak_reserved, S->reserved);
            S->inflight += (int64_t)g.size();
            S->peak_inflight = std::max(S->peak_inflight, S->inflight);
            S->groups += 1;
            S->peak_group = std::max<int64_t>(S->peak_group, (int64_t)g.size());
        }
        const Clock::time_point t0 = Clock::now();
        for (auto &r : g) r->t_start = t0;
        if (g.size() == 1) solve_alone(*g[0], s);
        else solve_group(g, s);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const Clock::time_point t1 = Clock::now();
            for (auto &r : g) {
                r->t_done = t1;
                r->done = true;
            }
            S->reserved -= bytes;
            S->inflight -= (int64_t)g.size();
            S->done_count += (int64_t)g.size();
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();  // memory was released: the queue head may fit now
    }
    cudaStreamDestroy(s);
}

hm_status bad(const char *msg) {
    set_error(msg);
    return HM_EINVAL;
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" {

hm_status hm_server_create(hm_server **out, int32_t slots, uint64_t hbm_budget_bytes) {
    if (!out) return bad("out is NULL");
    *out = nullptr;
    if (slots < 1 || slots > 256) return bad("slots must be in [1, 256]");
    Server *S = new (std::nothrow) Server();
    if (!S) return HM_ENOMEM;
    cudaError_t e = cudaGetDevice(&S->device);
    if (e != cudaSuccess) {
        delete S;
        return cuda_fail(e, "cudaGetDevice");
    }
    size_t free_b = 0, total_b = 0;
    if ((e = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess) {
        delete S;
        return cuda_fail(e, "cudaMemGetInfo");
    }
    const uint64_t cap = (uint64_t)((double)free_b * 0.9);
    S->budget = hbm_budget_bytes ? std::min<uint64_t>(hbm_budget_bytes, cap) : cap;
    S->slots = slots;
    try {
        for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker, S);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
        }
        S->cv_work.notify_all();
        for (auto &t : S->workers) t.join();
        delete S;
        return bad("could not start the worker threads");
    }
    *out = reinterpret_cast<hm_server *>(S);
    return HM_OK;
}

hm_status hm_server_submit(hm_server *ss, int64_t n, int64_t m, const int64_t *eoff, const int32_t *pins,
                           const float *weights, uint64_t seed, uint32_t flags, int64_t *ticket_out) {
    Server *S = reinterpret_cast<Server *>(ss);
    if (!S) return bad("server is NULL");
    if (!ticket_out) return bad("ticket_out is NULL");
    if (n < 0 || m < 0 || n > INT32_MAX || m > INT32_MAX) return bad("n, m must be in [0, 2^31-1]");
    if (!eoff) return bad("eoff is NULL");
    if (eoff[0] != 0 || eoff[m] < m || (uint64_t)eoff[m] > 0xFFFFFFFFull)
        return bad("eoff[0] must be 0 and eoff[m] in [m, 2^32-1]");
    auto r = std::make_shared<Request>();
    r->n = n;
    r->m = m;
    r->kappa = (uint64_t)eoff[m];
    r->eoff = eoff;
    r->pins = pins;
    r->w = weights;
    r->seed = seed;
    r->flags = flags;
    r->bytes = footprint(n, m, r->kappa);
    if (r->bytes > S->budget) {
        set_error("request needs more device memory than the server's budget");
        return HM_ENOMEM;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return bad("server is shutting down");
        r->ticket = S->next_ticket++;
        r->t_submit = Clock::now();
        S->queue.push_back(r);
        S->live.emplace(r->ticket, r);
    }
    S->cv_work.notify_one();
    *ticket_out = r->ticket;
    return HM_OK;
}

hm_status hm_server_wait(hm_server *ss, int64_t ticket, int32_t *edges_out, int64_t *count_out,
                         int32_t *rounds_out, double *weight_out, double *latency_ms_out) {
    Server *S = reinterpret_cast<Server *>(ss);
    if (!S) return bad("server is NULL");
    std::shared_ptr<Request> r;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->live.find(ticket);
        if (it == S->live.end()) return bad("unknown or already collected ticket");
        r = it->second;
        S->cv_done.wait(lk, [&] { return r->done; });
        S->live.erase(ticket);  // the map may have rehashed while we waited
    }
    if (edges_out && r->count) memcpy(edges_out, r->edges.data(), (size_t)r->count * 4);
    if (count_out) *count_out = r->count;
    if (rounds_out) *rounds_out = r->rounds;
    if (weight_out) *weight_out = r->weight;
    if (latency_ms_out)
        *latency_ms_out = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (r->status != HM_OK) set_error(r->err);
    return r->status;
}

hm_status hm_server_stats(hm_server *ss, int64_t *stats_out) {
    Server *S = reinterpret_cast<Server *>(ss);
    if (!S || !stats_out) return bad("NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    stats_out[0] = S->done_count;
    stats_out[1] = (int64_t)S->queue.size();
    stats_out[2] = S->inflight;
    stats_out[3] = S->peak_inflight;
    stats_out[4] = (int64_t)S->reserved;
    stats_out[5] = (int64_t)S->peak_reserved;
    stats_out[6] = (int64_t)S->budget;
    stats_out[7] = S->groups;
    stats_out[8] = S->peak_group;
    return HM_OK;
}

void hm_server_destroy(hm_server *ss) {
    Server *S = reinterpret_cast<Server *>(ss);
    if (!S) return;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        // finish what was submitted, then stop the workers
        S->cv_done.wait(lk, [&] { return S->queue.empty() && S->inflight == 0; });
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    delete S;
}

}  // extern "C"
