// rounds.cu - the round loop of locally-maximal hypergraph matching
// (Sec. 3.1, Alg. 1, Alg. 3) on the device.
//
// One round is four kernels:
//   k_argmax    a1: every active vertex v makes T[v] the highest-priority
//               live edge of its list. The list is sorted by decreasing
//               priority and edges only ever die, so T[v] is a cursor that
//               moves forward past dead entries (Alg. 3's argmax; Sec. 4.1
//               keeps T across rounds). When T[v] moves to a new edge e the
//               vertex counts down P[e]; the vertex that brings P[e] to 0 has
//               seen e chosen by all |e| of its vertices (the test P[e] = |e|
//               of Alg. 1, Sec. 4.1) and appends e to the winners.
//   k_win       a2: winners join M; their vertices become matched and emit
//               their remaining adjacency (from the cursor on) as kill ranges.
//   k_kill      a3: every edge in a kill range is deactivated (the vertex-side
//               deactivation of Alg. 1; the writes race benignly, Sec. 4.2).
//   k_round_end a4: counters, termination test, next active list, and the
//               conditional of the CUDA graph's while node.
// The active vertex list is compacted inside k_argmax (vertices that are
// matched or have no live edge left drop out), warp-aggregated.
#include "hm_internal.cuh"

#include <algorithm>
#include <cstdio>

namespace hm {
namespace {

constexpr int kT = 256;        // threads per block of the round kernels
constexpr int kPerSM = 8;      // resident blocks per SM targeted by the grids
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Warp-aggregated append of `val` for the lanes with `pred`; all 32 lanes call.
template <typename T>
__device__ __forceinline__ void warp_append(bool pred, T val, T *out, uint32_t *counter) {
    const unsigned mask = __ballot_sync(kFull, pred);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
    base = __shfl_sync(kFull, base, leader);
    if (pred) out[base + __popc(mask & lanemask_lt())] = val;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(kFull, x, d);
    return x;
}

__global__ void __launch_bounds__(kT) k_init(RoundArgs a) {
    const int64_t total = a.n > a.m ? a.n : a.m;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < total; i += (int64_t)gridDim.x * kT) {
        if (i < a.m) {
            a.alive[i] = 1;
            a.P[i] = (uint32_t)(a.eoffj[i + 1] - a.eoffj[i]);
            a.inM[i] = 0;
        }
        if (i < a.n) a.cur[i] = kCurNone;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        DevState *st = a.st;
        st->round = 1;
        st->parity = 0;
        st->cnt[0] = st->cnt[1] = 0;
        st->nwin = 0;
        st->nitems = 0;
        st->status = HM_OK;
        st->rounds_done = 0;
        st->finished = 0;
        st->fault = 0;
        st->adv = st->kills = st->winpins = st->proposals = 0;
    }
}

// a1: argmax (cursor advance) + proposals + list compaction.
__global__ void __launch_bounds__(kT) k_argmax(RoundArgs a) {
    DevState *st = a.st;
    const int r = st->round;
    const int par = st->parity;
    const uint64_t cnt = r == 1 ? (uint64_t)a.n : st->cnt[par];
    const int32_t *in = par ? a.list1 : a.list0;
    int32_t *out = par ? a.list0 : a.list1;
    uint32_t *out_cnt = &st->cnt[par ^ 1];
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)kT + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * kT) >> 5;
    unsigned long long adv = 0, props = 0;
    for (uint64_t base = warp * 32; base < cnt; base += nwarps * 32) {
        const uint64_t idx = base + lane;
        bool keep = false;
        int32_t v = 0, nb = -1;
        if (idx < cnt) {
            if (r == 1) {
                v = (int32_t)idx;
                const int64_t c0 = a.voff[v], c1 = a.voff[v + 1];
                if (c0 < c1) {  // every edge is live in round 1: T[v] = first entry
                    a.cur[v] = c0;
                    nb = a.vadj[c0];
                    keep = true;
                }
            } else {
                v = in[idx];
                int64_t c = a.cur[v];
                if (c >= 0) {
                    int32_t j = a.vadj[c];
                    if (a.alive[j]) {
                        keep = true;  // T[v] still live: unchanged
                    } else {
                        const int64_t end = a.voff[v + 1];
                        const int64_t c0 = c;
                        for (++c; c < end; ++c) {
                            j = a.vadj[c];
                            if (a.alive[j]) break;
                        }
                        adv += (unsigned long long)(c - c0);
                        if (c < end) {
                            a.cur[v] = c;
                            nb = j;
                            keep = true;
                        } else {
                            a.cur[v] = kCurNone;
                        }
                    }
                }
            }
        }
        bool won = false;
        if (nb >= 0) {
            ++props;
            won = atomicSub(&a.P[nb], 1u) == 1u;
        }
        warp_append<int32_t>(keep, v, out, out_cnt);
        warp_append<int32_t>(won, nb, a.win, &st->nwin);
    }
    adv = warp_sum_u64(adv);
    props = warp_sum_u64(props);
    if (lane == 0) {
        if (adv) atomicAdd(&st->adv, adv);
        if (props) atomicAdd(&st->proposals, props);
    }
}

// a2: warp per winner. Marks e in M and every vertex of e as matched; each
// vertex emits [cursor, end of its list) as kill ranges of <= kKillChunk.
__global__ void __launch_bounds__(kT) k_win(RoundArgs a) {
    DevState *st = a.st;
    const uint32_t nw = st->nwin;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)kT + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * kT) >> 5;
    unsigned long long kills = 0, winpins = 0;
    for (uint64_t w = warp; w < nw; w += nwarps) {
        const int32_t j = a.win[w];
        const int64_t b = a.eoffj[j], e = a.eoffj[j + 1];
        if (lane == 0) {
            a.inM[a.order[j]] = 1;
            winpins += (unsigned long long)(e - b);
        }
        for (int64_t i0 = b; i0 < e; i0 += 32) {
            const int64_t i = i0 + lane;
            int64_t c = 0, end = 0;
            uint32_t nch = 0;
            if (i < e) {
                const int32_t v = a.pinsj[i];
                c = a.cur[v];
                end = a.voff[v + 1];
                // T[v] must point at e: it chose e, and nothing moves it
                if (c >= a.voff[v] && c < end && a.vadj[c] == j) {
                    a.cur[v] = kCurMatched;
                    nch = (uint32_t)((end - c + kKillChunk - 1) / kKillChunk);
                    kills += (unsigned long long)(end - c);
                } else {
                    st->fault = 1;
                }
            }
            // warp exclusive scan of the chunk counts -> item slots
            uint32_t inc = nch;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, inc, d);
                if (lane >= d) inc += y;
            }
            const uint32_t total = __shfl_sync(kFull, inc, 31);
            uint32_t base = 0;
            if (lane == 0 && total) base = atomicAdd(&st->nitems, total);
            base = __shfl_sync(kFull, base, 0);
            uint64_t slot = (uint64_t)base + inc - nch;
            if (slot + nch > a.item_cap) {
                if (nch) st->fault = 2;
                nch = 0;
            }
            for (uint32_t k = 0; k < nch; ++k) {
                const int64_t lo = c + (int64_t)k * kKillChunk;
                const int64_t hi = lo + kKillChunk < end ? lo + kKillChunk : end;
                a.items[slot + k] = KillItem{lo, hi};
            }
        }
    }
    kills = warp_sum_u64(kills);
    winpins = warp_sum_u64(winpins);
    if (lane == 0) {
        if (kills) atomicAdd(&st->kills, kills);
        if (winpins) atomicAdd(&st->winpins, winpins);
    }
}

// a3: deactivate every edge listed in a kill range. Blocks take batches of
// kT ranges; the batch's entries are spread evenly over the block's threads
// by a prefix sum of the range lengths and a binary search per entry.
__global__ void __launch_bounds__(kT) k_kill(RoundArgs a) {
    __shared__ int64_t sbeg[kT];
    __shared__ uint32_t spre[kT + 1];
    __shared__ uint32_t warp_tot[kT / 32];
    DevState *st = a.st;
    const uint32_t ni = min(st->nitems, (uint32_t)a.item_cap);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint64_t ib = (uint64_t)blockIdx.x * kT; ib < ni; ib += (uint64_t)gridDim.x * kT) {
        uint32_t len = 0;
        if (ib + threadIdx.x < ni) {
            const KillItem it = a.items[ib + threadIdx.x];
            sbeg[threadIdx.x] = it.begin;
            len = (uint32_t)(it.end - it.begin);
        }
        uint32_t inc = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, inc, d);
            if (lane >= d) inc += y;
        }
        if (lane == 31) warp_tot[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            uint32_t t = lane < kT / 32 ? warp_tot[lane] : 0;
            uint32_t ti = t;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, ti, d);
                if (lane >= d) ti += y;
            }
            if (lane < kT / 32) warp_tot[lane] = ti - t;
            if (lane == kT / 32 - 1) spre[kT] = ti;
        }
        __syncthreads();
        spre[threadIdx.x] = warp_tot[wid] + inc - len;
        __syncthreads();
        const uint32_t total = spre[kT];
        for (uint32_t k = threadIdx.x; k < total; k += kT) {
            int lo = 0, hi = kT - 1;  // last item with spre[item] <= k
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (spre[mid] <= k) lo = mid; else hi = mid - 1;
            }
            const int64_t pos = sbeg[lo] + (int64_t)(k - spre[lo]);
            a.alive[a.vadj[pos]] = 0;
        }
        __syncthreads();
    }
}

// a4: one thread. Records the round, decides whether another round runs.
__global__ void k_round_end(RoundArgs a) {
    if (threadIdx.x != 0) return;
    DevState *st = a.st;
    const int r = st->round, par = st->parity;
    const uint32_t nw = st->nwin, next = st->cnt[par ^ 1];
    if (r - 1 < kStatRounds) {
        int64_t *row = a.stats + (int64_t)(r - 1) * HM_STATS_COLS;
        row[HM_STAT_ACTIVE] = r == 1 ? a.n : (int64_t)st->cnt[par];
        row[HM_STAT_ADVANCE] = (int64_t)st->adv;
        row[HM_STAT_PROPOSALS] = (int64_t)st->proposals;
        row[HM_STAT_WINNERS] = nw;
        row[HM_STAT_WINPINS] = (int64_t)st->winpins;
        row[HM_STAT_KILLS] = (int64_t)st->kills;
        row[HM_STAT_ITEMS] = st->nitems;
        row[HM_STAT_NEXT] = next;
    }
    int cont = 0;
    if (st->fault) {
        st->status = HM_ECUDA;
    } else if (nw == 0) {
        // No winner: no edge was live at the start of this round. Vertices
        // still holding a live T[v] would contradict that (a vertex repeated
        // inside an edge can never let the edge reach P = 0).
        st->rounds_done = r - 1;
        if (next > 0) st->status = HM_EINVAL;
    } else {
        st->rounds_done = r;
        if (next > 0) {
            if (r >= a.cap) st->status = HM_ETIMEOUT;
            else cont = 1;
        }
    }
    st->nwin = 0;
    st->nitems = 0;
    st->adv = st->kills = st->winpins = st->proposals = 0;
    if (cont) {
        st->round = r + 1;
        st->parity = par ^ 1;
        st->cnt[par] = 0;
    } else {
        st->finished = 1;
    }
    if (a.use_cond) cudaGraphSetConditional(a.cond, cont ? 1u : 0u);
}

__global__ void k_vertex_state(const int64_t *cur, const int32_t *vadj, const int32_t *order,
                               int64_t n, int32_t *out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = cur[v];
        out[v] = c >= 0 ? order[vadj[c]] : (c == kCurMatched ? HM_VERTEX_MATCHED : HM_VERTEX_NONE);
    }
}

unsigned round_grid(const Handle *h) { return (unsigned)std::max(1, h->sm_count * kPerSM); }

void launch_round(const Handle *h, const RoundArgs &a, cudaStream_t s, cudaEvent_t *ev) {
    const unsigned g = round_grid(h);
    if (ev) cudaEventRecord(ev[0], s);
    k_argmax<<<g, kT, 0, s>>>(a);
    if (ev) cudaEventRecord(ev[1], s);
    k_win<<<g, kT, 0, s>>>(a);
    if (ev) cudaEventRecord(ev[2], s);
    k_kill<<<g, kT, 0, s>>>(a);
    if (ev) cudaEventRecord(ev[3], s);
    k_round_end<<<1, 32, 0, s>>>(a);
    if (ev) cudaEventRecord(ev[4], s);
}

unsigned init_grid(const Handle *h) {
    return grid_for((uint64_t)std::max(h->n, h->m), kT, h->sm_count, 16);
}

template <typename T>
hm_status dalloc(T **p, uint64_t count, cudaStream_t s, const char *what) {
    cudaError_t e = cudaMallocAsync((void **)p, (size_t)std::max<uint64_t>(count, 1) * sizeof(T), s);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        char buf[160];
        snprintf(buf, sizeof buf, "out of device memory allocating %s (%llu bytes)", what,
                 (unsigned long long)(count * sizeof(T)));
        set_error(buf);
        return HM_ENOMEM;
    }
    return HM_OK;
}

hm_status build_graph(Handle *h) {
    cudaError_t e;
    if (h->exec) {
        cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
    }
    if (!h->cap_stream) {
        e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    }
    cudaGraph_t g = nullptr;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
    struct G {
        cudaGraph_t g;
        ~G() { cudaGraphDestroy(g); }
    } guard{g};
    cudaGraphConditionalHandle cond;
    if ((e = cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphConditionalHandleCreate");
    RoundArgs a = round_args(h);
    a.cond = cond;
    a.use_cond = 1;

    // init node
    if ((e = cudaStreamBeginCaptureToGraph(h->cap_stream, g, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "capture (init)");
    k_init<<<init_grid(h), kT, 0, h->cap_stream>>>(a);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(h->cap_stream, &out);
    if (e != cudaSuccess) return cuda_fail(e, "end capture (init)");
    size_t nn = 0;
    cudaGraphNode_t init_node = nullptr;
    if ((e = cudaGraphGetNodes(g, nullptr, &nn)) != cudaSuccess || nn != 1)
        return cuda_fail(e == cudaSuccess ? cudaErrorUnknown : e, "graph init node");
    if ((e = cudaGraphGetNodes(g, &init_node, &nn)) != cudaSuccess) return cuda_fail(e, "graph nodes");

    // while node around one round
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if ((e = cudaGraphAddNode(&wnode, g, &init_node, nullptr, 1, &cp)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphAddNode (while)");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "capture (round)");
    launch_round(h, a, h->cap_stream, nullptr);
    e = cudaStreamEndCapture(h->cap_stream, &out);
    if (e != cudaSuccess) return cuda_fail(e, "end capture (round)");
    if ((e = cudaGraphInstantiate(&h->exec, g, 0)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphInstantiate");
    h->graph_cap = h->cap;
    return HM_OK;
}

}  // namespace

RoundArgs round_args(const Handle *h) {
    RoundArgs a{};
    a.st = h->st;
    a.voff = h->voff;
    a.vadj = h->vadj;
    a.eoffj = h->eoffj;
    a.pinsj = h->pinsj;
    a.order = h->order;
    a.alive = h->alive;
    a.P = h->P;
    a.cur = h->cur;
    a.list0 = h->list0;
    a.list1 = h->list1;
    a.win = h->win;
    a.items = h->items;
    a.inM = h->inM;
    a.stats = h->stats;
    a.n = h->n;
    a.m = h->m;
    a.cap = h->cap;
    a.item_cap = h->item_cap;
    a.win_cap = h->win_cap;
    a.use_cond = 0;
    return a;
}

hm_status alloc_round_state(Handle *h, cudaStream_t s) {
    const uint64_t n = (uint64_t)h->n, m = (uint64_t)h->m;
    h->win_cap = std::min(n, m) + 1;
    h->item_cap = n + h->kappa / kKillChunk + 1;
    hm_status st;
    if ((st = dalloc(&h->alive, m, s, "alive")) != HM_OK) return st;
    if ((st = dalloc(&h->P, m, s, "P")) != HM_OK) return st;
    if ((st = dalloc(&h->cur, n, s, "cursors")) != HM_OK) return st;
    if ((st = dalloc(&h->list0, n, s, "active list")) != HM_OK) return st;
    if ((st = dalloc(&h->list1, n, s, "active list")) != HM_OK) return st;
    if ((st = dalloc(&h->win, h->win_cap, s, "winners")) != HM_OK) return st;
    if ((st = dalloc(&h->items, h->item_cap, s, "kill items")) != HM_OK) return st;
    if ((st = dalloc(&h->inM, m, s, "result mask")) != HM_OK) return st;
    if ((st = dalloc(&h->stats, (uint64_t)kStatRounds * HM_STATS_COLS, s, "round stats")) != HM_OK) return st;
    if ((st = dalloc(&h->st, 1, s, "loop state")) != HM_OK) return st;
    if ((st = dalloc(&h->res_idx, m, s, "result ids")) != HM_OK) return st;
    if ((st = dalloc(&h->res_w, m, s, "result weights")) != HM_OK) return st;
    if ((st = dalloc(&h->res_part, compact_scratch_elems(m) + 1, s, "result scratch")) != HM_OK) return st;
    cudaError_t e = cudaMemsetAsync(h->stats, 0, (size_t)kStatRounds * HM_STATS_COLS * sizeof(int64_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "stats reset");
    if (cudaMallocHost((void **)&h->h_st, sizeof(DevState)) != cudaSuccess) {
        cudaGetLastError();
        set_error("out of pinned host memory");
        return HM_ENOMEM;
    }
    return HM_OK;
}

hm_status launch_match_graph(Handle *h, cudaStream_t s) {
    if (!h->exec || h->graph_cap != h->cap) {
        hm_status st = build_graph(h);
        if (st != HM_OK) return st;
    }
    cudaError_t e = cudaGraphLaunch(h->exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return HM_OK;
}

hm_status profile_match(Handle *h, cudaStream_t s, double *ms, int64_t *launches) {
    for (int k = 0; k < HM_K_COUNT; ++k) {
        ms[k] = 0;
        launches[k] = 0;
    }
    cudaEvent_t ev[6];
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    struct E {
        cudaEvent_t *ev;
        ~E() {
            for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
        }
    } guard{ev};
    RoundArgs a = round_args(h);
    float t = 0;
    cudaEventRecord(ev[5], s);
    k_init<<<init_grid(h), kT, 0, s>>>(a);
    cudaEventRecord(ev[0], s);
    cudaError_t e = cudaEventSynchronize(ev[0]);
    if (e != cudaSuccess) return cuda_fail(e, "profile init");
    cudaEventElapsedTime(&t, ev[5], ev[0]);
    ms[HM_K_INIT] += t;
    launches[HM_K_INIT] += 1;
    for (;;) {
        launch_round(h, a, s, ev);
        cudaMemcpyAsync(h->h_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "profile round");
        for (int k = 0; k < 4; ++k) {
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            ms[HM_K_ARGMAX + k] += t;
            launches[HM_K_ARGMAX + k] += 1;
        }
        if (h->h_st->finished) break;
    }
    cudaEventRecord(h->done, s);
    return HM_OK;
}

cudaError_t launch_vertex_state(const Handle *h, int32_t *out_dev, cudaStream_t s) {
    k_vertex_state<<<grid_for((uint64_t)h->n, kT, h->sm_count, 16), kT, 0, s>>>(h->cur, h->vadj, h->order,
                                                                                h->n, out_dev);
    return cudaGetLastError();
}

void free_handle_buffers(Handle *h) {
    void *bufs[] = {h->voff, h->vadj, h->eoffj, h->pinsj, h->order, h->weights, h->alive, h->P,
                    h->cur, h->list0, h->list1, h->win, h->items, h->inM, h->stats, h->st,
                    h->res_idx, h->res_w, h->res_part};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (h->h_st) cudaFreeHost(h->h_st);
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->done) cudaEventDestroy(h->done);
}

}  // namespace hm
