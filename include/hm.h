/*
 * hm.h - C ABI of the GB300 (sm_103a) locally-maximal hypergraph matching
 * library (libhm.so).
 *
 * Method: "Efficient Parallel Algorithms for Hypergraph Matching"
 * (Reinstaedtler, Schulz, Sitchinava, Walliser). A weighted hypergraph
 * H = (V, E, w) with w > 0 (Sec. 2.1) is matched in rounds (Sec. 3.1,
 * Alg. 1, Alg. 3): every vertex takes its highest-priority live incident
 * edge, every live edge chosen by all of its vertices joins the matching M,
 * and every live edge touching a vertex of a new matching edge is
 * deactivated; rounds repeat until no edge is live. The result is a maximal
 * matching with w(M) >= OPT/d (Lemma 1).
 *
 * Order on edges. The paper re-draws random weights before every round
 * (Sec. 3.1, Sec. 5.1). This library fixes one strict total order for the
 * whole run instead, which makes the result unique:
 *   weighted:   heavier edge first; equal weight -> smaller edge id first;
 *   unweighted: priority fmix32(e ^ s), s = low 32 bits of the first
 *               SplitMix64 output for `seed` (MurmurHash3 finaliser, Appleby;
 *               SplitMix64, Steele/Lea/Flood 2014). fmix32 is a bijection,
 *               so the order is strict.
 * Under a fixed order the matching equals the sequential greedy matching
 * (sort by priority, take an edge when all its vertices are free; the
 * paper's Greedy baseline, Sec. 5.2).
 *
 * Conventions for every entry point:
 *  - Return value: an hm_status. On failure hm_last_error() returns a
 *    thread-local, NUL-terminated message describing the first problem.
 *  - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Work is enqueued on it in stream order.
 *  - Device pointers must be memory of the current CUDA device (or managed
 *    memory); memory of another GPU is refused with HM_EINVAL. Host
 *    pointers must be ordinary host memory unless stated.
 *  - A handle is bound to the device that was current at hm_create.
 *  - No entry point traps or aborts on bad input; nothing is printed.
 */
#ifndef HM_H
#define HM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hm_handle hm_handle;
typedef struct hm_batch hm_batch;
typedef struct hm_server hm_server;

typedef enum {
    HM_OK = 0,
    HM_EINVAL = 1,    /* invalid argument or invalid hypergraph */
    HM_ENOMEM = 2,    /* a device or host allocation failed */
    HM_ECUDA = 3,     /* a CUDA runtime call failed (message has the CUDA error) */
    HM_ETIMEOUT = 4,  /* the round cap stopped the loop before it finished */
    HM_EBUSY = 5      /* a match on this handle is still running on another stream */
} hm_status;

/* hm_create flags */
#define HM_UNWEIGHTED   0x1u  /* ignore weights (may be NULL); priority = fmix32(e ^ s) */
#define HM_BORROW_INPUT 0x2u  /* accepted for compatibility: inputs are never kept (see hm_create) */
#define HM_VALIDATE     0x4u  /* accepted for compatibility: full validation always runs */
#define HM_AUTOTUNE     0x8u  /* hm_batch_create: autotune every size class's launch shape */
#define HM_ONE_CLASS    0x10u /* hm_batch_create: one size class for all instances (one union, one
                                 build: less setup for small batches; the result is the same) */

/*
 * hm_create - build a matching handle for one hypergraph.
 *
 * Input (edge CSR, the E_id/E_p pair of Sec. 4.1): edge e (0 <= e < m) has
 * the vertices pins[eoff[e] .. eoff[e+1]-1]; kappa = eoff[m] (Sec. 2.1:
 * kappa = sum of edge sizes = sum of degrees).
 *   n        number of vertices, 0 <= n <= 2^31-1 (degree-0 vertices allowed)
 *   m        number of edges,    0 <= m <= 2^31-1
 *   eoff     DEVICE int64[m+1], eoff[0] == 0, strictly increasing (no empty
 *            edge), eoff[m] = kappa <= 2^32-1
 *   pins     DEVICE int32[kappa], every value in [0, n), no vertex twice in
 *            one edge (edges are sets, Sec. 2.1)
 *   weights  DEVICE float32[m], every weight finite and > 0 (Sec. 2.1);
 *            ignored and may be NULL with HM_UNWEIGHTED
 *   seed     priority seed for HM_UNWEIGHTED, otherwise unused
 *   flags    HM_UNWEIGHTED | HM_BORROW_INPUT | HM_VALIDATE
 *   out      receives the handle (set to NULL on failure)
 *
 * Work: validates the input on the device, fixes the order on edges,
 * relabels edges by decreasing priority and builds the vertex CSR (V_id/V_p,
 * Sec. 4.1) with every vertex's edges in decreasing priority. All of it is
 * preprocessing, excluded from match time like the paper's load and
 * transfer time (Sec. 5.1).
 *
 * Ownership: the inputs are only read; they may be freed or changed once
 * hm_create returns (it synchronises `cuda_stream` before returning). The
 * handle owns all device memory it allocates (stream-ordered, on
 * `cuda_stream`) until hm_destroy.
 *
 * Errors: HM_EINVAL for n, m out of range, NULL pointers, eoff[0] != 0,
 * kappa out of range, an empty or decreasing edge range, a pin outside
 * [0, n), a vertex repeated inside an edge, a weight that is not finite or
 * is <= 0 (including -0.0), or NULL weights without HM_UNWEIGHTED;
 * HM_ENOMEM; HM_ECUDA.
 */
hm_status hm_create(hm_handle **out, int64_t n, int64_t m,
                    const int64_t *eoff, const int32_t *pins, const float *weights,
                    uint64_t seed, uint32_t flags, void *cuda_stream);

/*
 * hm_match - enqueue the whole round loop (Alg. 1 / Alg. 3 rounds until no
 * edge is live, Sec. 3.1) on `cuda_stream`; returns without waiting.
 * The loop runs on the device as one CUDA graph with a conditional while
 * node; no host round trip happens between rounds. A handle can be matched
 * any number of times; every call recomputes the same result from scratch.
 * Errors: HM_EINVAL (NULL handle), HM_EBUSY (a match of this handle is still
 * running on a different stream), HM_ECUDA. Loop outcomes (round cap,
 * detected inconsistency) are reported by hm_result.
 */
hm_status hm_match(hm_handle *h, void *cuda_stream);

/*
 * hm_set_round_cap - stop the loop after at most `cap` rounds (cap >= 1).
 * The loop of Sec. 3.1 runs while a live edge exists; the default cap is
 * m + 1, which no valid input reaches: under a strict order the best live
 * edge wins every round, so at most m rounds run.
 * Errors: HM_EINVAL.
 */
hm_status hm_set_round_cap(hm_handle *h, int64_t cap);

/*
 * hm_set_noise - choose the priority rule of the following hm_match and
 * hm_profile_match calls.
 *
 * amplitude == 0 (the default): one fixed strict order for the whole run
 * (the key defined at hm_create).
 * amplitude > 0: the paper's re-randomised rounds (Sec. 3.1: random
 * priorities drawn again before every round; Sec. 5.1). Before round r
 * (1-based) every live edge e gets
 *     p_r(e) = base_e + amplitude * U_r(e)          (float32, the product
 *                                                    and the sum each rounded)
 *     key_r(e) = (bits(p_r(e)) << 32) | (0xFFFFFFFF - e)
 * with base_e = weights[e] (1.0f for HM_UNWEIGHTED), U_r(e) = (top 24 bits
 * of output number (r << 32) + e + 1 of the SplitMix64 generator whose
 * state starts at the first SplitMix64 output for `seed`) * 2^-24, and e the
 * input edge id. A vertex's best edge in round r is its live edge of
 * largest key_r. The result is still unique for a given (input, seed,
 * amplitude). The 1/d bound of Lemma 1 holds for the cardinality of the
 * matching (unweighted input) in this mode; with weights plus noise the
 * matching is locally maximal for the noisy priorities, not for w.
 * The first match with amplitude > 0 allocates 8*kappa + 33*n + 60*m bytes
 * more on the device (12*m more when some edge has more than 65535 pins;
 * 8*kappa + 32*n + 56*m for a graph, every edge with two pins) plus 4 bytes
 * per 1024 pins and a few KB (owned by the handle until hm_destroy).
 * hm_autotune tunes the fixed-order loop and leaves the amplitude set.
 * Errors: HM_EINVAL (NULL handle, amplitude negative, NaN or infinite).
 */
hm_status hm_set_noise(hm_handle *h, float amplitude);

/*
 * hm_launch_config - read and/or set the launch shape of the round kernels
 * (no counterpart in the paper; the result never depends on it).
 *   set  HOST int32[4] or NULL: {least list entries one warp of the kill
 *        kernel takes (64..2^20), blocks per SM of the argmax, win and kill
 *        kernels of the fixed order (0 = as many as fit)}; takes effect at
 *        the next hm_match. A new handle starts at {64, 0, 0, 0}.
 *   get  HOST int32[4] or NULL: the config in force
 * Errors: HM_EINVAL.
 */
hm_status hm_launch_config(hm_handle *h, const int32_t *set, int32_t *get);

/*
 * hm_autotune - pick the launch shape of this handle by measurement (no
 * counterpart in the paper; the result never depends on it): a
 * coordinate-descent search over the least kill slice per warp and the blocks per SM
 * of the three round kernels, each candidate timed as the median of three
 * hm_match graph launches (CUDA events on `cuda_stream`). Leaves the best
 * config applied and reports it (HOST int32[4], as hm_launch_config) and its
 * time in ms. Runs about 40 matches; waits for them. The match result is
 * the same under every config. Errors: as hm_match.
 */
hm_status hm_autotune(hm_handle *h, void *cuda_stream, int32_t *config_out, double *ms_out);

/*
 * hm_result - wait for the last hm_match and report its result.
 *   edges_out   HOST int32[m] or NULL: the matched edge ids, ascending
 *               (input numbering)
 *   count_out   HOST, may be NULL: |M|
 *   rounds_out  HOST, may be NULL: rounds that started with a live edge
 *   weight_out  HOST, may be NULL: w(M) = the exact sum of the matched
 *               float32 weights (Sec. 2.1), rounded once to the nearest
 *               float64, ties to even (|M| for unweighted handles)
 * Errors: HM_EINVAL (NULL handle, no match run yet), HM_ETIMEOUT (the round
 * cap stopped the loop; outputs then describe the partial matching),
 * HM_EINVAL with message "duplicate pin" if a round found no winner while
 * vertices still had live edges (impossible for valid input), HM_ECUDA.
 */
hm_status hm_result(hm_handle *h, int32_t *edges_out, int64_t *count_out,
                    int32_t *rounds_out, double *weight_out);

/*
 * hm_result_device - enqueue on `cuda_stream` a copy of the membership mask
 * of the last match into DEVICE uint8[m] `in_matching` (1 = e in M, the
 * matching of Sec. 2.1), input edge numbering. Does not wait.
 * Errors: HM_EINVAL, HM_ECUDA.
 */
hm_status hm_result_device(hm_handle *h, uint8_t *in_matching, void *cuda_stream);

/*
 * hm_round_stats - per-round counters of the last match (waits for it): the
 * work of every round, whose sum over rounds Sec. 4.3 bounds by O(kappa).
 * For round r (0-based, r < min(rounds_cap, 4096)) row r of HOST
 * int64[max_rounds][HM_STATS_COLS] receives the counters below. In the
 * re-randomised rounds (hm_set_noise) rounds from the second on are
 * edge-driven: there ADVANCE counts the pins tested, PROPOSALS and LIVE the
 * keys offered (the live pins), KILLS the pins of the edges found dead
 * (killed by the previous round's winners), ITEMS is 0, and ACTIVE, NEXT
 * (the vertices offered a key: those active at the round's start) and DEG
 * are counted by hm_profile_match only (0 after hm_match).
 */
#define HM_STAT_ACTIVE    0  /* vertices visited by the argmax step */
#define HM_STAT_ADVANCE   1  /* adjacency entries skipped by the argmax step (fixed
                                order) or scanned by it (re-randomised rounds) */
#define HM_STAT_PROPOSALS 2  /* vertices that chose a new best edge */
#define HM_STAT_WINNERS   3  /* edges that joined M */
#define HM_STAT_WINPINS   4  /* sum of |e| over those edges */
#define HM_STAT_KILLS     5  /* adjacency entries deactivated by the kill step (0 for
                                graphs in the fixed order, which read an edge's
                                liveness from its endpoints and have no kill step) */
#define HM_STAT_ITEMS     6  /* kill ranges (one per newly matched vertex) */
#define HM_STAT_NEXT      7  /* vertices kept for the next round */
#define HM_STAT_LIVE      8  /* re-randomised rounds: live list entries (the live
                                pins) of the round; 0 in the fixed order */
#define HM_STAT_DEG       9  /* after hm_profile_match only (a counting kernel it
                                runs between its timed kernels): sum of the degrees
                                of the vertices kept (HM_STAT_NEXT: the unmatched
                                vertices with a live edge at the start of the
                                round); 0 after hm_match */
#define HM_STAT_LEDGES   10  /* after hm_profile_match only (a counting kernel it runs
                                before each round's timed kernels): edges live at the
                                start of the round; 0 after hm_match */
#define HM_STAT_LPINS    11  /* after hm_profile_match only: sum of |e| over those
                                edges; 0 after hm_match */
#define HM_STATS_COLS     12
/* Returns the number of rows written in *rows_out. Errors: HM_EINVAL. */
hm_status hm_round_stats(hm_handle *h, int64_t *stats, int32_t max_rounds, int32_t *rows_out);

/*
 * hm_vertex_state - per-vertex state after the last match (waits for it),
 * into HOST int32[n]: the input id of the vertex's current best edge, or
 * HM_VERTEX_MATCHED if the vertex is covered by M, or HM_VERTEX_NONE if it
 * has no live edge (or degree 0). After a match stopped by a round cap of r
 * this is T[v] of round r (Alg. 3) for unmatched vertices.
 */
#define HM_VERTEX_MATCHED (-1)
#define HM_VERTEX_NONE    (-2)
hm_status hm_vertex_state(hm_handle *h, int32_t *best_edge_out);

/*
 * hm_profile_match - run one match (Sec. 3.1 rounds, as hm_match) with the
 * rounds driven from the host,
 * one launch per kernel with a CUDA event pair around every launch on
 * `cuda_stream`, and report per kernel kind k (HM_K_*):
 *   ms_out[k]        summed device time of its launches (CUDA events)
 *   launches_out[k]  number of launches
 *   round_ms_out     HOST double[max_rounds][4] or NULL: per round r the
 *                    times of the argmax, win, kill and round-end launches
 *   max_rounds       rows available in round_ms_out (0 if NULL)
 * The result equals hm_match's. Waits for completion. Used to measure each
 * kernel; hm_match is the production path. Errors: as hm_match.
 */
#define HM_K_INIT    0  /* per-match state reset */
#define HM_K_ARGMAX  1  /* a1: vertex argmax (cursor advance) + proposals; in the
                           fixed order also a2's win test (the countdown that
                           reaches 0); the edge rounds' offers */
#define HM_K_WIN     2  /* a2: winners join M, their vertices are marked (the
                           fixed order also emits the kill ranges here); the
                           edge rounds' win test */
#define HM_K_KILL    3  /* a3: deactivate edges of newly matched vertices, and a4 */
#define HM_K_ROUND   4  /* a4: round bookkeeping, termination test: part of the
                           kill kernel, so no launches and no time of its own */
#define HM_K_COUNT   5
hm_status hm_profile_match(hm_handle *h, void *cuda_stream, double *ms_out, int64_t *launches_out,
                           double *round_ms_out, int32_t max_rounds);

/*
 * hm_create_ms - device time of the hm_create phases of this handle (the
 * preprocessing Sec. 5.1 leaves out of the match time; CUDA events):
 * [0] validation, [1] priority sort, [2] edge relabel,
 * [3] vertex CSR build, [4] total. HOST double[5]. Errors: HM_EINVAL.
 */
hm_status hm_create_ms(hm_handle *h, double *ms_out);

/*
 * hm_solve_host - one call from HOST buffers to HOST result (the problem of
 * Sec. 2.1 solved by the rounds of Sec. 3.1, load and transfer included):
 * copies eoff,
 * pins, weights (host memory; pinned memory gives full link bandwidth) to
 * the device on `cuda_stream`, runs hm_create + hm_match + hm_result and
 * frees everything. From 4M pins on, the pins cross in chunks on a second
 * stream while the edge phase of the build runs; the call returns only
 * after every copy has ended, so the caller may reuse its buffers at once.
 * Up to 2^17 pins with no edge above 256 pins, one thread block runs the
 * whole matching instead (same matching, rounds, weight and errors; its
 * working memory comes from the stream's pool, so concurrent calls are
 * safe), which saves the build and graph costs of a handle.
 * Arguments as hm_create and hm_result (edges_out is HOST int32[m] or
 * NULL). Errors: union of those calls.
 */
hm_status hm_solve_host(int64_t n, int64_t m, const int64_t *eoff, const int32_t *pins,
                        const float *weights, uint64_t seed, uint32_t flags,
                        int32_t *edges_out, int64_t *count_out, int32_t *rounds_out,
                        double *weight_out, void *cuda_stream);

/*
 * hm_match_noalloc - match one small hypergraph with one kernel launch and
 * no memory allocation at all. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they
 * need a matching - for example a framework that hands out all device
 * memory from its own arena and allows no other allocator, or a
 * latency-bound loop that cannot afford cudaMalloc's synchronisation. The
 * caller passes inputs and outputs;
 * the working memory is a fixed 8 MiB array declared once in the library
 * (every GPU that loads libhm.so reserves it until the process exits).
 *
 *   n, m, eoff, pins, weights, seed, flags   as hm_create (DEVICE memory)
 *   in_matching  DEVICE uint8[m]: 1 = edge in M (same matching as hm_match)
 *   result       DEVICE int32[2]: [0] = rounds, [1] = hm_status of the run
 *                (HM_OK, or HM_EINVAL for an invalid edge range, pin or
 *                weight; a vertex repeated inside an edge is not rejected
 *                here and counts once)
 *   cuda_stream  the launch is enqueued there; the call does not wait
 *
 * Limit: 9*n + m bytes (each part rounded up to 256) must fit in 8 MiB,
 * e.g. n = 500,000 and m = 3,000,000. Larger inputs return HM_EINVAL with a
 * message naming the size; use hm_create/hm_match for them.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current). All calls share the
 * one array and every call
 * clears the parts it uses, so calls whose kernels overlap on the GPU
 * (different streams, or several host threads) race and corrupt each other;
 * serialise them. Errors returned directly: HM_EINVAL (sizes, flags, NULL or
 * host pointers, or memory of another device than the current one),
 * HM_ECUDA (symbol lookup or launch failure).
 */
hm_status hm_match_noalloc(int64_t n, int64_t m, const int64_t *eoff, const int32_t *pins,
                           const float *weights, uint64_t seed, uint32_t flags,
                           uint8_t *in_matching, int32_t *result, void *cuda_stream);

/*
 * hm_batch_create - many independent hypergraphs, matched together by one
 * graph launch (no counterpart in the paper; it serves a preloaded set of
 * hypergraphs inside a larger computation, the setting of Sec. 5.1).
 *   count    number of instances (>= 1)
 *   n, m     HOST int64[count]: vertices and edges of each instance
 *   eoff     DEVICE int64[sum(m[i]+1)]: each instance's edge offsets as for
 *            hm_create (starting at 0), concatenated in instance order
 *   pins     DEVICE int32[sum(kappa_i)]: instance-local vertex ids, concatenated
 *   weights  DEVICE float32[sum(m[i])], concatenated; NULL with HM_UNWEIGHTED
 *   seed, flags  as hm_create, plus HM_AUTOTUNE and HM_ONE_CLASS
 * Instances are grouped into size classes by kappa (factors of four); each
 * class is matched as the disjoint union of its instances, and all classes
 * are independent branches of one CUDA graph. A class whose every instance
 * has fewer than 65,536 pins (and whose largest instance needs at most 2 MiB
 * of working memory, 9n + m bytes) is instead one persistent kernel of
 * one-block workers, each taking instances from a counter and running all
 * of an instance's rounds inside the block. Every instance gets exactly
 * the matching and round count it would get from its own hm_create/hm_match
 * (unweighted priorities use instance-local edge ids). With HM_AUTOTUNE each
 * union class's launch shape is chosen by hm_autotune's search (a class of
 * one-block workers keeps the default shape, which it does not use). The
 * inputs may be freed once the call returns (it synchronises `cuda_stream`).
 * Errors: HM_EINVAL (as hm_create, per instance; a class beyond 2^31-1
 * vertices or edges or 2^32-1 pins), HM_ENOMEM, HM_ECUDA.
 */
hm_status hm_batch_create(hm_batch **out, int32_t count, const int64_t *n, const int64_t *m,
                          const int64_t *eoff, const int32_t *pins, const float *weights, uint64_t seed,
                          uint32_t flags, void *cuda_stream);

/* hm_batch_match - enqueue the whole batch (one graph launch); does not wait.
 * The batch calls have no counterpart in the paper (see hm_batch_create).
 * Errors: HM_EINVAL, HM_EBUSY (running on another stream), HM_ECUDA. */
hm_status hm_batch_match(hm_batch *b, void *cuda_stream);

/*
 * hm_batch_result - wait for the last hm_batch_match; per instance i:
 *   edges_out    HOST int32[sum(m)] or NULL: instance-local matched edge ids,
 *                ascending, instance after instance (instance i's block starts
 *                at sum of counts_out[k] for k < i)
 *   counts_out   HOST int64[count] or NULL: |M_i|
 *   rounds_out   HOST int32[count] or NULL: rounds instance i takes alone
 *   weights_out  HOST double[count] or NULL: w(M_i), the exact sum rounded
 *                once to float64 as in hm_result (|M_i| when unweighted)
 * Errors: HM_EINVAL, HM_ETIMEOUT / HM_EINVAL / HM_ECUDA if a class's loop did
 * not finish cleanly (outputs are still written), HM_ECUDA.
 */
hm_status hm_batch_result(hm_batch *b, int32_t *edges_out, int64_t *counts_out, int32_t *rounds_out,
                          double *weights_out);

/* hm_batch_info - number of size classes, class of every instance (HOST
 * int32[count] or NULL) and each class's launch shape (HOST
 * int32[nclasses][4] or NULL, as hm_launch_config). Errors: HM_EINVAL. */
hm_status hm_batch_info(hm_batch *b, int32_t *nclasses_out, int32_t *class_of, int32_t *configs);

/* hm_batch_destroy - wait for outstanding work and free the batch. NULL is a no-op. */
void hm_batch_destroy(hm_batch *b);

/*
 * hm_server_create - a request loop with continuous batching (no
 * counterpart in the paper). `slots` worker threads, each with its own CUDA
 * stream on the current device, take requests from a FIFO queue. A free
 * worker admits the queue head and the requests queued right behind it
 * that are compatible (same flags; for HM_UNWEIGHTED the same seed), up to
 * 256 requests and 2^26 pins, as long as their estimated device footprints
 * (36*kappa + 64*m + 72*n bytes + 16 MiB each) fit under the budget:
 * `hbm_budget_bytes`, capped at 90 % of the free device memory at creation
 * (0 = that cap). A lone request runs the hm_solve_host path on the
 * worker's stream; a group runs as one batch (hm_batch_create with
 * HM_ONE_CLASS, one match). Requests arriving while others are on the GPU
 * overlap with them, and each gets the same result as alone.
 * Errors: HM_EINVAL (slots outside [1, 256]), HM_ENOMEM, HM_ECUDA.
 */
hm_status hm_server_create(hm_server **out, int32_t slots, uint64_t hbm_budget_bytes);

/*
 * hm_server_submit - queue one request (the server calls, like
 * hm_server_create, have no counterpart in the paper): HOST eoff/pins/weights as for
 * hm_solve_host (pinned host memory gives full copy bandwidth). The caller
 * keeps the three arrays unchanged until hm_server_wait returns for the
 * ticket. Returns at once with a ticket (> 0).
 * Errors: HM_EINVAL (sizes, eoff), HM_ENOMEM (the request alone exceeds the
 * budget). Input errors found on the device are reported by hm_server_wait.
 */
hm_status hm_server_submit(hm_server *s, int64_t n, int64_t m, const int64_t *eoff, const int32_t *pins,
                           const float *weights, uint64_t seed, uint32_t flags, int64_t *ticket_out);

/*
 * hm_server_wait - wait for a ticket and collect its result (once): outputs
 * as hm_result (edges_out HOST int32[m] or NULL), plus latency_ms_out (may
 * be NULL): milliseconds from hm_server_submit to completion.
 * Errors: HM_EINVAL (unknown ticket), or the request's own status.
 */
hm_status hm_server_wait(hm_server *s, int64_t ticket, int32_t *edges_out, int64_t *count_out,
                         int32_t *rounds_out, double *weight_out, double *latency_ms_out);

/* hm_server_stats - HOST int64[9]: completed, queued, in flight, peak in
 * flight, reserved bytes, peak reserved bytes, budget, units of work started
 * (single requests or groups), largest group. Errors: HM_EINVAL. */
hm_status hm_server_stats(hm_server *s, int64_t *stats_out);

/* hm_server_destroy - finish every submitted request, stop the workers and
 * free the server (results not yet collected are dropped). NULL is a no-op. */
void hm_server_destroy(hm_server *s);

/* hm_last_error - message of the last failure on this thread ("" if none; no
 * counterpart in the paper, nor has any of the lifetime calls). */
const char *hm_last_error(void);

/* hm_destroy - wait for outstanding work of the handle and free it. NULL is a no-op. */
void hm_destroy(hm_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* HM_H */
