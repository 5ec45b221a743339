/*
 * oracle.c - plain, sequential CPU oracle for locally-maximal hypergraph
 * matching ("Efficient Parallel Algorithms for Hypergraph Matching",
 * Reinstaedtler, Schulz, Sitchinava, Walliser).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg and reference arm may load this library. It
 * shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (Sec. 3.1 "Sequential Algorithm", Alg. 1 and Alg. 3):
 * rounds; in each round every vertex determines its highest-priority live
 * incident edge, every live edge chosen by all of its vertices joins the
 * matching, and every live edge that touches a vertex of a new matching
 * edge is deactivated (soft delete, Sec. 3.1). Rounds repeat until no edge
 * is live. The maximality argument of Sec. 3.1 bounds the loop.
 *
 * Strict total order on edges (the reading used throughout this project):
 *   key(e) = (bits(w_e) << 32) | (0xFFFFFFFF - e)        weighted input
 *   key(e) = (bits(1.0f) << 32) | fmix32(e ^ s)           unweighted input
 * with s = low 32 bits of the first SplitMix64 output for `seed`. A larger
 * key wins. Positive finite float32 bit patterns order like the values
 * (weights are positive, Sec. 2.1), so the weighted order is "heavier wins,
 * equal weight -> smaller edge id wins". fmix32 is the MurmurHash3 32-bit
 * finaliser (Appleby); SplitMix64 is from Steele, Lea, Flood (OOPSLA 2014).
 * The paper instead re-draws random weights every round (Sec. 3.1, Sec. 5.1);
 * the fixed order makes the result unique and so exactly comparable. With
 * noise > 0 the rounds follow the paper instead: before round r every edge
 * gets the priority p_r(e) = base_e + noise * U_r(e) in float32 arithmetic
 * (base_e = w_e, or 1.0f for unweighted input; U_r(e) in [0,1) is the top 24
 * bits of output number (r << 32) + e + 1 of a SplitMix64 stream whose
 * state starts at the first SplitMix64 output for `seed`, times 2^-24), and
 * key_r(e) = (bits(p_r(e)) << 32) | (0xFFFFFFFF - e).
 *
 * Also here: the sequential greedy algorithm (sort by key, take an edge when
 * all its vertices are free; the paper's single-core baseline, Sec. 5.2),
 * an exhaustive maximum-weight matching for tiny inputs (Lemma 1 checks) and
 * checkers for the matching / maximality / local-maximality properties
 * (Sec. 2.1 definitions).
 *
 * Build: gcc -O2 -shared -fPIC -std=c11 oracle.c -o liboracle.so
 * Compile-time ORACLE_MUTANT=k plants a deliberate mistake (tests only).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* ---------------------------------------------------------- priorities */

uint64_t oracle_splitmix64_first(uint64_t seed)
{
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint32_t oracle_fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

/* Output number k (k >= 1) of SplitMix64 started at state s0. */
uint64_t oracle_splitmix64_at(uint64_t s0, uint64_t k)
{
    uint64_t z = s0 + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint32_t float_bits(float f)
{
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return u;
}

/* key(e) as defined in the header comment */
uint64_t oracle_key(const float *w, int unweighted, uint64_t seed, int64_t e)
{
    if (unweighted) {
        uint32_t s = (uint32_t)oracle_splitmix64_first(seed);
        return ((uint64_t)float_bits(1.0f) << 32) | oracle_fmix32((uint32_t)e ^ s);
    }
#if ORACLE_MUTANT == 1 /* tie-break reversed: larger id wins */
    return ((uint64_t)float_bits(w[e]) << 32) | (uint64_t)(uint32_t)e;
#else
    return ((uint64_t)float_bits(w[e]) << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)e);
#endif
}

/* Per-round priority p_r(e) of the re-randomised rounds (see header). */
float oracle_round_priority(const float *w, int unweighted, uint64_t seed, float noise, int64_t r, int64_t e)
{
    uint64_t s0 = oracle_splitmix64_first(seed);
    uint64_t h = oracle_splitmix64_at(s0, ((uint64_t)r << 32) + (uint64_t)e + 1u);
    float u24 = (float)(uint32_t)(h >> 40);
    float scaled = u24 * (noise * (1.0f / 16777216.0f));
    float base = unweighted ? 1.0f : w[e];
    return base + scaled;
}

static uint64_t round_key(const float *w, int unweighted, uint64_t seed, float noise, int64_t r, int64_t e)
{
    float p = oracle_round_priority(w, unweighted, seed, noise, r, e);
    return ((uint64_t)float_bits(p) << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)e);
}

static uint64_t *all_keys(int64_t m, const float *w, int unweighted, uint64_t seed)
{
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
    if (!key) return NULL;
    for (int64_t e = 0; e < m; ++e) key[e] = oracle_key(w, unweighted, seed, e);
    return key;
}

/* ---------------------------------------------------------- round loop */

/*
 * Runs the rounds. Outputs (all caller-owned, host memory):
 *   in_matching[m]    1 if e is in M, else 0
 *   decided_round[m]  round (1-based) in which e was matched or deactivated
 *                     (NULL allowed)
 *   round_stats[3*max_rounds]  per round r (0-based): live edges at the start,
 *                     live pins at the start, edges matched (NULL allowed;
 *                     only written when max_rounds > 0)
 *   rounds_out        number of rounds that started with a live edge
 *   best_edge_out[n]  T[v] of the last round run (Alg. 3): the edge with the
 *                     largest key among v's live edges at the start of that
 *                     round, or -2 if v had none (NULL allowed)
 *   matched_out[n]    1 if v is covered by M after the last round (NULL allowed)
 * noise == 0: one fixed order for the whole run; noise > 0: priorities
 * re-drawn before every round (see header).
 * max_rounds <= 0 means no cap. Returns 0 when every edge is decided, 1 when
 * the cap stopped the loop first, -1 on allocation failure.
 */
int oracle_match(int64_t n, int64_t m, const int64_t *eoff, const int32_t *pins,
                 const float *w, int unweighted, uint64_t seed, float noise, int64_t max_rounds,
                 uint8_t *in_matching, int32_t *decided_round, int64_t *round_stats,
                 int32_t *rounds_out, int32_t *best_edge_out, uint8_t *matched_out)
{
    const uint64_t NONE = 0; /* every real key is > 0: weights are > 0 */
    uint64_t *key = all_keys(m, w, unweighted, seed);
    uint64_t *best = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *alive = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    uint8_t *matched = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t *winners = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t *best_e = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!key || !best || !alive || !matched || !winners || !best_e) {
        free(key); free(best); free(alive); free(matched); free(winners); free(best_e);
        return -1;
    }
    for (int64_t v = 0; v < n; ++v) best_e[v] = -2;
    for (int64_t e = 0; e < m; ++e) {
        alive[e] = 1;
        in_matching[e] = 0;
        if (decided_round) decided_round[e] = 0;
    }
    int64_t live = m;
    int32_t r = 0;
    int status = 0;
    while (live > 0) {
        if (max_rounds > 0 && r >= max_rounds) { status = 1; break; }
        r += 1;
        int64_t live_pins = 0;
#if ORACLE_MUTANT == 6 /* priorities drawn once, not before every round */
        if (noise > 0.0f && r == 1)
#else
        if (noise > 0.0f) /* re-draw the priorities of the live edges */
#endif
            for (int64_t e = 0; e < m; ++e)
                if (alive[e]) key[e] = round_key(w, unweighted, seed, noise, r, e);
        /* step 1: best[v] = max key over live edges containing v */
        for (int64_t v = 0; v < n; ++v) { best[v] = NONE; best_e[v] = -2; }
        for (int64_t e = 0; e < m; ++e) {
#if ORACLE_MUTANT == 5 /* dead edges still compete */
            if (alive[e]) live_pins += eoff[e + 1] - eoff[e];
#else
            if (!alive[e]) continue;
            live_pins += eoff[e + 1] - eoff[e];
#endif
            for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i) {
                int32_t v = pins[i];
#if ORACLE_MUTANT == 2 /* argmin instead of argmax */
                if (best[v] == NONE || key[e] < best[v]) { best[v] = key[e]; best_e[v] = e; }
#else
                if (key[e] > best[v]) { best[v] = key[e]; best_e[v] = e; }
#endif
            }
        }
        /* step 2: winners = live edges chosen by all of their vertices */
        int64_t nw = 0;
        for (int64_t e = 0; e < m; ++e) {
            if (!alive[e]) continue;
            int all = 1;
#if ORACLE_MUTANT == 3 /* only the first vertex is consulted */
            for (int64_t i = eoff[e]; i < eoff[e] + 1; ++i)
#else
            for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i)
#endif
                if (best[pins[i]] != key[e]) { all = 0; break; }
            if (all) winners[nw++] = e;
        }
        if (round_stats && max_rounds > 0) {
            round_stats[3 * (r - 1) + 0] = live;
            round_stats[3 * (r - 1) + 1] = live_pins;
            round_stats[3 * (r - 1) + 2] = nw;
        }
        /* step 3: winners join M; their vertices become matched */
        for (int64_t k = 0; k < nw; ++k) {
            int64_t e = winners[k];
            in_matching[e] = 1;
            alive[e] = 0;
            live -= 1;
            if (decided_round) decided_round[e] = r;
            for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i) matched[pins[i]] = 1;
        }
        /* step 4: live edges touching a matched vertex are deactivated */
#if ORACLE_MUTANT != 4 /* mutant 4 drops this step */
        for (int64_t e = 0; e < m; ++e) {
            if (!alive[e]) continue;
            for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i) {
                if (matched[pins[i]]) {
                    alive[e] = 0;
                    live -= 1;
                    if (decided_round) decided_round[e] = r;
                    break;
                }
            }
        }
#else
        if (nw == 0) break;
#endif
    }
    *rounds_out = r;
    for (int64_t v = 0; v < n; ++v) {
        if (best_edge_out) best_edge_out[v] = (int32_t)best_e[v];
        if (matched_out) matched_out[v] = matched[v];
    }
    free(key); free(best); free(alive); free(matched); free(winners); free(best_e);
    return status;
}

/* ---------------------------------------------------------- greedy */

typedef struct { uint64_t key; int64_t e; } keyed_t;

static int by_key_desc(const void *a, const void *b)
{
    uint64_t x = ((const keyed_t *)a)->key, y = ((const keyed_t *)b)->key;
    return x < y ? 1 : (x > y ? -1 : 0);
}

/* Sequential greedy: visit edges by decreasing key, take an edge when all of
 * its vertices are still free (the paper's single-core Greedy baseline). */
int oracle_greedy(int64_t n, int64_t m, const int64_t *eoff, const int32_t *pins,
                  const float *w, int unweighted, uint64_t seed, uint8_t *in_matching)
{
    keyed_t *order = (keyed_t *)malloc(sizeof(keyed_t) * (size_t)(m > 0 ? m : 1));
    uint8_t *used = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!order || !used) { free(order); free(used); return -1; }
    for (int64_t e = 0; e < m; ++e) {
        order[e].key = oracle_key(w, unweighted, seed, e);
        order[e].e = e;
        in_matching[e] = 0;
    }
    qsort(order, (size_t)m, sizeof(keyed_t), by_key_desc);
    for (int64_t k = 0; k < m; ++k) {
        int64_t e = order[k].e;
        int free_all = 1;
        for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i)
            if (used[pins[i]]) { free_all = 0; break; }
        if (!free_all) continue;
        in_matching[e] = 1;
        for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i) used[pins[i]] = 1;
    }
    free(order); free(used);
    return 0;
}

/* ---------------------------------------------------------- exhaustive OPT */

typedef struct {
    int64_t m;
    const uint64_t *mask;
    const double *wt;
    const double *suffix;
    double best;
    uint64_t best_set;
} bb_t;

static void bb(bb_t *s, int64_t i, uint64_t used, double acc, uint64_t set)
{
    if (acc > s->best) { s->best = acc; s->best_set = set; }
    if (i >= s->m || acc + s->suffix[i] <= s->best) return;
    if (!(s->mask[i] & used))
        bb(s, i + 1, used | s->mask[i], acc + s->wt[i], set | (1ULL << i));
    bb(s, i + 1, used, acc, set);
}

/* Maximum-weight matching by branch and bound over all edge subsets, for
 * n <= 64 and m <= 40. Weights are summed in double. Returns -1.0 if the
 * input is too large. best_set[m] receives one optimal matching. */
double oracle_brute_opt(int64_t n, int64_t m, const int64_t *eoff, const int32_t *pins,
                        const float *w, uint8_t *best_set)
{
    if (n > 64 || m > 40) return -1.0;
    uint64_t mask[40];
    double wt[40], suffix[41];
    for (int64_t e = 0; e < m; ++e) {
        mask[e] = 0;
        for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i) mask[e] |= 1ULL << pins[i];
        wt[e] = w ? (double)w[e] : 1.0;
    }
    suffix[m] = 0.0;
    for (int64_t e = m - 1; e >= 0; --e) suffix[e] = suffix[e + 1] + wt[e];
    bb_t s = {m, mask, wt, suffix, 0.0, 0};
    bb(&s, 0, 0, 0.0, 0);
    for (int64_t e = 0; e < m; ++e) best_set[e] = (uint8_t)((s.best_set >> e) & 1);
    return s.best;
}

/* ---------------------------------------------------------- checkers */

/* Sec. 2.1: M is a matching iff its edges are pairwise vertex-disjoint.
 * Returns -1 if so, else the first edge that reuses a vertex. */
int64_t oracle_check_disjoint(int64_t n, int64_t m, const int64_t *eoff, const int32_t *pins,
                              const uint8_t *in_matching)
{
    uint8_t *used = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!used) return -2;
    int64_t bad = -1;
    for (int64_t e = 0; e < m && bad < 0; ++e) {
        if (!in_matching[e]) continue;
        for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i) {
            if (used[pins[i]]) { bad = e; break; }
            used[pins[i]] = 1;
        }
    }
    free(used);
    return bad;
}

/* Sec. 2.1: M is maximal iff every edge outside M shares a vertex with M.
 * Returns -1 if so, else the first edge that could still be added. */
int64_t oracle_check_maximal(int64_t n, int64_t m, const int64_t *eoff, const int32_t *pins,
                             const uint8_t *in_matching)
{
    uint8_t *used = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!used) return -2;
    for (int64_t e = 0; e < m; ++e)
        if (in_matching[e])
            for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i) used[pins[i]] = 1;
    int64_t bad = -1;
    for (int64_t e = 0; e < m && bad < 0; ++e) {
        if (in_matching[e]) continue;
        int hit = 0;
        for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i)
            if (used[pins[i]]) { hit = 1; break; }
        if (!hit) bad = e;
    }
    free(used);
    return bad;
}

/* Local maximality (Sec. 2.1 "locally maximal"; Sec. 3.1): an edge matched in
 * round r is heavier than every edge sharing a vertex with it that was still
 * live at the start of round r (decided in round >= r), under the keys of
 * round r (the fixed keys when noise == 0). Checked vertex by
 * vertex: the matched edge at v must carry the largest key among the edges
 * at v decided in its round or later. Returns -1 if it holds, else the index
 * of an offending vertex. O(kappa) time. */
int64_t oracle_check_local_max(int64_t n, int64_t m, const int64_t *eoff, const int32_t *pins,
                               const float *w, int unweighted, uint64_t seed, float noise,
                               const uint8_t *in_matching, const int32_t *decided_round)
{
    uint64_t *key = all_keys(m, w, unweighted, seed);
    int64_t *mate = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!key || !mate) { free(key); free(mate); return -2; }
    for (int64_t v = 0; v < n; ++v) mate[v] = -1;
    for (int64_t e = 0; e < m; ++e)
        if (in_matching[e])
            for (int64_t i = eoff[e]; i < eoff[e + 1]; ++i) mate[pins[i]] = e;
    int64_t bad = -1;
    for (int64_t f = 0; f < m && bad < 0; ++f) {
        for (int64_t i = eoff[f]; i < eoff[f + 1]; ++i) {
            int64_t v = pins[i], e = mate[v];
            if (e < 0 || e == f) continue;
            if (decided_round[f] < decided_round[e]) continue;
            if (noise > 0.0f) {
                int64_t r = decided_round[e];
                if (round_key(w, unweighted, seed, noise, r, f) > round_key(w, unweighted, seed, noise, r, e)) {
                    bad = v;
                    break;
                }
            } else if (key[f] > key[e]) {
                bad = v;
                break;
            }
        }
    }
    free(key); free(mate);
    return bad;
}
