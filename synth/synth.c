/*
 * synth.c - seeded synthetic hypergraph generators.
 *
 * This module only PRODUCES inputs (edge CSR + float32 weights). It holds
 * none of the matching method's arithmetic and is shared, as an input
 * producer, by the CPU oracle tests and by the GPU path's tests and bench.
 *
 * Shapes follow the instance statistics of the paper (Appendix tables:
 * heavy-tailed edge sizes and vertex degrees, maximum edge size d and
 * maximum degree Delta into the millions) and the weight recipe of the
 * experimental section (random weights; here float32 uniform in (0,1]).
 *
 * Randomness: every edge e owns a SplitMix64 stream (Steele, Lea, Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014) whose start
 * state is derived from (seed, purpose, e). Output is therefore independent
 * of the number of OpenMP threads.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC synth.c -o libsynth.so
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s; } stream_t;

/* purpose tags keep the size, pin, weight and shuffle streams apart */
enum { P_SIZE = 1, P_PIN = 2, P_WEIGHT = 3, P_SHUFFLE = 4, P_BATCH = 5, P_POINT = 7 };

static inline stream_t stream_for(uint64_t seed, uint64_t purpose, uint64_t idx)
{
    stream_t r;
    r.s = sm_mix(sm_mix(seed ^ (purpose * 0xD1B54A32D192ED03ULL)) + idx * GOLDEN);
    return r;
}

static inline uint64_t next64(stream_t *r)
{
    r->s += GOLDEN;
    return sm_mix(r->s);
}

/* uniform integer in [0, bound) by 64x64->128 multiply (Lemire) */
static inline uint64_t below(stream_t *r, uint64_t bound)
{
    return (uint64_t)(((unsigned __int128)next64(r) * bound) >> 64);
}

static inline double unit(stream_t *r) /* [0,1) */
{
    return (double)(next64(r) >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------ sizes */

/* dist 0: uniform integer in [kmin,kmax]; dist 1: Zipf(s) on [kmin,kmax] by
 * inverse CDF over the finite support. Writes eoff[0..m]; returns kappa. */
int64_t synth_sizes(int64_t m, int dist, int kmin, int kmax, double zipf_s,
                    uint64_t seed, int64_t *eoff)
{
    if (m < 0 || kmin < 1 || kmax < kmin) return -1;
    int span = kmax - kmin + 1;
    double *cdf = NULL;
    if (dist == 1) {
        cdf = (double *)malloc(sizeof(double) * (size_t)span);
        if (!cdf) return -1;
        double acc = 0.0;
        for (int k = 0; k < span; ++k) {
            acc += pow((double)(kmin + k), -zipf_s);
            cdf[k] = acc;
        }
        for (int k = 0; k < span; ++k) cdf[k] /= acc;
        cdf[span - 1] = 1.0;
    }
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        stream_t r = stream_for(seed, P_SIZE, (uint64_t)e);
        int k;
        if (dist == 1) {
            double u = unit(&r);
            int lo = 0, hi = span - 1; /* first k with cdf[k] > u */
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (cdf[mid] > u) hi = mid; else lo = mid + 1;
            }
            k = kmin + lo;
        } else {
            k = kmin + (int)below(&r, (uint64_t)span);
        }
        eoff[e + 1] = k;
    }
    free(cdf);
    eoff[0] = 0;
    for (int64_t e = 0; e < m; ++e) eoff[e + 1] += eoff[e];
    return eoff[m];
}

/* ------------------------------------------------------------------- pins */

typedef struct {
    int64_t n;
    float *prob;     /* alias table (Walker / Vose) */
    int32_t *alias;
} alias_t;

/* P(v) proportional to (v+1)^(-alpha), alpha = 1/(gamma-1): the expected
 * degree sequence of a Chung-Lu power-law graph with exponent gamma. */
static int alias_build(alias_t *a, int64_t n, double gamma)
{
    double alpha = 1.0 / (gamma - 1.0);
    a->n = n;
    a->prob = (float *)malloc(sizeof(float) * (size_t)n);
    a->alias = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *small = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *large = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!a->prob || !a->alias || !q || !small || !large) {
        free(a->prob); free(a->alias); free(q); free(small); free(large);
        return -1;
    }
    double sum = 0.0;
    for (int64_t v = 0; v < n; ++v) { q[v] = pow((double)(v + 1), -alpha); sum += q[v]; }
    int64_t ns = 0, nl = 0;
    for (int64_t v = 0; v < n; ++v) {
        q[v] = q[v] * (double)n / sum;
        if (q[v] < 1.0) small[ns++] = (int32_t)v; else large[nl++] = (int32_t)v;
    }
    while (ns > 0 && nl > 0) {
        int32_t s = small[--ns], l = large[nl - 1];
        a->prob[s] = (float)q[s];
        a->alias[s] = l;
        q[l] = (q[l] + q[s]) - 1.0;
        if (q[l] < 1.0) { --nl; small[ns++] = l; }
    }
    while (nl > 0) { int32_t l = large[--nl]; a->prob[l] = 1.0f; a->alias[l] = l; }
    while (ns > 0) { int32_t s = small[--ns]; a->prob[s] = 1.0f; a->alias[s] = s; }
    free(q); free(small); free(large);
    return 0;
}

static inline int32_t alias_draw(const alias_t *a, stream_t *r)
{
    uint64_t x = next64(r);
    int64_t i = (int64_t)(((unsigned __int128)x * (uint64_t)a->n) >> 64);
    float u = (float)(uint32_t)(x & 0xFFFFFF) * (1.0f / 16777216.0f);
    return u < a->prob[i] ? (int32_t)i : a->alias[i];
}

/* dist 0: pins uniform over [0,n); dist 1: power-law (alias table) with the
 * vertex ids relabelled by a seeded permutation when shuffle != 0, so the
 * heaviest vertices are scattered over the id range. No vertex repeats
 * within an edge (rejection). Requires n >= max edge size. */
int synth_pins(int64_t n, int64_t m, const int64_t *eoff, int dist, double gamma,
               int shuffle, uint64_t seed, int32_t *pins)
{
    if (n <= 0 && m > 0) return -1;
    int64_t kmax = 0;
    for (int64_t e = 0; e < m; ++e) {
        int64_t k = eoff[e + 1] - eoff[e];
        if (k > kmax) kmax = k;
    }
    if (kmax > n) return -2;
    alias_t at = {0, NULL, NULL};
    if (dist == 1 && alias_build(&at, n, gamma) != 0) return -3;
    int32_t *perm = NULL;
    if (dist == 1 && shuffle) {
        perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        if (!perm) { free(at.prob); free(at.alias); return -3; }
        for (int64_t v = 0; v < n; ++v) perm[v] = (int32_t)v;
        stream_t r = stream_for(seed, P_SHUFFLE, 0);
        for (int64_t v = n - 1; v > 0; --v) { /* Fisher-Yates */
            int64_t j = (int64_t)below(&r, (uint64_t)(v + 1));
            int32_t t = perm[v]; perm[v] = perm[j]; perm[j] = t;
        }
    }
    int err = 0;
    #pragma omp parallel
    {
        uint64_t *bits = NULL; /* per-thread membership bitmap for big edges */
        #pragma omp for schedule(dynamic, 4096)
        for (int64_t e = 0; e < m; ++e) {
            int64_t b = eoff[e], k = eoff[e + 1] - b;
            int32_t *out = pins + b;
            stream_t r = stream_for(seed, P_PIN, (uint64_t)e);
            int big = k > 32;
            if (big && !bits) {
                bits = (uint64_t *)calloc((size_t)((n + 63) / 64), sizeof(uint64_t));
                if (!bits) { err = 1; continue; }
            }
            for (int64_t i = 0; i < k; ++i) {
                for (;;) {
                    int32_t v = dist == 1 ? alias_draw(&at, &r)
                                          : (int32_t)below(&r, (uint64_t)n);
                    int dup = 0;
                    if (big) {
                        dup = (int)((bits[v >> 6] >> (v & 63)) & 1);
                        if (!dup) bits[v >> 6] |= 1ULL << (v & 63);
                    } else {
                        for (int64_t t = 0; t < i; ++t)
                            if (out[t] == v) { dup = 1; break; }
                    }
                    if (!dup) { out[i] = v; break; }
                }
            }
            if (big)
                for (int64_t i = 0; i < k; ++i) bits[out[i] >> 6] = 0;
            if (perm)
                for (int64_t i = 0; i < k; ++i) out[i] = perm[out[i]];
        }
        free(bits);
    }
    free(perm);
    free(at.prob);
    free(at.alias);
    return err ? -3 : 0;
}

/* float32 weights uniform on the 2^24-point grid {1,2,...,2^24} * 2^-24,
 * i.e. in (0,1]; every value is exact in float32. */
void synth_weights(int64_t m, uint64_t seed, float *w)
{
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        stream_t r = stream_for(seed, P_WEIGHT, (uint64_t)e);
        uint32_t q = (uint32_t)(next64(&r) >> 40) + 1u; /* 1 .. 2^24 */
        w[e] = (float)q * (1.0f / 16777216.0f);
    }
}

/* Per-instance sizes of a batch: n_i = round(exp(U[ln lo, ln hi])). */
void synth_loguniform(int64_t count, double lo, double hi, uint64_t seed, int64_t *out)
{
    double a = log(lo), b = log(hi);
    for (int64_t i = 0; i < count; ++i) {
        stream_t r = stream_for(seed, P_BATCH, (uint64_t)i);
        out[i] = (int64_t)llround(exp(a + (b - a) * unit(&r)));
    }
}

/* Poisson arrival times (seconds) at `rate` per second: exponential gaps. */
void synth_arrivals(int64_t count, double rate, uint64_t seed, double *t)
{
    stream_t r = stream_for(seed, P_BATCH + 1, 0);
    double acc = 0.0;
    for (int64_t i = 0; i < count; ++i) {
        double u = unit(&r);
        acc += -log1p(-u) / rate;
        t[i] = acc;
    }
}

/* ---------------------------------------------------------- graphs (d = 2)
 *
 * Random geometric graph, the "rgg" class of the DIMACS graph instances the
 * paper's graph experiments use: n points uniform in the unit square (point
 * i draws its coordinates from its own stream), an edge {i, j} for every
 * pair closer than `radius`. Points are bucketed in a grid of cells no
 * smaller than the radius, so each point only looks at its 3 x 3 cell
 * neighbourhood. Edges are listed by their smaller endpoint i ascending,
 * then by the larger one, so the output does not depend on the thread
 * count. Pass 1 (pins == NULL) fills deg[i] = edges {i, j} with j > i and
 * returns their total; pass 2 writes the pairs at the prefix offsets. */
static void rgg_point(uint64_t seed, int64_t i, double *x, double *y)
{
    stream_t r = stream_for(seed, P_POINT, (uint64_t)i);
    *x = unit(&r);
    *y = unit(&r);
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

int64_t synth_rgg(int64_t n, double radius, uint64_t seed, int64_t *deg, int32_t *pins)
{
    if (n < 0 || n > 0x7FFFFFFF || !(radius > 0.0) || !deg) return -1;
    int64_t g = (int64_t)(1.0 / radius);
    if (g < 1) g = 1;
    if (g > 65536) g = 65536;
    const int64_t cells = g * g;
    double *px = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *py = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    int64_t *cstart = (int64_t *)calloc((size_t)cells + 1, sizeof(int64_t));
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    if (!px || !py || !cell || !cstart || !members) {
        free(px); free(py); free(cell); free(cstart); free(members);
        return -2;
    }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        rgg_point(seed, i, &px[i], &py[i]);
        int64_t cx = (int64_t)(px[i] * (double)g), cy = (int64_t)(py[i] * (double)g);
        if (cx >= g) cx = g - 1;
        if (cy >= g) cy = g - 1;
        cell[i] = cy * g + cx;
    }
    for (int64_t i = 0; i < n; ++i) cstart[cell[i] + 1]++;
    for (int64_t c = 0; c < cells; ++c) cstart[c + 1] += cstart[c];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)cells);
        if (!fill) {
            free(px); free(py); free(cell); free(cstart); free(members);
            return -2;
        }
        memcpy(fill, cstart, sizeof(int64_t) * (size_t)cells);
        for (int64_t i = 0; i < n; ++i) members[fill[cell[i]]++] = i; /* ascending i per cell */
        free(fill);
    }
    const double r2 = radius * radius;
    int64_t total = 0;
    int err = 0;
    #pragma omp parallel for schedule(dynamic, 4096) reduction(+ : total)
    for (int64_t i = 0; i < n; ++i) {
        const int64_t cx = cell[i] % g, cy = cell[i] / g;
        int64_t nb[64];
        int64_t k = 0;
        int64_t base = pins ? deg[i] : 0; /* pass 2: deg holds the offsets */
        for (int64_t dy = -1; dy <= 1; ++dy) {
            for (int64_t dx = -1; dx <= 1; ++dx) {
                const int64_t x = cx + dx, y = cy + dy;
                if (x < 0 || y < 0 || x >= g || y >= g) continue;
                const int64_t c = y * g + x;
                for (int64_t t = cstart[c]; t < cstart[c + 1]; ++t) {
                    const int64_t j = members[t];
                    if (j <= i) continue;
                    const double ddx = px[i] - px[j], ddy = py[i] - py[j];
                    if (ddx * ddx + ddy * ddy < r2) {
                        if (!pins) {
                            ++k;
                        } else if (k < 64) {
                            nb[k++] = j;
                        } else {
                            ++k; /* more than 64 larger neighbours: not expected at these radii */
                        }
                    }
                }
            }
        }
        if (!pins) {
            deg[i] = k;
            total += k;
        } else if (k > 64) {
            #pragma omp atomic write
            err = 1;
        } else {
            qsort(nb, (size_t)k, sizeof(int64_t), cmp_i64);
            for (int64_t q = 0; q < k; ++q) {
                pins[2 * (base + q)] = (int32_t)i;
                pins[2 * (base + q) + 1] = (int32_t)nb[q];
            }
            total += k;
        }
    }
    free(px); free(py); free(cell); free(cstart); free(members);
    return err ? -3 : total;
}

int synth_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
