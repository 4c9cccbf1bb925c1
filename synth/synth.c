/*
 * Seeded synthetic inputs for the TS-SpGEMM workloads: Erdos-Renyi and R-MAT
 * square matrices A (n x n), sparse tall-and-skinny matrices B (n x d) with a
 * fixed per-row density, and value arrays.  This file holds no arithmetic of
 * the product itself; it only draws inputs.  Both the CUDA path's tests and
 * the oracle's tests take their inputs from here.
 *
 * Randomness is counter based so that generation can run on many threads and
 * still give the same matrices for the same seed on any machine and any
 * thread count: draw(key, ctr) is the ctr-th output of a SplitMix64 sequence
 * started at `key` (Steele, Lea and Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014: state advances by the golden-ratio gamma,
 * the output is the 64-bit finaliser with shifts 30/27/31).
 *
 * Conventions (input recipe):
 *  - "s% sparse B" means each row of B holds (1 - s/100) * d entries; the
 *    fractional part is resolved per row by stochastic rounding, columns are
 *    distinct and uniform, stored ascending (paper Sec. V-A, Datasets).
 *  - Erdos-Renyi A with average degree k has exactly k distinct uniform
 *    columns per row (paper Table of datasets, ER row).
 *  - R-MAT: each edge descends `scale` levels choosing a quadrant with
 *    probabilities (a, b, c, 1-a-b-c); self-loops and duplicates are removed,
 *    vertices are relabelled by a seeded random permutation, and symmetrising
 *    is optional.  With n < 2^scale, edges with an endpoint >= n are redrawn.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ctr-th output of the SplitMix64 sequence whose initial state is key. */
static inline uint64_t draw(uint64_t key, uint64_t ctr) {
    return mix64(key + (ctr + 1) * GAMMA);
}

/* Independent key for sub-stream `s` of a seed. */
static inline uint64_t subkey(uint64_t seed, uint64_t s) {
    return draw(mix64(seed ^ 0x5851F42D4C957F2DULL), s);
}

/* Double in [0, 1) with 53 random bits. */
static inline double u01(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

/* Integer uniform in [0, m) by the multiply-shift reduction (Lemire 2019). */
static inline uint64_t below(uint64_t x, uint64_t m) {
    return (uint64_t)(((__uint128_t)x * (__uint128_t)m) >> 64);
}

enum { STREAM_COUNT = 1, STREAM_COLS = 2, STREAM_PERM = 3, STREAM_EDGE = 4 };

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static void insertion_sort_i32(int32_t* v, int64_t k) {
    for (int64_t i = 1; i < k; ++i) {
        int32_t x = v[i];
        int64_t j = i - 1;
        while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; --j; }
        v[j + 1] = x;
    }
}

/*
 * k distinct uniform integers from [0, m), ascending, written to out.
 * Dense requests (16k > m) use Knuth's selection sampling (TAOCP vol. 2,
 * Algorithm S), which emits in order; sparse requests redraw duplicates.
 * Draw counters are ctr_base + t for t = 0, 1, ...
 */
static void pick_distinct(uint64_t key, uint64_t ctr_base, int64_t k, int64_t m, int32_t* out) {
    if (k <= 0) return;
    if (k >= m) {
        for (int64_t j = 0; j < m; ++j) out[j] = (int32_t)j;
        return;
    }
    uint64_t t = 0;
    if (16 * k > m) {
        int64_t need = k;
        for (int64_t j = 0; j < m && need > 0; ++j) {
            double u = u01(draw(key, ctr_base + t++));
            if ((double)(m - j) * u < (double)need) { out[k - need] = (int32_t)j; --need; }
        }
        return;
    }
    int64_t got = 0;
    while (got < k) {
        int32_t c = (int32_t)below(draw(key, ctr_base + t++), (uint64_t)m);
        int dup = 0;
        for (int64_t q = 0; q < got; ++q) if (out[q] == c) { dup = 1; break; }
        if (!dup) out[got++] = c;
    }
    if (k <= 64) insertion_sort_i32(out, k);
    else qsort(out, (size_t)k, sizeof(int32_t), cmp_i32);
}

/* Row r's draws use counters r << 24 ... so rows never share a counter. */
#define ROW_CTR(r) ((uint64_t)(r) << 24)

/* Erdos-Renyi pattern: k distinct uniform columns per row; rowptr[i] = i*k. */
void synth_er(int64_t n, int64_t ncols, int64_t k, uint64_t seed, int64_t* rowptr, int32_t* col) {
    uint64_t key = subkey(seed, STREAM_COLS);
    if (k > ncols) k = ncols;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) pick_distinct(key, ROW_CTR(i), k, ncols, col + i * k);
    for (int64_t i = 0; i <= n; ++i) rowptr[i] = i * k;
}

/* Row counts of a tall-and-skinny B: floor(density*d) plus one with
 * probability frac(density*d); rowptr[n+1] is the running sum. */
void synth_ts_rowptr(int64_t n, int64_t d, double density, uint64_t seed, int64_t* rowptr) {
    uint64_t key = subkey(seed, STREAM_COUNT);
    double x = density * (double)d;
    if (x < 0) x = 0;
    if (x > (double)d) x = (double)d;
    int64_t base = (int64_t)floor(x);
    double frac = x - (double)base;
    rowptr[0] = 0;
    /* counts first (parallel), running sum after (serial, O(n)). */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = base + (u01(draw(key, (uint64_t)i)) < frac ? 1 : 0);
        if (c > d) c = d;
        rowptr[i + 1] = c;
    }
    for (int64_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
}

/* Columns of B for the counts in rowptr: distinct, uniform, ascending. */
void synth_ts_cols(int64_t n, int64_t d, uint64_t seed, const int64_t* rowptr, int32_t* col) {
    uint64_t key = subkey(seed, STREAM_COLS);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i)
        pick_distinct(key, ROW_CTR(i), rowptr[i + 1] - rowptr[i], d, col + rowptr[i]);
}

/* U[0,1) float32 values with 24 random bits, so every value is exact. */
void synth_uniform_f32(int64_t m, uint64_t seed, float* out) {
    uint64_t key = subkey(seed, 11);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) out[e] = (float)((double)(draw(key, (uint64_t)e) >> 40) * 0x1.0p-24);
}

/* N(0,1) float32 values by the Box-Muller transform (one output per pair). */
void synth_normal_f32(int64_t m, uint64_t seed, float* out) {
    uint64_t key = subkey(seed, 12);
    const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        double u1 = ((double)(draw(key, 2 * (uint64_t)e) >> 11) + 1.0) * 0x1.0p-53; /* (0,1] */
        double u2 = u01(draw(key, 2 * (uint64_t)e + 1));
        out[e] = (float)(sqrt(-2.0 * log(u1)) * cos(two_pi * u2));
    }
}

/* Seeded uniform permutation of [0, n) by Fisher-Yates (Durstenfeld). */
void synth_permutation(int64_t n, uint64_t seed, int32_t* perm) {
    uint64_t key = subkey(seed, STREAM_PERM);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)below(draw(key, (uint64_t)i), (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/* Distinct vertices with nonzero degree, chosen uniformly (Graph500 style
 * search keys).  Returns how many were found (< count when fewer exist). */
int64_t synth_sources(int64_t n, const int64_t* rowptr, int64_t count, uint64_t seed, int32_t* out) {
    uint64_t key = subkey(seed, 21);
    int64_t got = 0;
    uint64_t t = 0;
    int64_t nonempty = 0;
    for (int64_t v = 0; v < n; ++v) nonempty += rowptr[v + 1] > rowptr[v];
    if (count > nonempty) count = nonempty;
    while (got < count) {
        int32_t v = (int32_t)below(draw(key, t++), (uint64_t)n);
        if (rowptr[v + 1] == rowptr[v]) continue;
        int dup = 0;
        for (int64_t q = 0; q < got; ++q) if (out[q] == v) { dup = 1; break; }
        if (!dup) out[got++] = v;
    }
    return got;
}

/*
 * R-MAT edge list.  Edge e, attempt r descends `scale` levels; the quadrant
 * at each level is picked with probabilities a, b, c, 1-a-b-c.  An edge with
 * an endpoint >= n is redrawn (next attempt).  Endpoints are then relabelled
 * through perm (length n, may be NULL for identity).
 */
void synth_rmat_edges(int64_t scale, int64_t nedges, double a, double b, double c, int64_t n,
                      uint64_t seed, const int32_t* perm, int32_t* src, int32_t* dst) {
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
        for (uint64_t r = 0;; ++r) {
            uint64_t key = subkey(seed, STREAM_EDGE + 16 * r);
            uint64_t u = 0, v = 0;
            for (int64_t l = 0; l < scale; ++l) {
                double x = u01(draw(key, (uint64_t)e * 64 + (uint64_t)l));
                uint64_t bit = 1ULL << (scale - 1 - l);
                if (x < a) {
                } else if (x < ab) {
                    v |= bit;
                } else if (x < abc) {
                    u |= bit;
                } else {
                    u |= bit; v |= bit;
                }
            }
            if ((int64_t)u < n && (int64_t)v < n) {
                src[e] = perm ? perm[u] : (int32_t)u;
                dst[e] = perm ? perm[v] : (int32_t)v;
                break;
            }
        }
    }
}

/*
 * CSR pattern from an edge list: optionally add reversed edges, optionally
 * drop self-loops, sort each row and drop duplicate columns.  rowptr has n+1
 * entries; col must hold m (or 2m when symmetrising) entries; the number of
 * stored entries is returned.  The result does not depend on thread timing.
 */
int64_t synth_csr_from_edges(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                             int symmetrize, int drop_self, int64_t* rowptr, int32_t* col) {
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = src[e], v = dst[e];
        if (drop_self && u == v) continue;
#pragma omp atomic
        cnt[u + 1]++;
        if (symmetrize) {
#pragma omp atomic
            cnt[v + 1]++;
        }
    }
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    int64_t total = cnt[n];
    int32_t* tmp = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    int64_t* cur = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!tmp || !cur) { free(cnt); free(tmp); free(cur); return -1; }
    memcpy(cur, cnt, (size_t)n * sizeof(int64_t));
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = src[e], v = dst[e];
        if (drop_self && u == v) continue;
        int64_t p;
#pragma omp atomic capture
        p = cur[u]++;
        tmp[p] = v;
        if (symmetrize) {
#pragma omp atomic capture
            p = cur[v]++;
            tmp[p] = u;
        }
    }
    /* sort + unique per row; keep the unique count in cur[] */
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int32_t* r = tmp + cnt[i];
        int64_t len = cnt[i + 1] - cnt[i];
        if (len > 64) qsort(r, (size_t)len, sizeof(int32_t), cmp_i32);
        else insertion_sort_i32(r, len);
        int64_t u = 0;
        for (int64_t q = 0; q < len; ++q)
            if (u == 0 || r[q] != r[u - 1]) r[u++] = r[q];
        cur[i] = u;
    }
    rowptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) rowptr[i + 1] = rowptr[i] + cur[i];
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i)
        memcpy(col + rowptr[i], tmp + cnt[i], (size_t)cur[i] * sizeof(int32_t));
    int64_t nnz = rowptr[n];
    free(cnt); free(tmp); free(cur);
    return nnz;
}

int synth_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
