/*
 * A multi-threaded CPU statement of the paper's local kernel (Sec. III-C):
 * C = A * B (plus-times, Eq. 1) row by row, the rows of A spread over the
 * host's cores (OpenMP, dynamic chunks of rows), each thread with a dense
 * sparse accumulator (SPA) of d floats, a stamp per column that tells
 * whether the current row has reached it, and the list of the columns the
 * row reached, sorted before the row is written.  Two passes: counts (the
 * row pointers of C), then values.  FP32 arithmetic, like the GPU path.
 *
 * This is a baseline for the benchmark to report beside the GPU numbers;
 * the library does not use it.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

static int cmp_i32(const void* a, const void* b) {
    const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static void sort_cols(int32_t* c, int64_t m) {
    if (m < 24) {  /* insertion sort for short rows */
        for (int64_t i = 1; i < m; ++i) {
            const int32_t v = c[i];
            int64_t j = i - 1;
            while (j >= 0 && c[j] > v) {
                c[j + 1] = c[j];
                --j;
            }
            c[j + 1] = v;
        }
    } else {
        qsort(c, (size_t)m, sizeof(int32_t), cmp_i32);
    }
}

/* Row counts of C into Cp[1..n] and their running sum (Cp[0] = 0); returns
 * nnz(C), or -1 if a column of A or B is out of range or memory runs out. */
int64_t cpu_plain_count(int64_t n, int32_t d, const int64_t* Ap, const int32_t* Ai, const int64_t* Bp,
                        const int32_t* Bi, int64_t* Cp, int32_t nthreads) {
    int bad = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads) reduction(| : bad)
    {
        int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(d > 0 ? d : 1));
        if (!stamp) {
            bad = 1;
        } else {
            for (int32_t c = 0; c < d; ++c) stamp[c] = -1;
#pragma omp for schedule(dynamic, 256)
            for (int64_t i = 0; i < n; ++i) {
                int64_t cnt = 0;
                for (int64_t e = Ap[i]; e < Ap[i + 1]; ++e) {
                    const int32_t k = Ai[e];
                    if (k < 0 || k >= n) {
                        bad = 1;
                        continue;
                    }
                    for (int64_t j = Bp[k]; j < Bp[k + 1]; ++j) {
                        const int32_t c = Bi[j];
                        if (c < 0 || c >= d) {
                            bad = 1;
                            continue;
                        }
                        if (stamp[c] != i) {
                            stamp[c] = i;
                            ++cnt;
                        }
                    }
                }
                Cp[i + 1] = cnt;
            }
            free(stamp);
        }
    }
    if (bad) return -1;
    Cp[0] = 0;
    for (int64_t i = 0; i < n; ++i) Cp[i + 1] += Cp[i];
    return Cp[n];
}

/* Columns and values of C for the row pointers of cpu_plain_count; returns
 * 0, or -1 on an input error or when memory runs out. */
int cpu_plain_numeric(int64_t n, int32_t d, const int64_t* Ap, const int32_t* Ai, const float* Ax,
                      const int64_t* Bp, const int32_t* Bi, const float* Bx, const int64_t* Cp, int32_t* Ci,
                      float* Cx, int32_t nthreads) {
    int bad = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads) reduction(| : bad)
    {
        const size_t dd = (size_t)(d > 0 ? d : 1);
        float* spa = (float*)malloc(sizeof(float) * dd);
        int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * dd);
        int32_t* list = (int32_t*)malloc(sizeof(int32_t) * dd);
        if (!spa || !stamp || !list) {
            bad = 1;
        } else {
            for (int32_t c = 0; c < d; ++c) stamp[c] = -1;
#pragma omp for schedule(dynamic, 256)
            for (int64_t i = 0; i < n; ++i) {
                int64_t m = 0;
                for (int64_t e = Ap[i]; e < Ap[i + 1]; ++e) {
                    const int32_t k = Ai[e];
                    if (k < 0 || k >= n) {
                        bad = 1;
                        continue;
                    }
                    const float a = Ax ? Ax[e] : 1.0f;
                    for (int64_t j = Bp[k]; j < Bp[k + 1]; ++j) {
                        const int32_t c = Bi[j];
                        if (c < 0 || c >= d) {
                            bad = 1;
                            continue;
                        }
                        const float t = a * (Bx ? Bx[j] : 1.0f);
                        if (stamp[c] != i) {
                            stamp[c] = i;
                            spa[c] = t;
                            list[m++] = c;
                        } else {
                            spa[c] += t;
                        }
                    }
                }
                if (m != Cp[i + 1] - Cp[i]) {
                    bad = 1;
                    continue;
                }
                sort_cols(list, m);
                for (int64_t q = 0; q < m; ++q) {
                    Ci[Cp[i] + q] = list[q];
                    Cx[Cp[i] + q] = spa[list[q]];
                }
            }
        }
        free(spa);
        free(stamp);
        free(list);
    }
    return bad ? -1 : 0;
}

int32_t cpu_plain_max_threads(void) { return (int32_t)omp_get_max_threads(); }
