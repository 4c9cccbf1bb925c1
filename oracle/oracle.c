/*
 * ORACLE -- test infrastructure only.  A plain, slow, single-threaded CPU
 * statement of what the TS-SpGEMM hot path computes, used to check the CUDA
 * kernels.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it; the product path never calls into this file, and this
 * file shares no code with it.
 *
 * Matrices are CSR: row pointers int64[nrows+1], column indices int32
 * (ascending and distinct within a row), values double (the caller widens
 * float32 inputs exactly).  All accumulation is in double.
 *
 * Readings of the paper used here (where it is silent):
 *  - the output pattern is structural: (i,j) is stored iff at least one
 *    product A(i,k)*B(k,j) exists, even if the values cancel to zero;
 *  - columns of each output row are emitted in ascending order;
 *  - in the boolean (or, select2nd) semiring a stored entry of A means
 *    "true", so the product keeps B's truth value and the sum is OR;
 *  - BFS levels: sources are level 0, a vertex first entering the frontier
 *    of source s at iteration t gets level t, unreached is -1;
 *  - BFS parents with the (sel2nd, min) semiring (Sec. IV, the BFS-tree
 *    variant of Alg. 3): a frontier entry (u, s) carries the value u, the
 *    product of a stored A(v,u) with it selects that value and the sum is
 *    the minimum, so a newly reached (v, s) gets as parent the smallest
 *    neighbour u of v in the frontier of s; a source is its own parent,
 *    unreached is -1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

enum { SR_PLUS_TIMES = 0, SR_OR_SELECT2ND = 1 };

/*
 * Row counts of C = A*B (paper Sec. III-A, Eq. 1: row r of C is the sum over
 * the stored entries (r,c) of A of A(r,c) times row c of B; its pattern is the
 * union of the patterns of those rows of B).  rows selects which rows of A to
 * take (NULL: rows 0..nsel-1).  cnt[q] receives nnz of selected row q; the
 * total is returned, or -1 if memory runs out.
 */
int64_t oracle_spgemm_count(int64_t d, const int64_t* Ap, const int32_t* Ai, const int64_t* Bp,
                            const int32_t* Bi, const int64_t* rows, int64_t nsel, int64_t* cnt) {
    unsigned char* mark = (unsigned char*)calloc((size_t)(d > 0 ? d : 1), 1);
    int32_t* touched = (int32_t*)malloc((size_t)(d > 0 ? d : 1) * sizeof(int32_t));
    if (!mark || !touched) { free(mark); free(touched); return -1; }
    int64_t total = 0;
    for (int64_t q = 0; q < nsel; ++q) {
        int64_t r = rows ? rows[q] : q;
        int64_t nt = 0;
        for (int64_t e = Ap[r]; e < Ap[r + 1]; ++e) {
            int64_t c = Ai[e];
            for (int64_t f = Bp[c]; f < Bp[c + 1]; ++f) {
                int32_t j = Bi[f];
                if (!mark[j]) { mark[j] = 1; touched[nt++] = j; }
            }
        }
        for (int64_t t = 0; t < nt; ++t) mark[touched[t]] = 0;
        cnt[q] = nt;
        total += nt;
    }
    free(mark); free(touched);
    return total;
}

/*
 * C = A*B over the chosen semiring (paper Sec. II-A and Eq. 1), for the
 * selected rows.  Cp (nsel+1 entries) must hold the running sum of the
 * counts from oracle_spgemm_count.  For plus-times, Cx receives the double
 * sum and Cbound the sum of |A(i,k)|*|B(k,j)| per entry (the scale of the
 * rounding error any reordering of the sum can make).  For the boolean
 * semiring only Ci is written; Ax, Bx, Cx and Cbound may be NULL.
 * Returns 0, or -1 if memory runs out or the counts do not match.
 */
int oracle_spgemm(int64_t d, int semiring, const int64_t* Ap, const int32_t* Ai, const double* Ax,
                  const int64_t* Bp, const int32_t* Bi, const double* Bx, const int64_t* rows,
                  int64_t nsel, const int64_t* Cp, int32_t* Ci, double* Cx, double* Cbound) {
    size_t dd = (size_t)(d > 0 ? d : 1);
    unsigned char* mark = (unsigned char*)calloc(dd, 1);
    double* acc = (double*)calloc(dd, sizeof(double));
    double* bnd = (double*)calloc(dd, sizeof(double));
    if (!mark || !acc || !bnd) { free(mark); free(acc); free(bnd); return -1; }
    int status = 0;
    for (int64_t q = 0; q < nsel && status == 0; ++q) {
        int64_t r = rows ? rows[q] : q;
        for (int64_t e = Ap[r]; e < Ap[r + 1]; ++e) {
            int64_t c = Ai[e];
            for (int64_t f = Bp[c]; f < Bp[c + 1]; ++f) {
                int32_t j = Bi[f];
                mark[j] = 1;
                if (semiring == SR_PLUS_TIMES) {
                    acc[j] += Ax[e] * Bx[f];
                    bnd[j] += fabs(Ax[e]) * fabs(Bx[f]);
                }
            }
        }
        int64_t out = Cp[q];
        for (int64_t j = 0; j < d; ++j) {
            if (!mark[j]) continue;
            if (out >= Cp[q + 1]) { status = -1; break; }
            Ci[out] = (int32_t)j;
            if (semiring == SR_PLUS_TIMES) {
                Cx[out] = acc[j];
                Cbound[out] = bnd[j];
            }
            ++out;
            mark[j] = 0; acc[j] = 0.0; bnd[j] = 0.0;
        }
        if (status == 0 && out != Cp[q + 1]) status = -1;
    }
    free(mark); free(acc); free(bnd);
    return status;
}

/*
 * Multi-source BFS, paper Alg. 3, with the boolean TS-SpGEMM above as the
 * product.  A is the n x n adjacency pattern, src the d sources.  F (n x d)
 * starts with F(src[s], s) = 1 and S = F; while nnz(F) > 0: N = A*F over
 * (or, select2nd), F = N minus S, S = S or N.  levels (n*d, row-major by
 * vertex) gets the iteration at which each bit entered F, -1 if never.
 * frontier_nnz[t] (capacity maxlev) gets nnz(F) entering iteration t+1
 * (t = 0 is the initial frontier).  Returns the number of products computed,
 * or -1 on allocation failure / -2 if maxlev is too small.
 */
int64_t oracle_msbfs(int64_t n, const int64_t* Ap, const int32_t* Ai, int64_t d, const int32_t* src,
                     int32_t* levels, int64_t* frontier_nnz, int64_t maxlev) {
    unsigned char* S = (unsigned char*)calloc((size_t)(n * d > 0 ? n * d : 1), 1);
    int64_t* Fp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* Np = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* cnt = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    int32_t* Fi = NULL;
    int32_t* Ni = NULL;
    int64_t products = -1;
    if (!S || !Fp || !Np || !cnt) goto done;
    for (int64_t t = 0; t < n * d; ++t) levels[t] = -1;

    /* Init(f): column s of F holds the single vertex src[s]. */
    for (int64_t s = 0; s < d; ++s) Fp[src[s] + 1]++;
    for (int64_t v = 0; v < n; ++v) Fp[v + 1] += Fp[v];
    Fi = (int32_t*)malloc((size_t)(d > 0 ? d : 1) * sizeof(int32_t));
    if (!Fi) goto done;
    {
        int64_t* cur = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        if (!cur) goto done;
        memcpy(cur, Fp, (size_t)n * sizeof(int64_t));
        for (int64_t s = 0; s < d; ++s) Fi[cur[src[s]]++] = (int32_t)s;
        free(cur);
        /* columns ascending within a row: s was visited in increasing order */
    }
    for (int64_t s = 0; s < d; ++s) {
        S[(int64_t)src[s] * d + s] = 1;
        levels[(int64_t)src[s] * d + s] = 0;
    }
    products = 0;
    int64_t level = 0;
    if (maxlev < 1) { products = -2; goto done; }
    frontier_nnz[0] = Fp[n];
    while (Fp[n] > 0) {
        ++level;
        /* N = A * F over (or, select2nd) */
        int64_t tot = oracle_spgemm_count(d, Ap, Ai, Fp, Fi, NULL, n, cnt);
        if (tot < 0) { products = -1; goto done; }
        Np[0] = 0;
        for (int64_t v = 0; v < n; ++v) Np[v + 1] = Np[v] + cnt[v];
        free(Ni);
        Ni = (int32_t*)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int32_t));
        if (!Ni) { products = -1; goto done; }
        if (oracle_spgemm(d, SR_OR_SELECT2ND, Ap, Ai, NULL, Fp, Fi, NULL, NULL, n, Np, Ni, NULL, NULL)) {
            products = -1; goto done;
        }
        ++products;
        /* F = N \ S, then S = S | N (in place over the rows of N) */
        int64_t out = 0;
        free(Fi);
        Fi = (int32_t*)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int32_t));
        if (!Fi) { products = -1; goto done; }
        Fp[0] = 0;
        for (int64_t v = 0; v < n; ++v) {
            for (int64_t e = Np[v]; e < Np[v + 1]; ++e) {
                int64_t s = Ni[e];
                if (!S[v * d + s]) {
                    Fi[out++] = (int32_t)s;
                    levels[v * d + s] = (int32_t)level;
                }
            }
            Fp[v + 1] = out;
        }
        for (int64_t v = 0; v < n; ++v)
            for (int64_t e = Np[v]; e < Np[v + 1]; ++e) S[v * d + Ni[e]] = 1;
        if (level >= maxlev) { products = -2; goto done; }
        frontier_nnz[level] = Fp[n];
    }
done:
    free(S); free(Fp); free(Np); free(cnt); free(Fi); free(Ni);
    return products;
}

/*
 * Alg. 3 with the (sel2nd, min) semiring: the frontier F holds, for each
 * (u, s) in it, the value u; N(v, s) = min over the stored A(v, u) with
 * (u, s) in F of F(u, s); the new frontier is N minus S with each entry's
 * value reset to its own row index, and the value N(v, s) of a new entry is
 * v's parent in the BFS tree of source s.  Dense n x d arrays (small inputs
 * only).  Returns the number of products (iterations) or < 0 on failure.
 */
int64_t oracle_msbfs_parents(int64_t n, const int64_t* Ap, const int32_t* Ai, int64_t d, const int32_t* src,
                             int32_t* levels, int32_t* parents, int64_t* frontier_nnz, int64_t maxlev) {
    const int64_t nd = n * d > 0 ? n * d : 1;
    int32_t* F = (int32_t*)malloc((size_t)nd * sizeof(int32_t)); /* frontier values, -1 = absent */
    int32_t* N = (int32_t*)malloc((size_t)nd * sizeof(int32_t));
    unsigned char* S = (unsigned char*)calloc((size_t)nd, 1);
    int64_t products = -1;
    if (!F || !N || !S) goto done;
    for (int64_t t = 0; t < n * d; ++t) {
        levels[t] = -1;
        parents[t] = -1;
        F[t] = -1;
    }
    for (int64_t s = 0; s < d; ++s) {
        const int64_t v = src[s];
        F[v * d + s] = (int32_t)v;
        S[v * d + s] = 1;
        levels[v * d + s] = 0;
        parents[v * d + s] = (int32_t)v;
    }
    if (maxlev < 1) { products = -2; goto done; }
    int64_t fn = 0;
    for (int64_t t = 0; t < n * d; ++t) fn += F[t] >= 0;
    frontier_nnz[0] = fn;
    products = 0;
    int64_t level = 0;
    while (fn > 0) {
        ++level;
        /* N = A (sel2nd, min) F */
        for (int64_t t = 0; t < n * d; ++t) N[t] = -1;
        for (int64_t v = 0; v < n; ++v)
            for (int64_t e = Ap[v]; e < Ap[v + 1]; ++e) {
                const int64_t u = Ai[e];
                for (int64_t s = 0; s < d; ++s) {
                    const int32_t f = F[u * d + s];
                    if (f < 0) continue;                 /* no stored frontier entry */
                    int32_t* x = &N[v * d + s];
                    if (*x < 0 || f < *x) *x = f;       /* sel2nd, then min */
                }
            }
        ++products;
        /* F = N \ S with values reset to the row index; parents and levels
         * of the new entries; S = S | N */
        fn = 0;
        for (int64_t v = 0; v < n; ++v)
            for (int64_t s = 0; s < d; ++s) {
                const int64_t t = v * d + s;
                F[t] = -1;
                if (N[t] >= 0 && !S[t]) {
                    F[t] = (int32_t)v;
                    parents[t] = N[t];
                    levels[t] = (int32_t)level;
                    ++fn;
                }
                if (N[t] >= 0) S[t] = 1;
            }
        if (level >= maxlev) { products = -2; goto done; }
        frontier_nnz[level] = fn;
    }
done:
    free(F); free(N); free(S);
    return products;
}

/*
 * Gradients of L = sum over C's pattern of dC(i,j) * C(i,j) for C = A*B in
 * plus-times, with the patterns of A and B fixed:
 *   dA(i,k) = sum over j in row k of B of dC(i,j) * B(k,j)      for (i,k) in A
 *   dB(k,j) = sum over i with A(i,k) stored of A(i,k) * dC(i,j) for (k,j) in B
 * (dC is zero off C's pattern; C's pattern contains every (i,j) with a
 * product, so every lookup below finds its entry.)  A has n rows (it may be
 * a block of rows of a larger matrix), B has nB rows.  Rows of A are visited in
 * order; dB is summed by scattering each term to its entry.  dA_bound and
 * dB_bound receive the matching sums of absolute terms.  dA, dB and the bounds may each be NULL.
 * Returns 0, or -1 on allocation failure.
 */
int oracle_backward(int64_t n, int64_t d, const int64_t* Ap, const int32_t* Ai, const double* Ax,
                    int64_t nB, const int64_t* Bp, const int32_t* Bi, const double* Bx, const int64_t* Cp,
                    const int32_t* Ci, const double* dC, double* dA, double* dA_bound, double* dB,
                    double* dB_bound) {
    double* g = (double*)calloc((size_t)(d > 0 ? d : 1), sizeof(double));
    if (!g) return -1;
    if (dB) memset(dB, 0, (size_t)Bp[nB] * sizeof(double));
    if (dB_bound) memset(dB_bound, 0, (size_t)Bp[nB] * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = Cp[i]; e < Cp[i + 1]; ++e) g[Ci[e]] = dC[e];
        for (int64_t e = Ap[i]; e < Ap[i + 1]; ++e) {
            int64_t k = Ai[e];
            double s = 0.0, sb = 0.0;
            for (int64_t f = Bp[k]; f < Bp[k + 1]; ++f) {
                double gj = g[Bi[f]];
                s += gj * Bx[f];
                sb += fabs(gj) * fabs(Bx[f]);
                if (dB) dB[f] += Ax[e] * gj;
                if (dB_bound) dB_bound[f] += fabs(Ax[e]) * fabs(gj);
            }
            if (dA) dA[e] = s;
            if (dA_bound) dA_bound[e] = sb;
        }
        for (int64_t e = Cp[i]; e < Cp[i + 1]; ++e) g[Ci[e]] = 0.0;
    }
    free(g);
    return 0;
}

/* Position of column j in row i of C (binary search), -1 if absent. */
static int64_t find_in_row(const int64_t* Cp, const int32_t* Ci, int64_t i, int32_t j) {
    int64_t lo = Cp[i], hi = Cp[i + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (Ci[mid] < j) lo = mid + 1; else hi = mid;
    }
    return (lo < Cp[i + 1] && Ci[lo] == j) ? lo : -1;
}

/*
 * The dA formula above for selected rows of A only (a sample of a large
 * product): dA_out holds the entries of the selected rows, row after row.
 */
int oracle_backward_dA_rows(int64_t d, const int64_t* Ap, const int32_t* Ai, const int64_t* Bp,
                            const int32_t* Bi, const double* Bx, const int64_t* Cp, const int32_t* Ci,
                            const double* dC, const int64_t* rows, int64_t nsel, double* dA_out,
                            double* bound_out) {
    double* g = (double*)calloc((size_t)(d > 0 ? d : 1), sizeof(double));
    if (!g) return -1;
    int64_t out = 0;
    for (int64_t q = 0; q < nsel; ++q) {
        int64_t i = rows[q];
        for (int64_t e = Cp[i]; e < Cp[i + 1]; ++e) g[Ci[e]] = dC[e];
        for (int64_t e = Ap[i]; e < Ap[i + 1]; ++e) {
            int64_t k = Ai[e];
            double s = 0.0, sb = 0.0;
            for (int64_t f = Bp[k]; f < Bp[k + 1]; ++f) {
                s += g[Bi[f]] * Bx[f];
                sb += fabs(g[Bi[f]]) * fabs(Bx[f]);
            }
            dA_out[out] = s;
            bound_out[out] = sb;
            ++out;
        }
        for (int64_t e = Cp[i]; e < Cp[i + 1]; ++e) g[Ci[e]] = 0.0;
    }
    free(g);
    return 0;
}

/*
 * The dB formula above for selected rows k of B only: one pass over A finds
 * every stored (i,k) with k selected; dC(i,j) is looked up in row i of C.
 * dB_out holds the entries of the selected rows of B, row after row.
 * Returns 0, -1 on allocation failure, -2 if a lookup fails (C's pattern
 * does not contain the product's pattern).
 */
int oracle_backward_dB_rows(int64_t n, const int64_t* Ap, const int32_t* Ai, const double* Ax,
                            const int64_t* Bp, const int32_t* Bi, const int64_t* Cp, const int32_t* Ci,
                            const double* dC, const int64_t* krows, int64_t nsel, double* dB_out,
                            double* bound_out) {
    int64_t* slot = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t* base = (int64_t*)malloc((size_t)(nsel + 1) * sizeof(int64_t));
    if (!slot || !base) { free(slot); free(base); return -1; }
    for (int64_t v = 0; v < n; ++v) slot[v] = -1;
    base[0] = 0;
    for (int64_t q = 0; q < nsel; ++q) {
        slot[krows[q]] = q;
        base[q + 1] = base[q] + (Bp[krows[q] + 1] - Bp[krows[q]]);
    }
    memset(dB_out, 0, (size_t)base[nsel] * sizeof(double));
    memset(bound_out, 0, (size_t)base[nsel] * sizeof(double));
    int status = 0;
    for (int64_t i = 0; i < n && status == 0; ++i) {
        for (int64_t e = Ap[i]; e < Ap[i + 1]; ++e) {
            int64_t k = Ai[e];
            int64_t q = slot[k];
            if (q < 0) continue;
            for (int64_t f = Bp[k]; f < Bp[k + 1]; ++f) {
                int64_t pos = find_in_row(Cp, Ci, i, Bi[f]);
                if (pos < 0) { status = -2; break; }
                dB_out[base[q] + (f - Bp[k])] += Ax[e] * dC[pos];
                bound_out[base[q] + (f - Bp[k])] += fabs(Ax[e]) * fabs(dC[pos]);
            }
        }
    }
    free(slot); free(base);
    return status;
}

/*
 * Textbook single-source BFS with a FIFO queue (the definition of BFS level
 * = hop distance along stored edges (v -> A.col) of A): levels[v] = distance
 * from src, -1 if unreachable.  For a symmetric A this equals column s of the
 * level matrix of Alg. 3.  Returns the largest level, -1 on allocation failure.
 */
int64_t oracle_bfs_levels(int64_t n, const int64_t* Ap, const int32_t* Ai, int32_t src, int32_t* levels) {
    int32_t* queue = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!queue) return -1;
    for (int64_t v = 0; v < n; ++v) levels[v] = -1;
    int64_t head = 0, tail = 0, maxlev = 0;
    levels[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = Ap[u]; e < Ap[u + 1]; ++e) {
            int32_t v = Ai[e];
            if (levels[v] < 0) {
                levels[v] = levels[u] + 1;
                if (levels[v] > maxlev) maxlev = levels[v];
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return maxlev;
}

/*
 * Sparse Force2Vec step (paper Sec. IV, "Distributed sparse embedding"), for
 * the minibatch of rows [r0, r0 + b) of the embedding Z (n x d, exactly k
 * stored entries per row, Zp[i] = k*i).  Readings (the paper names the
 * parts, not the formulas): row i's neighbours in A carry +1 and its s
 * negative samples neg[(i-r0)*s + t] carry -1 (each occurrence one term);
 * x_ij = z_i . z_j; an attractive term weighs z_j by (1 - sigmoid(x_ij)), a
 * repulsive one by -sigmoid(x_ij) (the gradient of the usual
 * negative-sampling objective with respect to z_i); G_i = sum of the
 * weighted z_j (the TS-SpGEMM W * Z); U_i = z_i + lr * G_i; the new row keeps
 * the k entries of U_i of largest magnitude (ties: smaller column first).
 * All rows of the batch use the old Z (synchronous SGD).
 *
 * Outputs: U[b*d] (dense, double), Ub[b*d] (per entry: |z_i(c)| +
 * lr * sum over terms of (|w| + S_ij/4 + 1) * |z_j(c)| with S_ij = sum of
 * |z_i||z_j| over shared columns -- the sum of the magnitudes that U(c)
 * adds up, with the weights' sensitivity to their dot products (the
 * sigmoid's slope is at most 1/4) and to their own rounding (the 1)),
 * and the sparsified rows Ncol[b*k] (ascending) / Nval[b*k].
 * Returns 0 or -1 on allocation failure.
 */
static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

int oracle_f2v_topk(int64_t rows, int64_t d, int64_t k, const double* U, int32_t* Ncol, double* Nval) {
    /* the k columns of largest |U|, ties to the smaller column; emitted ascending */
    unsigned char* keep = (unsigned char*)malloc((size_t)(d > 0 ? d : 1));
    if (!keep) return -1;
    for (int64_t r = 0; r < rows; ++r) {
        const double* u = U + r * d;
        for (int64_t c = 0; c < d; ++c) {
            int64_t rank = 0; /* entries ranked before c */
            for (int64_t e = 0; e < d; ++e) {
                const double a = fabs(u[e]), x = fabs(u[c]);
                if (a > x || (a == x && e < c)) ++rank;
            }
            keep[c] = rank < k;
        }
        int64_t o = 0;
        for (int64_t c = 0; c < d; ++c)
            if (keep[c]) {
                Ncol[r * k + o] = (int32_t)c;
                Nval[r * k + o] = u[c];
                ++o;
            }
    }
    free(keep);
    return 0;
}

int oracle_f2v_step(int64_t n, const int64_t* Ap, const int32_t* Ai, int64_t d, int64_t k, const int32_t* Zcol,
                    const double* Zval, int64_t r0, int64_t b, const int32_t* neg, int64_t s, double lr,
                    double* U, double* Ub, int32_t* Ncol, double* Nval) {
    double* zi = (double*)calloc((size_t)(d > 0 ? d : 1), sizeof(double));
    if (!zi) return -1;
    for (int64_t r = 0; r < b; ++r) {
        const int64_t i = r0 + r;
        for (int64_t c = 0; c < d; ++c) zi[c] = 0.0;
        for (int64_t t = 0; t < k; ++t) zi[Zcol[i * k + t]] = Zval[i * k + t];
        double* u = U + r * d;
        double* ub = Ub + r * d;
        for (int64_t c = 0; c < d; ++c) {
            u[c] = zi[c];
            ub[c] = fabs(zi[c]);
        }
        const int64_t nA = Ap[i + 1] - Ap[i];
        for (int64_t t = 0; t < nA + s; ++t) {
            const int attract = t < nA;
            const int64_t j = attract ? Ai[Ap[i] + t] : neg[r * s + (t - nA)];
            double x = 0.0, S = 0.0;
            for (int64_t q = 0; q < k; ++q) {
                const int32_t c = Zcol[j * k + q];
                x += zi[c] * Zval[j * k + q];
                S += fabs(zi[c] * Zval[j * k + q]);
            }
            const double w = attract ? 1.0 - sigmoid(x) : -sigmoid(x);
            for (int64_t q = 0; q < k; ++q) {
                const int32_t c = Zcol[j * k + q];
                u[c] += lr * w * Zval[j * k + q];
                ub[c] += lr * (fabs(w) + S / 4.0 + 1.0) * fabs(Zval[j * k + q]);
            }
        }
    }
    free(zi);
    return oracle_f2v_topk(b, d, k, U, Ncol, Nval);
}
