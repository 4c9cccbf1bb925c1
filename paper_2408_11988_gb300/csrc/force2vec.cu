// Sparse Force2Vec minibatch step around the TS-SpGEMM (paper Sec. IV,
// "Distributed sparse embedding"), for the rows [r0, r0 + b) of a sparse
// embedding Z (n x d, exactly k stored entries per row, row i at [k*i, k*i+k)):
//
//   1. W's pattern: row r of the batch merges the neighbours of vertex r0 + r
//      in A (weight class +1) with its s negative samples (class -1); a column
//      met several times keeps its counts of both classes (k_f2v_newmask,
//      k_f2v_rowlen, k_f2v_fill_a, k_f2v_fill_n: a thread per sample or per
//      entry, so that hub rows add no tail);
//   2. weights (a sampled product on W's pattern): x = z_i . z_j by a merge
//      of the two rows of Z, w = npos * (1 - sigmoid(x)) - nneg * sigmoid(x)
//      (k_f2v_weights, a thread per entry of W);
//   3. G = W * Z, the plus-times TS-SpGEMM of this library (symbolic and
//      numeric passes, run by the C ABI layer);
//   4. U = Z_batch + lr * G, then the k entries of each row of U of largest
//      magnitude (ties: smaller column) in ascending column order, by a
//      radix select on the magnitude's bit pattern (k_f2v_update);
//   5. the new rows replace the batch rows of Z (k_f2v_commit), after every
//      row of the batch was computed from the old Z (synchronous SGD).
#include "common.cuh"
#include "kernels.h"

namespace ts {

constexpr int F2V_MAX_NEG = 32;

// Entry-parallel construction of W's pattern (no thread walks a whole row,
// so hub rows add no tail).  A negative sample of row r is "new" when it is
// the first occurrence of its vertex among the row's samples and not a
// neighbour; W's row r is A's row with the new negatives inserted in column
// order, each column carrying its count of neighbour (0/1) and negative
// occurrences.

// First position in the ascending A(i, :) whose column is >= c.
__device__ __forceinline__ long long f2v_lower(const int* __restrict__ Ai, long long a0, long long a1, int c) {
    long long lo = a0, hi = a1;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (__ldg(Ai + mid) < c) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Thread per (row, sample): the row's mask of new samples.
__global__ void __launch_bounds__(256) k_f2v_newmask(const long long* __restrict__ Ap, const int* __restrict__ Ai,
                                                     long long nnzA, int n, long long r0, long long b,
                                                     const int* __restrict__ neg, int s, unsigned* newmask,
                                                     unsigned long long* err) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= b * s) return;
    const long long r = q / s;
    const int t = (int)(q - r * s);
    const int v = __ldg(neg + q);
    if ((unsigned)v >= (unsigned)n) {
        atomicOr(err, ERR_A_COL);
        return;
    }
    for (int u = 0; u < t; ++u)
        if (__ldg(neg + r * s + u) == v) return;  // not the first occurrence
    const long long i = r0 + r;
    const long long a0 = clampll(__ldg(Ap + i), 0, nnzA), a1 = clampll(__ldg(Ap + i + 1), a0, nnzA);
    const long long p = f2v_lower(Ai, a0, a1, v);
    if (p < a1 && __ldg(Ai + p) == v) return;  // a neighbour
    atomicOr(newmask + r, 1u << t);
}

// Thread per row: W's row length (into Wp + 1, scanned afterwards).
__global__ void __launch_bounds__(256) k_f2v_rowlen(const long long* __restrict__ Ap, long long nnzA, long long r0,
                                                    long long b, const unsigned* __restrict__ newmask, long long* cnt) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= b) return;
    const long long a0 = clampll(__ldg(Ap + r0 + r), 0, nnzA), a1 = clampll(__ldg(Ap + r0 + r + 1), a0, nnzA);
    cnt[r] = (a1 - a0) + __popc(newmask[r]);
}

// Among row r's samples: how many new ones have a column below c, and how
// many samples (all occurrences) equal c.
__device__ __forceinline__ void f2v_negstats(const int* __restrict__ neg, long long r, int s, unsigned mask, int c,
                                             int& below, int& eq) {
    below = 0;
    eq = 0;
    for (int t = 0; t < s; ++t) {
        const int v = __ldg(neg + r * s + t);
        below += ((mask >> t) & 1u) && v < c;
        eq += v == c;
    }
}

// Thread per entry of A in the batch rows: its place in W.
__global__ void __launch_bounds__(256) k_f2v_fill_a(const long long* __restrict__ Ap, const int* __restrict__ Ai,
                                                    long long nnzA, long long r0, long long b,
                                                    const int* __restrict__ neg, int s,
                                                    const unsigned* __restrict__ newmask, const long long* Wp,
                                                    int* Wcol, int* Wmult, int* Wrow) {
    const long long base = clampll(__ldg(Ap + r0), 0, nnzA), top = clampll(__ldg(Ap + r0 + b), base, nnzA);
    for (long long e = base + (long long)blockIdx.x * blockDim.x + threadIdx.x; e < top;
         e += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = b;  // row: the last r with Ap[r0 + r] <= e
        while (hi - lo > 1) {
            const long long mid = (lo + hi) >> 1;
            if (__ldg(Ap + r0 + mid) <= e) lo = mid;
            else hi = mid;
        }
        const long long r = lo;
        const int c = __ldg(Ai + e);
        int below, eq;
        f2v_negstats(neg, r, s, newmask[r], c, below, eq);
        const long long pos = Wp[r] + (e - __ldg(Ap + r0 + r)) + below;
        if (pos < Wp[r + 1]) {
            Wcol[pos] = c;
            Wmult[pos] = 1 | (eq << 16);
            Wrow[pos] = (int)r;
        }
    }
}

// Thread per (row, new sample): its place in W.
__global__ void __launch_bounds__(256) k_f2v_fill_n(const long long* __restrict__ Ap, const int* __restrict__ Ai,
                                                    long long nnzA, long long r0, long long b,
                                                    const int* __restrict__ neg, int s,
                                                    const unsigned* __restrict__ newmask, const long long* Wp,
                                                    int* Wcol, int* Wmult, int* Wrow) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= b * s) return;
    const long long r = q / s;
    const int t = (int)(q - r * s);
    const unsigned mask = newmask[r];
    if (!((mask >> t) & 1u)) return;
    const int c = __ldg(neg + q);
    const long long i = r0 + r;
    const long long a0 = clampll(__ldg(Ap + i), 0, nnzA), a1 = clampll(__ldg(Ap + i + 1), a0, nnzA);
    int below, eq;
    f2v_negstats(neg, r, s, mask, c, below, eq);
    const long long pos = Wp[r] + (f2v_lower(Ai, a0, a1, c) - a0) + below;
    if (pos < Wp[r + 1]) {
        Wcol[pos] = c;
        Wmult[pos] = eq << 16;
        Wrow[pos] = (int)r;
    }
}

// Z must hold exactly k entries per row: Zp[i] = k * i (else ERR_CAPACITY).
__global__ void __launch_bounds__(256) k_f2v_check_rows(const long long* __restrict__ Zp, long long n, int k,
                                                        unsigned long long* err) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n && __ldg(Zp + i) != (long long)k * i) atomicOr(err, ERR_CAPACITY);
}

// Row i of Z scattered into the dense shared row g (or cleared again).
__device__ __forceinline__ void f2v_scatter(const int* __restrict__ Zc, const float* __restrict__ Zv, long long i,
                                            int k, int d, float* g, bool clear) {
    for (int t = lane_id(); t < k; t += 32) {
        const int c = __ldg(Zc + i * k + t);
        if ((unsigned)c < (unsigned)d) g[c] = clear ? 0.0f : __ldg(Zv + i * k + t);
    }
}

// Thread per entry of W: x = z_i . z_j by a merge of the two ascending rows
// of Z, then the entry's weight.
__global__ void __launch_bounds__(256) k_f2v_weights(const int* __restrict__ Zc, const float* __restrict__ Zv,
                                                     long long n, int k, long long r0, const long long* __restrict__ Wp,
                                                     long long b, const int* __restrict__ Wcol,
                                                     const int* __restrict__ Wmult, const int* __restrict__ Wrow,
                                                     float* Wval) {
    const long long nW = Wp[b];
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nW;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = r0 + __ldg(Wrow + e), j = __ldg(Wcol + e);
        if ((unsigned long long)j >= (unsigned long long)n || (unsigned long long)i >= (unsigned long long)n) {
            Wval[e] = 0.0f;  // a bad column of A: flagged by the product pass
            continue;
        }
        const int* ci = Zc + i * k;
        const int* cj = Zc + j * k;
        float x = 0.0f;
        int p = 0, q = 0;
        int a = __ldg(ci), c = __ldg(cj);
        while (p < k && q < k) {
            if (a == c) x += __ldg(Zv + i * k + p) * __ldg(Zv + j * k + q);
            const bool adv_p = a <= c, adv_q = c <= a;
            if (adv_p && ++p < k) a = __ldg(ci + p);
            if (adv_q && ++q < k) c = __ldg(cj + q);
        }
        const int m = __ldg(Wmult + e);
        const float sg = 1.0f / (1.0f + expf(-x));
        Wval[e] = (float)(m & 0xFFFF) * (1.0f - sg) - (float)(m >> 16) * sg;
    }
}

// U = Z_batch + lr * G per row (dense in shared memory), optional dense copy
// to U_out, then the k entries of largest magnitude into the staging rows.
__global__ void __launch_bounds__(256) k_f2v_update(const int* __restrict__ Zc, const float* __restrict__ Zv,
                                                    int d, int k, long long r0, long long b,
                                                    const long long* __restrict__ Gp, const int* __restrict__ Gc,
                                                    const float* __restrict__ Gv, float lr, float* U_out,
                                                    int* Sc, float* Sv, unsigned long long* err) {
    extern __shared__ __align__(16) float fsm[];
    const int nw = blockDim.x >> 5, warp = warp_id(), lane = lane_id();
    const int dpad = (d + 31) & ~31;
    const int mb = dpad >> 5;
    const unsigned lt = lanemask_lt();
    float* u = fsm + (size_t)warp * dpad;
    for (int c = lane; c < dpad; c += 32) u[c] = 0.0f;
    __syncwarp();
    for (long long r = (long long)blockIdx.x * nw + warp; r < b; r += (long long)gridDim.x * nw) {
        const long long i = r0 + r;
        f2v_scatter(Zc, Zv, i, k, d, u, false);
        __syncwarp();
        for (long long e = Gp[r] + lane; e < Gp[r + 1]; e += 32) {
            const int c = __ldg(Gc + e);
            if ((unsigned)c < (unsigned)d) u[c] += lr * __ldg(Gv + e);  // G's columns are distinct
            else atomicOr(err, ERR_C_ROW);
        }
        __syncwarp();
        if (U_out)
            for (int c = lane; c < d; c += 32) U_out[r * d + c] = u[c];
        // T = the k-th largest magnitude key (bits of |u|; monotone in |u|)
        unsigned T = 0u;
        for (int bit = 31; bit >= 0; --bit) {
            const unsigned cand = T | (1u << bit);
            int cnt = 0;
            for (int m = 0; m < mb; ++m) {
                const int c = 32 * m + lane;
                cnt += (c < d && (__float_as_uint(u[c]) & 0x7FFFFFFFu) >= cand) ? 1 : 0;
            }
            if (warp_sum(cnt) >= k) T = cand;
        }
        int gt = 0;
        for (int m = 0; m < mb; ++m) {
            const int c = 32 * m + lane;
            gt += (c < d && (__float_as_uint(u[c]) & 0x7FFFFFFFu) > T) ? 1 : 0;
        }
        const int need = k - warp_sum(gt);  // keys equal to T to keep, smallest columns first
        int eq_before = 0, out = 0;
        for (int m = 0; m < mb; ++m) {
            const int c = 32 * m + lane;
            const float v = c < d ? u[c] : 0.0f;
            const unsigned key = __float_as_uint(v) & 0x7FFFFFFFu;
            const bool valid = c < d;
            const bool eq = valid && key == T;
            const unsigned beq = __ballot_sync(FULL, eq);
            const bool keep = (valid && key > T) || (eq && eq_before + __popc(beq & lt) < need);
            const unsigned bk = __ballot_sync(FULL, keep);
            if (keep) {
                const int pos = out + __popc(bk & lt);
                if (pos < k) {
                    Sc[r * k + pos] = c;
                    Sv[r * k + pos] = v;
                }
            }
            eq_before += __popc(beq);
            out += __popc(bk);
        }
        __syncwarp();
        for (int c = lane; c < dpad; c += 32) u[c] = 0.0f;
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256) k_f2v_commit(long long r0, long long b, int k, const int* __restrict__ Sc,
                                                    const float* __restrict__ Sv, int* Zc, float* Zv) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < b * k;
         t += (long long)gridDim.x * blockDim.x) {
        Zc[r0 * k + t] = Sc[t];
        Zv[r0 * k + t] = Sv[t];
    }
}

static unsigned f2v_blocks_exact(long long m) { return (unsigned)((m + 255) / 256 > 0 ? (m + 255) / 256 : 1); }

static unsigned f2v_blocks(long long m) {
    long long g = (m + 255) / 256;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)g;
}

cudaError_t launch_f2v_pattern(const DevCsr& A, long long r0, long long b, const int* neg, int s, long long* Wp,
                               unsigned* newmask, long long* partial, WsHeader* hdr, cudaStream_t st) {
    cudaError_t e;
    if (s < 0 || s > F2V_MAX_NEG) return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(Wp, 0, sizeof(long long), st))) return e;
    if (b == 0) return cudaSuccess;
    if ((e = cudaMemsetAsync(newmask, 0, sizeof(unsigned) * (size_t)b, st))) return e;
    if (s > 0) {
        count_launch();
        k_f2v_newmask<<<f2v_blocks_exact(b * s), 256, 0, st>>>(A.rowptr, A.col, A.nnz, (int)A.nrows, r0, b, neg, s,
                                                               newmask, &hdr->err);
    }
    count_launch();
    k_f2v_rowlen<<<f2v_blocks_exact(b), 256, 0, st>>>(A.rowptr, A.nnz, r0, b, newmask, Wp + 1);
    if ((e = cudaGetLastError())) return e;
    return launch_scan_inplace(Wp + 1, b, partial, st);
}

cudaError_t launch_f2v_fill(const DevCsr& A, long long r0, long long b, const int* neg, int s, const long long* Wp,
                            const unsigned* newmask, int* Wcol, int* Wmult, int* Wrow, cudaStream_t st) {
    if (b == 0) return cudaSuccess;
    count_launch();
    k_f2v_fill_a<<<152 * 8, 256, 0, st>>>(A.rowptr, A.col, A.nnz, r0, b, neg, s, newmask, Wp, Wcol, Wmult, Wrow);
    if (s > 0) {
        count_launch();
        k_f2v_fill_n<<<f2v_blocks_exact(b * s), 256, 0, st>>>(A.rowptr, A.col, A.nnz, r0, b, neg, s, newmask, Wp,
                                                              Wcol, Wmult, Wrow);
    }
    return cudaGetLastError();
}

cudaError_t launch_f2v_check(const DevCsr& Z, int k, WsHeader* hdr, cudaStream_t st) {
    count_launch();
    k_f2v_check_rows<<<(unsigned)((Z.nrows + 1 + 255) / 256), 256, 0, st>>>(Z.rowptr, Z.nrows, k, &hdr->err);
    return cudaGetLastError();
}

cudaError_t launch_f2v_weights(const DevCsr& Z, int k, long long r0, long long b, const long long* Wp,
                               const int* Wcol, const int* Wmult, const int* Wrow, float* Wval, cudaStream_t st) {
    if (b == 0) return cudaSuccess;
    count_launch();
    k_f2v_weights<<<152 * 16, 256, 0, st>>>(Z.col, Z.val, Z.nrows, k, r0, Wp, b, Wcol, Wmult, Wrow, Wval);
    return cudaGetLastError();
}

cudaError_t launch_f2v_update(const DevCsr& Z, int k, long long r0, long long b, const long long* Gp, const int* Gc,
                              const float* Gv, float lr, float* U_out, int* Sc, float* Sv, int sms, WsHeader* hdr,
                              cudaStream_t st) {
    if (b == 0) return cudaSuccess;
    const int d = (int)Z.ncols, dpad = (d + 31) & ~31;
    const size_t smem = sizeof(float) * (size_t)dpad * 8;
    cudaError_t e;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute((const void*)k_f2v_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
        return e;
    const int grid = persistent_grid((const void*)k_f2v_update, 256, smem, sms);
    count_launch();
    k_f2v_update<<<grid, 256, smem, st>>>(Z.col, Z.val, d, k, r0, b, Gp, Gc, Gv, lr, U_out, Sc, Sv, &hdr->err);
    if ((e = cudaGetLastError())) return e;
    count_launch();
    k_f2v_commit<<<f2v_blocks(b * k), 256, 0, st>>>(r0, b, k, Sc, Sv, const_cast<int*>(Z.col),
                                                     const_cast<float*>(Z.val));
    return cudaGetLastError();
}

}  // namespace ts
