// Sparse Force2Vec minibatch step around the TS-SpGEMM (paper Sec. IV,
// "Distributed sparse embedding"), for the rows [r0, r0 + b) of a sparse
// embedding Z (n x d, exactly k stored entries per row, row i at [k*i, k*i+k)):
//
//   1. W's pattern: row r of the batch merges the neighbours of vertex r0 + r
//      in A (weight class +1) with its s negative samples (class -1); a column
//      met several times keeps its counts of both classes (k_f2v_count /
//      k_f2v_fill, thread per row);
//   2. weights (a sampled dense-dense product on W's pattern):
//      x = z_i . z_j, w = npos * (1 - sigmoid(x)) - nneg * sigmoid(x)
//      (k_f2v_weights, warp per row, z_i scattered into shared memory);
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

__device__ __forceinline__ void sort_small(int* v, int m) {
    for (int a = 1; a < m; ++a) {
        const int x = v[a];
        int b = a - 1;
        while (b >= 0 && v[b] > x) {
            v[b + 1] = v[b];
            --b;
        }
        v[b + 1] = x;
    }
}

// Merge of A's (ascending) row with the row's sorted negatives: calls
// emit(col, npos, nneg) once per distinct column, ascending.
template <class Emit>
__device__ __forceinline__ void f2v_merge(const int* __restrict__ Ai, long long a0, long long a1, const int* negs,
                                          int s, int n, unsigned long long* err, Emit&& emit) {
    long long e = a0;
    int q = 0;
    while (e < a1 || q < s) {
        const int ca = e < a1 ? __ldg(Ai + e) : 0x7FFFFFFF;
        const int cn = q < s ? negs[q] : 0x7FFFFFFF;
        const int c = ca < cn ? ca : cn;
        int np = 0, nn = 0;
        while (e < a1 && __ldg(Ai + e) == c) {
            ++np;
            ++e;
        }
        while (q < s && negs[q] == c) {
            ++nn;
            ++q;
        }
        if ((unsigned)c < (unsigned)n) emit(c, np, nn);
        else atomicOr(err, ERR_A_COL);
    }
}

__device__ __forceinline__ int f2v_load_negs(const int* __restrict__ neg, long long r, int s, int* negs) {
    for (int t = 0; t < s; ++t) negs[t] = __ldg(neg + r * s + t);
    sort_small(negs, s);
    return s;
}

__global__ void __launch_bounds__(256) k_f2v_count(const long long* __restrict__ Ap, const int* __restrict__ Ai,
                                                   long long nnzA, int n, long long r0, long long b,
                                                   const int* __restrict__ neg, int s, long long* cnt,
                                                   unsigned long long* err) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= b) return;
    int negs[F2V_MAX_NEG];
    f2v_load_negs(neg, r, s, negs);
    const long long i = r0 + r;
    const long long a0 = clampll(__ldg(Ap + i), 0, nnzA), a1 = clampll(__ldg(Ap + i + 1), a0, nnzA);
    long long c = 0;
    f2v_merge(Ai, a0, a1, negs, s, n, err, [&](int, int, int) { ++c; });
    cnt[r] = c;
}

__global__ void __launch_bounds__(256) k_f2v_fill(const long long* __restrict__ Ap, const int* __restrict__ Ai,
                                                  long long nnzA, int n, long long r0, long long b,
                                                  const int* __restrict__ neg, int s, const long long* Wp, int* Wcol,
                                                  int* Wmult, unsigned long long* err) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= b) return;
    int negs[F2V_MAX_NEG];
    f2v_load_negs(neg, r, s, negs);
    const long long i = r0 + r;
    const long long a0 = clampll(__ldg(Ap + i), 0, nnzA), a1 = clampll(__ldg(Ap + i + 1), a0, nnzA);
    long long o = Wp[r];
    const long long end = Wp[r + 1];
    f2v_merge(Ai, a0, a1, negs, s, n, err, [&](int c, int np, int nn) {
        if (o < end) {
            Wcol[o] = c;
            Wmult[o] = np | (nn << 16);
        }
        ++o;
    });
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

__global__ void __launch_bounds__(256) k_f2v_weights(const int* __restrict__ Zc, const float* __restrict__ Zv,
                                                     int d, int k, long long r0, long long b,
                                                     const long long* __restrict__ Wp, const int* __restrict__ Wcol,
                                                     const int* __restrict__ Wmult, float* Wval,
                                                     unsigned long long* err) {
    extern __shared__ __align__(16) float fsm[];
    const int nw = blockDim.x >> 5, warp = warp_id(), lane = lane_id();
    const int dpad = (d + 31) & ~31;
    float* g = fsm + (size_t)warp * dpad;
    for (int c = lane; c < dpad; c += 32) g[c] = 0.0f;
    __syncwarp();
    for (long long r = (long long)blockIdx.x * nw + warp; r < b; r += (long long)gridDim.x * nw) {
        const long long i = r0 + r;
        f2v_scatter(Zc, Zv, i, k, d, g, false);
        __syncwarp();
        for (long long e = Wp[r]; e < Wp[r + 1]; ++e) {
            const long long j = __ldg(Wcol + e);
            float x = 0.0f;
            for (int t = lane; t < k; t += 32) {
                const int c = __ldg(Zc + j * k + t);
                if ((unsigned)c < (unsigned)d) x += g[c] * __ldg(Zv + j * k + t);
                else atomicOr(err, ERR_B_COL);
            }
            x = warp_sum(x);
            if (lane == 0) {
                const int m = __ldg(Wmult + e);
                const float sg = 1.0f / (1.0f + expf(-x));
                Wval[e] = (float)(m & 0xFFFF) * (1.0f - sg) - (float)(m >> 16) * sg;
            }
        }
        __syncwarp();
        f2v_scatter(Zc, Zv, i, k, d, g, true);
        __syncwarp();
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

static unsigned f2v_blocks(long long m) {
    long long g = (m + 255) / 256;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)g;
}

cudaError_t launch_f2v_pattern(const DevCsr& A, long long r0, long long b, const int* neg, int s, long long* Wp,
                               long long* partial, WsHeader* hdr, cudaStream_t st) {
    cudaError_t e;
    if (s < 0 || s > F2V_MAX_NEG) return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(Wp, 0, sizeof(long long), st))) return e;
    if (b == 0) return cudaSuccess;
    count_launch();
    k_f2v_count<<<(unsigned)((b + 255) / 256), 256, 0, st>>>(A.rowptr, A.col, A.nnz, (int)A.nrows, r0, b, neg, s,
                                                             Wp + 1, &hdr->err);
    if ((e = cudaGetLastError())) return e;
    return launch_scan_inplace(Wp + 1, b, partial, st);
}

cudaError_t launch_f2v_fill(const DevCsr& A, long long r0, long long b, const int* neg, int s, const long long* Wp,
                            int* Wcol, int* Wmult, WsHeader* hdr, cudaStream_t st) {
    if (b == 0) return cudaSuccess;
    count_launch();
    k_f2v_fill<<<(unsigned)((b + 255) / 256), 256, 0, st>>>(A.rowptr, A.col, A.nnz, (int)A.nrows, r0, b, neg, s,
                                                            Wp, Wcol, Wmult, &hdr->err);
    return cudaGetLastError();
}

cudaError_t launch_f2v_check(const DevCsr& Z, int k, WsHeader* hdr, cudaStream_t st) {
    count_launch();
    k_f2v_check_rows<<<(unsigned)((Z.nrows + 1 + 255) / 256), 256, 0, st>>>(Z.rowptr, Z.nrows, k, &hdr->err);
    return cudaGetLastError();
}

cudaError_t launch_f2v_weights(const DevCsr& Z, int k, long long r0, long long b, const long long* Wp,
                               const int* Wcol, const int* Wmult, float* Wval, int sms, WsHeader* hdr,
                               cudaStream_t st) {
    if (b == 0) return cudaSuccess;
    const int d = (int)Z.ncols, dpad = (d + 31) & ~31;
    const size_t smem = sizeof(float) * (size_t)dpad * 8;
    cudaError_t e;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute((const void*)k_f2v_weights, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
        return e;
    const int grid = persistent_grid((const void*)k_f2v_weights, 256, smem, sms);
    count_launch();
    k_f2v_weights<<<grid, 256, smem, st>>>(Z.col, Z.val, d, k, r0, b, Wp, Wcol, Wmult, Wval, &hdr->err);
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
