// Batched TS-SpGEMM: many independent products C_b = A_b * B_b of uneven
// shapes.  The batch is the single product of the block-diagonal matrix
// diag(A_1, ..., A_m) with the stacked matrix [B_1; ...; B_m] (every B_b has
// columns < d_b <= d_max), whose row block b is exactly C_b.  One kernel
// gathers the instances into that product's arrays, the single-product passes
// run once over all rows (one launch per phase), and one kernel scatters the
// rows back into the instances' own C (and gradient) arrays.  Nothing here
// synchronises with the host, so the whole sequence can be captured in a
// CUDA graph and replayed.
#include "common.cuh"
#include "kernels.h"

namespace ts {

// Gather the instances into the concatenated CSR arrays.  Row r of instance
// b becomes row row_off + r; column k of A_b becomes row_off + k (block
// diagonal); B's columns are unchanged.  blockIdx.y = instance.
__global__ void __launch_bounds__(256) k_batch_gather(const InstDesc* __restrict__ inst, long long* Ap, int* Ai,
                                                      float* Ax, long long* Bp, int* Bi, float* Bx) {
    const InstDesc I = inst[blockIdx.y];
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = t0; i <= I.n; i += stride) {
        Ap[I.row_off + i] = clampll(I.A_rowptr[i], 0, I.annz) + I.annz_off;
        Bp[I.row_off + i] = clampll(I.B_rowptr[i], 0, I.bnnz) + I.bnnz_off;
    }
    for (long long e = t0; e < I.annz; e += stride) {
        const int k = I.A_col[e];
        Ai[I.annz_off + e] = ((unsigned)k < (unsigned)I.n) ? (int)(I.row_off + k) : -1;  // -1: caught as bad column
        if (Ax) Ax[I.annz_off + e] = I.A_val[e];
    }
    for (long long e = t0; e < I.bnnz; e += stride) {
        const int c = I.B_col[e];
        Bi[I.bnnz_off + e] = ((unsigned)c < (unsigned)I.d) ? c : -1;
        if (Bx) Bx[I.bnnz_off + e] = I.B_val[e];
    }
}

// Scatter rows of the concatenated C back into each instance's C: rebased row
// pointers, then the instance's range of columns and values.  An instance
// whose C does not fit its capacity gets ERR_CAPACITY and its rowptr only.
__global__ void __launch_bounds__(256) k_batch_scatter(const InstDesc* __restrict__ inst, const long long* Cp,
                                                       const int* Ci, const float* Cx, unsigned long long* err) {
    const InstDesc I = inst[blockIdx.y];
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long base = Cp[I.row_off], end = Cp[I.row_off + I.n];
    const long long cnt = end - base;
    for (long long i = t0; i <= I.n; i += stride) I.C_rowptr[i] = Cp[I.row_off + i] - base;
    if (cnt > I.cap) {
        if (t0 == 0) atomicOr(err, ERR_CAPACITY);
        return;
    }
    for (long long e = t0; e < cnt; e += stride) {
        I.C_col[e] = Ci[base + e];
        if (I.C_val && Cx) I.C_val[e] = Cx[base + e];
    }
}

// Upper bound on nnz(C_b): sum over its rows of min(d_b, flops_i), from the
// flops of the concatenated product.  Block per instance.
__global__ void __launch_bounds__(256) k_batch_bounds(const InstDesc* __restrict__ inst, const long long* flops,
                                                      long long* bound) {
    const InstDesc I = inst[blockIdx.x];
    long long s = 0;
    for (long long i = threadIdx.x; i < I.n; i += blockDim.x) {
        const long long f = flops[I.row_off + i];
        s += f < I.d ? f : I.d;
    }
    s = warp_sum(s);
    __shared__ long long red[8];
    if (lane_id() == 0) red[warp_id()] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        bound[blockIdx.x] = t;
    }
}

// dC of every instance into the concatenated layout (C's rows of instance b
// start at Cp[row_off]).
__global__ void __launch_bounds__(256) k_batch_gather_dc(const InstDesc* __restrict__ inst, const long long* Cp,
                                                         float* dC) {
    const InstDesc I = inst[blockIdx.y];
    if (!I.dC) return;
    const long long base = Cp[I.row_off], cnt = Cp[I.row_off + I.n] - base;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = t0; e < cnt && e < I.cap; e += stride) dC[base + e] = I.dC[e];
}

// dA and dB of the concatenated product back to the instances.
__global__ void __launch_bounds__(256) k_batch_scatter_grads(const InstDesc* __restrict__ inst, const float* dA,
                                                             const float* dB) {
    const InstDesc I = inst[blockIdx.y];
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (I.dA && dA)
        for (long long e = t0; e < I.annz; e += stride) I.dA[e] = dA[I.annz_off + e];
    if (I.dB && dB)
        for (long long e = t0; e < I.bnnz; e += stride) I.dB[e] = dB[I.bnnz_off + e];
}

static unsigned grid_x(long long max_work) {
    long long g = (max_work + 255) / 256;
    if (g < 1) g = 1;
    if (g > 64) g = 64;
    return (unsigned)g;
}

cudaError_t launch_batch_gather(const InstDesc* inst, int count, long long max_work, long long* Ap, int* Ai,
                                float* Ax, long long* Bp, int* Bi, float* Bx, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    count_launch();
    k_batch_gather<<<dim3(grid_x(max_work), count), 256, 0, st>>>(inst, Ap, Ai, Ax, Bp, Bi, Bx);
    return cudaGetLastError();
}

cudaError_t launch_batch_scatter(const InstDesc* inst, int count, long long max_work, const long long* Cp,
                                 const int* Ci, const float* Cx, unsigned long long* err, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    count_launch();
    k_batch_scatter<<<dim3(grid_x(max_work), count), 256, 0, st>>>(inst, Cp, Ci, Cx, err);
    return cudaGetLastError();
}

cudaError_t launch_batch_bounds(const InstDesc* inst, int count, const long long* flops, long long* bound,
                                cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    count_launch();
    k_batch_bounds<<<count, 256, 0, st>>>(inst, flops, bound);
    return cudaGetLastError();
}

cudaError_t launch_batch_gather_dc(const InstDesc* inst, int count, long long max_work, const long long* Cp,
                                   float* dC, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    count_launch();
    k_batch_gather_dc<<<dim3(grid_x(max_work), count), 256, 0, st>>>(inst, Cp, dC);
    return cudaGetLastError();
}

cudaError_t launch_batch_scatter_grads(const InstDesc* inst, int count, long long max_work, const float* dA,
                                       const float* dB, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    count_launch();
    k_batch_scatter_grads<<<dim3(grid_x(max_work), count), 256, 0, st>>>(inst, dA, dB);
    return cudaGetLastError();
}

}  // namespace ts
