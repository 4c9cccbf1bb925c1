// Backward of C = A*B (plus-times) with fixed patterns, for L = <dC, C>:
//   dA(i,k) = sum over j in B_k of dC(i,j) * B(k,j)        (SDDMM on A's pattern)
//   dB(k,j) = sum over i with (i,k) in A of A(i,k) * dC(i,j) (A^T dC on B's pattern)
// Both are computed in one traversal with the forward's schedule: row i of dC
// is scattered into a dense shared-memory row g (width d), then every product
// (k, j) of row i reads g[B.col[j]] once: the dot products for dA are reduced
// across lanes, and the dB terms are added to dB[j] with float atomics.
#include "common.cuh"
#include "kernels.h"

namespace ts {

constexpr int MAX_BWD_D = 8192;

struct BwdParams {
    const long long* Ap;
    const int* Ai;
    const float* Ax;
    long long nnzA;
    const long long* Bp;
    const int* Bi;
    const float* Bx;
    long long nnzB;
    int nB;
    int d;
    int dpad;
    const long long* Cp;
    const int* Ci;
    const float* dC;
    long long nnzC;
    float* dA;
    float* dB;
    const int* perm;
    WsHeader* hdr;
    int cta_class;
};

// Sum of v over the run of equal keys that starts at this lane (keys are
// non-decreasing across lanes); only a run's first lane's result is used.
__device__ __forceinline__ float seg_sum_down(float v, int key) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_down_sync(FULL, v, o);
        const int k = __shfl_down_sync(FULL, key, o);
        if (lane + o < 32 && k == key) v += t;
    }
    return v;
}

struct BwdVisit {
    const int* __restrict__ Bi;
    const float* __restrict__ Bx;
    const float* g;
    float* sdA;  // 32 partial dot products of this warp's chunk
    float* dB;
    bool want_dA;
    int d;
    unsigned long long* err;
    __device__ __forceinline__ void one(long long j, float a, int q, bool ok) {
        float contrib = 0.0f;
        if (ok) {
            const int c = __ldg(Bi + j);
            if ((unsigned)c < (unsigned)d) {
                const float gj = g[c];
                contrib = __ldg(Bx + j) * gj;
                if (dB) atomicAdd(dB + j, a * gj);
            } else {
                atomicOr(err, ERR_B_COL);
            }
        }
        if (want_dA) {
            const float s = seg_sum_down(contrib, q);
            const int prevq = __shfl_up_sync(FULL, q, 1);
            if (ok && (lane_id() == 0 || prevq != q)) atomicAdd(sdA + q, s);
        }
    }
    __device__ __forceinline__ void step4(const long long* j, const float* a, const int* q) {
        int c[4];
        float b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = __ldg(Bi + j[u]);
            b[u] = __ldg(Bx + j[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float contrib = 0.0f;
            if ((unsigned)c[u] < (unsigned)d) {
                const float gj = g[c[u]];
                contrib = b[u] * gj;
                if (dB) atomicAdd(dB + j[u], a[u] * gj);
            } else {
                atomicOr(err, ERR_B_COL);
            }
            if (want_dA) {
                const float s = seg_sum_down(contrib, q[u]);
                const int prevq = __shfl_up_sync(FULL, q[u], 1);
                if (lane_id() == 0 || prevq != q[u]) atomicAdd(sdA + q[u], s);
            }
        }
    }
    __device__ __forceinline__ void step1(long long j, float a, int q, bool ok) { one(j, a, q, ok); }
};

template <bool CTA>
__device__ __forceinline__ void backward_row(const BwdParams& p, int row, float* g, float* sdA) {
    unsigned long long* err = &p.hdr->err;
    const int lane = lane_id();
    const long long a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
    const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
    const long long c0 = clampll(__ldg(p.Cp + row), 0, p.nnzC);
    const long long c1 = clampll(__ldg(p.Cp + row + 1), c0, p.nnzC);
    const int tid = CTA ? threadIdx.x : lane;
    const int nthr = CTA ? blockDim.x : 32;
    for (long long e = c0 + tid; e < c1; e += nthr) {
        const int c = __ldg(p.Ci + e);
        if ((unsigned)c < (unsigned)p.d) g[c] = __ldg(p.dC + e);
        else atomicOr(err, ERR_C_ROW);
    }
    if (CTA) __syncthreads();
    else __syncwarp();
    const int nw = blockDim.x >> 5;
    const long long first = CTA ? a0 + 32LL * warp_id() : a0;
    const long long stride = CTA ? 32LL * nw : 32LL;
    const SegWhole seg{p.Bp, p.nnzB, p.d};
    BwdVisit vis{p.Bi, p.Bx, g, sdA, p.dB, p.dA != nullptr, p.d, err};
    for (long long e0 = first; e0 < a1; e0 += stride) {
        const int nv = (int)(a1 - e0 < 32 ? a1 - e0 : 32);
        expand_chunk(e0, nv, p.Ai, p.Ax, p.nB, seg, vis, err);
        __syncwarp();
        if (p.dA) {
            if (lane < nv) p.dA[e0 + lane] = sdA[lane];
            sdA[lane] = 0.0f;
            __syncwarp();
        }
    }
    if (CTA) __syncthreads();
    else __syncwarp();
    for (long long e = c0 + tid; e < c1; e += nthr) {
        const int c = __ldg(p.Ci + e);
        if ((unsigned)c < (unsigned)p.d) g[c] = 0.0f;
    }
    if (CTA) __syncthreads();
    else __syncwarp();
}

__global__ void __launch_bounds__(1024) k_backward(BwdParams p) {
    extern __shared__ __align__(16) float fsm[];
    __shared__ long long s_item, s_nheavy, s_nrows;
    const int nw = blockDim.x >> 5, warp = warp_id(), tid = threadIdx.x;
    // layout: [nw][dpad] dense dC rows, then [nw][32] dA partials
    for (int i = tid; i < nw * (p.dpad + 32); i += blockDim.x) fsm[i] = 0.0f;
    if (tid == 0) {
        long long nh = 0, nr = 0;
        for (int c = 1; c < NUM_CLASSES; ++c) {
            nr += p.hdr->hist[c];
            if (c >= p.cta_class) nh += p.hdr->hist[c];
        }
        s_nheavy = nh;
        s_nrows = nr;
    }
    __syncthreads();
    const long long nheavy = s_nheavy, nrows = s_nrows;
    float* sdA = fsm + (size_t)nw * p.dpad + 32 * warp;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&p.hdr->heavy_ctr, 1ull);
        __syncthreads();
        const long long h = s_item;
        __syncthreads();
        if (h >= nheavy) break;
        backward_row<true>(p, p.perm[h], fsm, sdA);
    }
    float* g = fsm + (size_t)warp * p.dpad;
    for (long long idx = nheavy + (long long)blockIdx.x * nw + warp; idx < nrows;
         idx += (long long)gridDim.x * nw)
        backward_row<false>(p, p.perm[idx], g, sdA);
}

size_t backward_smem(long long d, int warps) {
    const long long dpad = (d + 31) / 32 * 32;
    return sizeof(float) * (size_t)warps * (size_t)(dpad + 32);
}

cudaError_t launch_backward(const DevCsr& A, const DevCsr& B, long long d, const long long* Cp,
                            const int* Ci, long long nnzC, const float* dC, float* dA, float* dB,
                            const Sched& s, const LaunchCfg& cfg, cudaStream_t st) {
    cudaError_t e;
    if (d > MAX_BWD_D) return cudaErrorInvalidValue;
    if (dA && A.nnz && (e = cudaMemsetAsync(dA, 0, sizeof(float) * A.nnz, st))) return e;
    if (dB && B.nnz && (e = cudaMemsetAsync(dB, 0, sizeof(float) * B.nnz, st))) return e;
    if (A.nrows == 0 || (!dA && !dB)) return cudaSuccess;
    if ((e = cudaMemsetAsync(&s.hdr->heavy_ctr, 0, sizeof(unsigned long long), st))) return e;
    BwdParams p;
    p.Ap = A.rowptr;
    p.Ai = A.col;
    p.Ax = A.val;
    p.nnzA = A.nnz;
    p.Bp = B.rowptr;
    p.Bi = B.col;
    p.Bx = B.val;
    p.nnzB = B.nnz;
    p.nB = (int)B.nrows;
    p.d = (int)d;
    p.dpad = (int)((d + 31) / 32 * 32);
    p.Cp = Cp;
    p.Ci = Ci;
    p.dC = dC;
    p.nnzC = nnzC;
    p.dA = dA;
    p.dB = dB;
    p.perm = s.perm;
    p.hdr = s.hdr;
    p.cta_class = cfg.cta_class;
    int warps = cfg.warps_per_cta;
    size_t smem = backward_smem(d, warps);
    while (smem > 200 * 1024 && warps > 1) {
        warps /= 2;
        smem = backward_smem(d, warps);
    }
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute((const void*)k_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
        return e;
    const int grid = persistent_grid((const void*)k_backward, 32 * warps, smem, cfg.sms);
    count_launch();
    k_backward<<<grid, 32 * warps, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace ts
