// Device pieces of the dense-B numeric form (numeric_denseb.cu), shared with
// the batched kernels: a lane's V columns of a row of the dense copy of B,
// the register accumulation of a row's entries, the block sum of partial
// rows and the read-out of the occupied columns.
#pragma once

#include "common.cuh"
#include "numeric.cuh"

namespace ts {

// V columns of row k of the dense copy for this lane, and their pattern bits
// (bit v = column cb + V * lane + v; cb, a multiple of 32 V, selects a band
// of a row wider than 32 V).
template <int V>
__device__ __forceinline__ void dense_row_load(const float* __restrict__ Bd, const unsigned* __restrict__ bits,
                                               int dpad, int k, float (&b)[V], unsigned& m, int cb = 0) {
    const int lane = lane_id();
    const float* r = Bd + (size_t)k * dpad + cb + V * lane;
    if constexpr (V == 8) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(r));
        const float4 y = __ldg(reinterpret_cast<const float4*>(r) + 1);
        b[0] = x.x; b[1] = x.y; b[2] = x.z; b[3] = x.w; b[4] = y.x; b[5] = y.y; b[6] = y.z; b[7] = y.w;
    } else if constexpr (V == 4) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(r));
        b[0] = x.x; b[1] = x.y; b[2] = x.z; b[3] = x.w;
    } else if constexpr (V == 2) {
        const float2 x = __ldg(reinterpret_cast<const float2*>(r));
        b[0] = x.x; b[1] = x.y;
    } else {
        b[0] = __ldg(r);
    }
    const int dw = dpad >> 5;
    const unsigned w = __ldg(bits + (size_t)k * dw + ((cb + V * lane) >> 5));
    m = (w >> ((V * lane) & 31)) & ((V == 32 ? 0u : (1u << V)) - 1u);
}

// Entries [e0, e1) of A (this warp takes e0 + lane, e0 + lane + 32 * stride... in
// chunks): row sums into acc and the union of the patterns into m (columns
// cb .. cb + 32 V - 1).
template <int V>
__device__ __forceinline__ void dense_accumulate(const NumParams& p, const float* __restrict__ Bd,
                                                 const unsigned* __restrict__ bits, int dpad, long long first,
                                                 long long e1, long long stride, float (&acc)[V], unsigned& m,
                                                 unsigned long long* err, int cb = 0) {
    const int lane = lane_id();
    for (long long e = first; e < e1; e += stride) {
        const int nv = e1 - e < 32 ? (int)(e1 - e) : 32;
        int k = -1;
        float a = 0.0f;
        if (lane < nv) {
            k = __ldg(p.Ai + e + lane);
            a = __ldg(p.Ax + e + lane);
            if ((unsigned)k >= (unsigned)p.nB) {
                atomicOr(err, ERR_A_COL);
                k = -1;
            }
        }
        // two rows of B in flight per step
        int u = 0;
        for (; u + 2 <= nv; u += 2) {
            const int k0 = __shfl_sync(FULL, k, u), k1 = __shfl_sync(FULL, k, u + 1);
            const float a0 = __shfl_sync(FULL, a, u), a1 = __shfl_sync(FULL, a, u + 1);
            float b0[V], b1[V];
            unsigned m0 = 0, m1 = 0;
            if (k0 >= 0) dense_row_load<V>(Bd, bits, dpad, k0, b0, m0, cb);
            if (k1 >= 0) dense_row_load<V>(Bd, bits, dpad, k1, b1, m1, cb);
            if (k0 >= 0) {
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = fmaf(a0, b0[v], acc[v]);
                m |= m0;
            }
            if (k1 >= 0) {
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = fmaf(a1, b1[v], acc[v]);
                m |= m1;
            }
        }
        if (u < nv) {
            const int k0 = __shfl_sync(FULL, k, u);
            const float a0 = __shfl_sync(FULL, a, u);
            if (k0 >= 0) {
                float b0[V];
                unsigned m0 = 0;
                dense_row_load<V>(Bd, bits, dpad, k0, b0, m0, cb);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = fmaf(a0, b0[v], acc[v]);
                m |= m0;
            }
        }
    }
}

// The warp's occupied columns (cb + V * lane + v) written to C[out, out_end)
// in ascending order; returns the count.
template <int V>
__device__ __forceinline__ int dense_emit(const float (&acc)[V], unsigned m, long long out, long long out_end,
                                          int* Ci, float* Cx, int cb = 0) {
    const int lane = lane_id();
    const int cnt = __popc(m);
    const int incl = warp_incl_scan(cnt);
    long long pos = out + incl - cnt;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        if ((m >> v) & 1u) {
            if (pos < out_end) {
                Ci[pos] = cb + V * lane + v;
                Cx[pos] = acc[v];
            }
            ++pos;
        }
    }
    return __shfl_sync(FULL, incl, 31);
}

// Block sum of the warps' partial rows (shared: warps x dpad floats and
// warps x 32 masks); warp 0 ends with the row in acc / m.
template <int V>
__device__ __forceinline__ void dense_block_sum(float (&acc)[V], unsigned& m, float* s_rows, unsigned* s_mask) {
    const int warp = warp_id(), lane = lane_id(), nw = blockDim.x >> 5;
    const int dpad = 32 * V;
#pragma unroll
    for (int v = 0; v < V; ++v) s_rows[warp * dpad + V * lane + v] = acc[v];
    s_mask[warp * 32 + lane] = m;
    __syncthreads();
    if (warp == 0) {
        for (int w = 1; w < nw; ++w) {
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += s_rows[w * dpad + V * lane + v];
            m |= s_mask[w * 32 + lane];
        }
    }
    __syncthreads();
}

}  // namespace ts
