// Numeric pass with B held dense (plus-times, d <= 256): the dense-B SpMM
// form of the product that the paper weighs against TS-SpGEMM (Sec. V, the
// comparison with SpMM: once B is dense enough, a row-wise SpMM over a dense
// B beats the sparse accumulation).  Row i of C is still the structural
// product of Eq. 1: its columns are the union of the patterns of the rows
// B(k,:) that row i of A selects and its values the sums over the stored
// products, so the output is the same CSR C as the sparse path gives.
//
// B is first expanded into a dense row-major copy of w floats per row (w =
// 32 V, V the smallest power of two with 32 V >= d; zeros off the pattern)
// and a bitmap of its pattern (V words per row), both in the workspace.  A
// warp then owns the row: lane l holds the V consecutive columns
// [V l, V l + V) in registers, and for every
// entry (i, k) of A reads the V values and V pattern bits of row k of the
// copy (one or two 16-byte loads: a warp reads the whole row of B in one
// pass), adds a(i,k) * B(k, c) into its registers and ORs the bits.  No
// shared-memory accumulator, no atomics.  The lanes' occupied columns are
// then written out in ascending order (a warp scan of the lanes' counts).
// Heavy rows take a whole block (the warps take shares of the row's entries
// and their partial rows are summed through shared memory); parts of split
// rows are added into the row's staging slot and the block completing the
// last part reads the row out, as in the sparse kernels.
#include "common.cuh"
#include "kernels.h"
#include "numeric.cuh"
#include "denseb.cuh"

namespace ts {

// B expanded: Bd[k * dpad + c] = B(k, c) (0 off the pattern); bits[k * dw + w]
// bit b = (k, 32 w + b) is stored.  Grid-stride over B's entries, after the
// caller has zeroed both arrays.  A column outside [0, d) is an input error.
__global__ void __launch_bounds__(256) k_densify_b(int nB, const long long* __restrict__ Bp, long long nnzB,
                                                   const int* __restrict__ Bi, const float* __restrict__ Bx, int d,
                                                   int dpad, float* __restrict__ Bd, unsigned* __restrict__ bits,
                                                   unsigned long long* err) {
    const int dw = dpad >> 5;
    // one warp per row of B: its entries are contiguous
    for (long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nB;
         k += ((long long)gridDim.x * blockDim.x) >> 5) {
        const long long s = clampll(__ldg(Bp + k), 0, nnzB);
        const long long e = clampll(__ldg(Bp + k + 1), s, nnzB);
        bool bad = false;
        for (long long j = s + lane_id(); j < e; j += 32) {
            const int c = __ldg(Bi + j);
            if ((unsigned)c < (unsigned)d) {
                Bd[k * dpad + c] = __ldg(Bx + j);
                atomicOr(bits + k * dw + (c >> 5), 1u << (c & 31));
            } else {
                bad = true;
            }
        }
        if (bad) atomicOr(err, ERR_B_COL);
    }
}

// Persistent kernel: split parts, heavy rows (one block each), light rows
// (one warp each, natural row order).
template <int V>
__global__ void __launch_bounds__(256) k_numeric_denseb(NumParams p, const float* __restrict__ Bd,
                                                        const unsigned* __restrict__ bits) {
    __shared__ float s_rows[8 * 32 * V];
    __shared__ unsigned s_mask[8 * 32];
    __shared__ long long s_item, s_nheavy;
    __shared__ int s_last;
    __shared__ int s_wcnt[MAX_DENSE_W / 32 + 1];
    constexpr int dpad = 32 * V;
    const int nwarps = blockDim.x >> 5, warp = warp_id(), lane = lane_id(), tid = threadIdx.x;
    if (tid < 32) {
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
    }
    __syncthreads();
    const long long nheavy = s_nheavy;
    unsigned long long* err = &p.hdr->err;
    const bool split_ok = p.s.stg_vals != nullptr;
    const long long* mark = split_ok ? p.s.flops : nullptr;
    const long long nitems = split_ok ? min(*(volatile long long*)&p.hdr->scratch[2], p.item_cap) : 0;
    SplitItem it;
    while (next_split_item(p.s, p.Ap, p.nnzA, nitems, &s_item, it)) {
        float acc[V];
        unsigned m = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0.0f;
        dense_accumulate<V>(p, Bd, bits, dpad, it.e0 + 32LL * warp, it.e1, 32LL * nwarps, acc, m, err);
        dense_block_sum<V>(acc, m, s_rows, s_mask);
        if (warp == 0) {
            float* sv = p.s.stg_vals + (size_t)it.slot * p.s.dpad;
            unsigned char* sf = p.s.stg_flags + (size_t)it.slot * p.s.dpad;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if ((m >> v) & 1u) {
                    atomicAdd(sv + V * lane + v, acc[v]);
                    sf[V * lane + v] = 1;
                }
            }
        }
        if (!split_part_done(p.s, it.slot, it.nsub, &s_last)) continue;
        split_row_readout<true>(p, it, s_wcnt);
    }
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&p.hdr->heavy_ctr, 1ull);
        __syncthreads();
        const long long h = s_item;
        __syncthreads();
        if (h >= nheavy) break;
        const int row = p.perm[h];
        const long long a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
        const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
        if (mark && is_split_row(mark, row, a1 - a0)) continue;
        float acc[V];
        unsigned m = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0.0f;
        dense_accumulate<V>(p, Bd, bits, dpad, a0 + 32LL * warp, a1, 32LL * nwarps, acc, m, err);
        dense_block_sum<V>(acc, m, s_rows, s_mask);
        if (warp == 0) {
            const long long out = clampll(__ldg(p.Cp + row), 0, p.nnzC);
            const long long out_end = clampll(__ldg(p.Cp + row + 1), out, p.nnzC);
            const int tot = dense_emit<V>(acc, m, out, out_end, p.Ci, p.Cx);
            if (lane == 0 && out + tot != out_end) atomicOr(err, ERR_C_ROW);
        }
    }
    // light rows, one per warp, in natural row order (chunks of 32 rows)
    const long long nchunks = ((long long)p.nB + 31) / 32;
    for (long long c = (long long)blockIdx.x * nwarps + warp; c < nchunks; c += (long long)gridDim.x * nwarps) {
        const long long r = c * 32 + lane;
        const long long f = r < p.nB ? __ldg(p.s.flops + r) : 0;
        unsigned rows = __ballot_sync(FULL, f > 0 && flops_class(f) < p.cta_class);
        while (rows) {
            const int row = (int)(c * 32 + __ffs(rows) - 1);
            rows &= rows - 1;
            const long long a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
            const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
            const long long out = clampll(__ldg(p.Cp + row), 0, p.nnzC);
            const long long out_end = clampll(__ldg(p.Cp + row + 1), out, p.nnzC);
            float acc[V];
            unsigned m = 0;
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = 0.0f;
            dense_accumulate<V>(p, Bd, bits, dpad, a0, a1, 32, acc, m, err);
            const int tot = dense_emit<V>(acc, m, out, out_end, p.Ci, p.Cx);
            if (lane == 0 && out + tot != out_end) atomicOr(err, ERR_C_ROW);
        }
    }
}

// Columns per row of the dense copy: 32 times the smallest power of two
// that covers d/32 (so that every lane owns the same power-of-two share).
static int dense_b_width(long long d) {
    int v = 1;
    while (32LL * v < d) v *= 2;
    return 32 * v;
}

size_t dense_b_bytes(long long nB, long long d) {
    const long long w = dense_b_width(d);
    return (size_t)nB * (size_t)w * 4 + (size_t)nB * (size_t)(w / 32) * 4;
}

cudaError_t launch_numeric_denseb(const DevCsr& A, const DevCsr& B, long long d, const Sched& s,
                                  const LaunchCfg& cfg, const long long* Cp, int* Ci, float* Cx, long long nnzC,
                                  void* dense_ws, cudaStream_t st) {
    cudaError_t e;
    if (A.nrows == 0) return cudaSuccess;
    const int dw = dense_b_width(d);
    if (dw > 256 || !dense_ws) return cudaErrorInvalidValue;
    const int V = dw / 32;
    // the dense copy and its pattern, zeroed then filled
    float* Bd = reinterpret_cast<float*>(dense_ws);
    unsigned* bits = reinterpret_cast<unsigned*>(Bd + (size_t)B.nrows * dw);
    if ((e = cudaMemsetAsync(dense_ws, 0, dense_b_bytes(B.nrows, d), st))) return e;
    if (B.nrows > 0 && B.nnz > 0) {
        long long blocks = (B.nrows * 32 + 255) / 256;
        if (blocks > 152LL * 32) blocks = 152LL * 32;
        count_launch();
        k_densify_b<<<(unsigned)blocks, 256, 0, st>>>((int)B.nrows, B.rowptr, B.nnz, B.col, B.val, (int)d, dw, Bd,
                                                      bits, &s.hdr->err);
        if ((e = cudaGetLastError())) return e;
    }
    if ((e = cudaMemsetAsync(&s.hdr->heavy_ctr, 0, 2 * sizeof(unsigned long long), st))) return e;
    NumParams p = numeric_params(A, B, d, dw, 1, nullptr, nullptr, s, cfg, Cp, Ci, Cx, nnzC);
    const void* k = V == 1 ? (const void*)k_numeric_denseb<1>
                  : V == 2 ? (const void*)k_numeric_denseb<2>
                  : V == 4 ? (const void*)k_numeric_denseb<4>
                           : (const void*)k_numeric_denseb<8>;
    const int grid = persistent_grid(k, 256, 0, cfg.sms);
    void* args[] = {&p, &Bd, &bits};
    count_launch();
    if ((e = cudaLaunchKernel(k, dim3(grid), dim3(256), args, 0, st))) return e;
    return cudaGetLastError();
}

}  // namespace ts
