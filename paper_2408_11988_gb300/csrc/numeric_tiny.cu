// Tiny rows of the wide numeric pass (plus-times, one column tile of
// 256 < W <= 1024): rows with 1 .. TINY_MAX products.  In R-MAT products
// about half of the non-empty rows are of this kind (at d = 1024, 1 %; under
// 5 % of the products), and on the wide kernel's path each costs a whole
// pass of a warp over a 1024-column accumulator and a bitmap read-out for a
// few dozen products.
// Here a row is expanded, sorted and compressed in registers (Eq. 1 written
// as a sum over the row's products grouped by column): lane j takes the
// row's j-th product, the warp sorts the (column, value) pairs by column
// (bitonic network over the lanes; a row of one entry needs no sort and a
// row of two only the merge), sums each run of equal columns into its first
// lane and writes the runs' heads to the row of C in ascending column order
// with one coalesced store.  No shared memory, no atomics; duplicates
// are summed in sorted order.  The wide kernel, launched after this one
// with tiny_max = TINY_MAX, leaves these rows alone.
#include "common.cuh"
#include "kernels.h"
#include "numeric.cuh"
#include "wide.cuh"

namespace ts {

// Ascending bitonic sort of one (key, value) pair per lane across the warp.
__device__ __forceinline__ void warp_sort_kv(int& key, float& val) {
    const int lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int pk = __shfl_xor_sync(FULL, key, j);
            const float pv = __shfl_xor_sync(FULL, val, j);
            const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
            if (keep_min ? pk < key : pk > key) {
                key = pk;
                val = pv;
            }
        }
    }
}

// The row's products, sorted by column (key; 0x7FFFFFFF on lanes without
// one), summed per column into the first lane of each run and written to
// C[out, out_end) in ascending column order; dup = whether equal columns can
// occur (more than one row of B), runs = their longest possible length.
__device__ __forceinline__ void tiny_emit(const NumParams& p, int key, float val, bool dup, int runs, long long out,
                                          long long out_end, unsigned long long* err) {
    const int lane = lane_id();
    float sum = val;
    if (dup) {
        for (int o = 1; o < runs; o <<= 1) {  // warp-uniform bound
            const float t = __shfl_down_sync(FULL, sum, o);
            const int ko = __shfl_down_sync(FULL, key, o);
            if (lane + o < 32 && ko == key) sum += t;
        }
    }
    const int prev = __shfl_up_sync(FULL, key, 1);
    const bool head = key != 0x7FFFFFFF && (!dup || lane == 0 || prev != key);
    const unsigned hb = __ballot_sync(FULL, head);
    if (head) {
        const long long pos = out + __popc(hb & lanemask_lt());
        if (pos < out_end) {
            p.Ci[pos] = key;
            if (p.Cx) p.Cx[pos] = sum;
        }
    }
    if (lane == 0 && out + __popc(hb) != out_end) atomicOr(err, ERR_C_ROW);
}

// Row [a0, a1) of A with at most 32 products.  Rows of up to TINY_ENT
// entries arrive with their rows of B described (first pair g[u], entries
// n[u], value x[u], loaded for the whole chunk at once), so only the rows of
// B themselves remain to be read.  One entry: its row of B, scaled, is the
// row of C (already sorted, no duplicates).  Two entries: the two sorted
// rows of B side by side, the second reversed at the top lanes, form a
// bitonic sequence that five merge steps sort.  More: the products placed
// one per lane and sorted by the full network.
constexpr int TINY_ENT = 3;

__device__ __forceinline__ void tiny_row(const NumParams& p, const int2* __restrict__ Q, long long a0, long long a1,
                                         long long out, long long out_end, const unsigned (&g)[TINY_ENT],
                                         const int (&n)[TINY_ENT], const float (&x)[TINY_ENT],
                                         unsigned long long* err) {
    const int lane = lane_id();
    const unsigned W = (unsigned)p.W;
    int key = 0x7FFFFFFF;  // no product: sorts last
    float val = 0.0f;
    const long long na = a1 - a0;
    if (na == 1) {
        if (lane < n[0]) {
            const int2 v = __ldg(Q + 2 * (size_t)g[0] + lane);
            if ((unsigned)v.x < W) {  // a bad column (-1) adds nothing
                key = v.x;
                val = x[0] * __int_as_float(v.y);
            }
        }
        tiny_emit(p, key, val, false, 1, out, out_end, err);
        return;
    }
    if (na == 2 && n[0] + n[1] <= 32) {
        const int j1 = 31 - lane;  // the second row, reversed, at the top lanes
        int2 v = make_int2(-1, 0);
        float a = 0.0f;
        if (lane < n[0]) {
            v = __ldg(Q + 2 * (size_t)g[0] + lane);
            a = x[0];
        } else if (j1 < n[1]) {
            v = __ldg(Q + 2 * (size_t)g[1] + j1);
            a = x[1];
        }
        if ((unsigned)v.x < W) {
            key = v.x;
            val = a * __int_as_float(v.y);
        }
        // bitonic merge: ascending (first row), empty lanes, descending (second row)
#pragma unroll
        for (int j = 16; j > 0; j >>= 1) {
            const int pk = __shfl_xor_sync(FULL, key, j);
            const float pv = __shfl_xor_sync(FULL, val, j);
            if (((lane & j) == 0) ? pk < key : pk > key) {
                key = pk;
                val = pv;
            }
        }
        tiny_emit(p, key, val, true, 2, out, out_end, err);
        return;
    }
    if (na <= TINY_ENT && n[0] + n[1] + n[2] <= 32) {
        int2 v = make_int2(-1, 0);
        float a = 0.0f;
        if (lane < n[0]) {
            v = __ldg(Q + 2 * (size_t)g[0] + lane);
            a = x[0];
        } else if (lane < n[0] + n[1]) {
            v = __ldg(Q + 2 * (size_t)g[1] + (lane - n[0]));
            a = x[1];
        } else if (lane < n[0] + n[1] + n[2]) {
            v = __ldg(Q + 2 * (size_t)g[2] + (lane - n[0] - n[1]));
            a = x[2];
        }
        if ((unsigned)v.x < W) {
            key = v.x;
            val = a * __int_as_float(v.y);
        }
        warp_sort_kv(key, val);
        tiny_emit(p, key, val, true, 4, out, out_end, err);
        return;
    }
    // longer runs of entries (rows of B that are empty among them)
    int base = 0;  // products placed so far (warp-uniform)
    for (long long ec = a0; ec < a1 && base < 32; ec += 32) {
        const long long e = ec + lane;
        int len = 0;
        long long s = 0;
        unsigned g0 = 0;
        float a = 0.0f;
        if (e < a1) {
            const int k = __ldg(p.Ai + e);
            a = p.Ax ? __ldg(p.Ax + e) : 1.0f;
            if ((unsigned)k < (unsigned)p.nB) padded_row<2>(p.Bp, p.nnzB, p.d, k, s, len, g0);
            else atomicOr(err, ERR_A_COL);
        }
        const int incl = warp_incl_scan(len), excl = incl - len;
        const int tot = __shfl_sync(FULL, incl, 31);
        // lane j takes product j - base of this round of entries
        const int pj = lane - base;
        const int q = owner_lane(excl, pj < 0 ? 0 : pj);
        const unsigned gq = __shfl_sync(FULL, g0, q);
        const int eq = __shfl_sync(FULL, excl, q);
        const float aq = __shfl_sync(FULL, a, q);
        if (pj >= 0 && pj < tot) {
            const int2 v = __ldg(Q + 2 * (size_t)gq + (pj - eq));
            if ((unsigned)v.x < W) {
                key = v.x;
                val = aq * __int_as_float(v.y);
            }
        }
        base += tot;
    }
    warp_sort_kv(key, val);
    tiny_emit(p, key, val, true, 32, out, out_end, err);
}

// Every light row with 1 .. TINY_MAX products (split rows carry negative
// marks in the flops array and are never tiny; with a heavy threshold that
// low, heavy rows stay with the wide kernel's blocks), 32-row chunks dealt
// to the warps in turn.  Lane l loads what row l of the chunk needs before
// its rows of B (bounds in A and C, up to TINY_ENT entries of A and their
// rows' descriptions), all rows of the chunk at once, so that a row then
// waits for one round of loads only.
__global__ void __launch_bounds__(256, 6) k_numeric_tiny(NumParams p) {
    const int lane = lane_id();
    unsigned long long* err = &p.hdr->err;
    const int2* Q = reinterpret_cast<const int2*>(p.Bq);
    const long long nchunks = ((long long)p.nB + 31) / 32;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long c = gw; c < nchunks; c += nw) {
        const long long r = c * 32 + lane;
        const long long f = r < p.nB ? __ldg(p.s.flops + r) : 0;
        const bool tiny = f >= 1 && f <= TINY_MAX && flops_class(f) < p.cta_class;  // light rows only
        long long a0 = 0, a1 = 0, o0 = 0, o1 = 0;
        if (tiny) {
            a0 = clampll(__ldg(p.Ap + r), 0, p.nnzA);
            a1 = clampll(__ldg(p.Ap + r + 1), a0, p.nnzA);
            o0 = clampll(__ldg(p.Cp + r), 0, p.nnzC);
            o1 = clampll(__ldg(p.Cp + r + 1), o0, p.nnzC);
        }
        unsigned gl[TINY_ENT];
        int nl[TINY_ENT];
        float xl[TINY_ENT];
        int kl[TINY_ENT];
#pragma unroll
        for (int u = 0; u < TINY_ENT; ++u) {
            kl[u] = -1;
            xl[u] = 0.0f;
            if (tiny && a0 + u < a1 && a1 - a0 <= TINY_ENT) {
                kl[u] = __ldg(p.Ai + a0 + u);
                xl[u] = p.Ax ? __ldg(p.Ax + a0 + u) : 1.0f;
            }
        }
#pragma unroll
        for (int u = 0; u < TINY_ENT; ++u) {
            gl[u] = 0;
            nl[u] = 0;
            if (tiny && a0 + u < a1 && a1 - a0 <= TINY_ENT) {
                long long s;
                if ((unsigned)kl[u] < (unsigned)p.nB) padded_row<2>(p.Bp, p.nnzB, p.d, kl[u], s, nl[u], gl[u]);
                else atomicOr(err, ERR_A_COL);
            }
        }
        unsigned rows = __ballot_sync(FULL, tiny);
        while (rows) {
            const int src = __ffs(rows) - 1;
            rows &= rows - 1;
            unsigned g[TINY_ENT];
            int n[TINY_ENT];
            float x[TINY_ENT];
#pragma unroll
            for (int u = 0; u < TINY_ENT; ++u) {
                g[u] = __shfl_sync(FULL, gl[u], src);
                n[u] = __shfl_sync(FULL, nl[u], src);
                x[u] = __shfl_sync(FULL, xl[u], src);
            }
            tiny_row(p, Q, shfl64(a0, src), shfl64(a1, src), shfl64(o0, src), shfl64(o1, src), g, n, x, err);
        }
    }
}

cudaError_t launch_numeric_tiny(const NumParams& p, int sms, cudaStream_t st) {
    if (p.nB == 0 || !p.Bq) return cudaSuccess;
    const int grid = persistent_grid((const void*)k_numeric_tiny, 256, 0, sms);
    count_launch();
    k_numeric_tiny<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace ts
