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

// Rows of up to TINY_ENT entries arrive with their rows of B described
// (first pair g[u], entries n[u], value x[u], loaded for the whole chunk at
// once), so only the rows of B themselves remain to be read: tiny_fetch
// issues this lane's load for one row, and the kernel issues the next row's
// before it processes the current one.
constexpr int TINY_ENT = 3;

// A tiny row as the pipeline carries it.
struct TinyRow {
    long long a0, a1, out, out_end;
};

// This lane's product of a row of at most TINY_ENT entries (v.x = -1: none).
// One entry: lane j takes entry j of the row of B.  Two: the first row of B
// from lane 0 up, the second reversed from lane 31 down (a bitonic sequence
// once sorted keys sit in the lanes).  Three: the rows one after another.
__device__ __forceinline__ void tiny_fetch(const int2* __restrict__ Q, int na, const unsigned (&g)[TINY_ENT],
                                           const int (&n)[TINY_ENT], const float (&x)[TINY_ENT], int2& v, float& a) {
    const int lane = lane_id();
    v = make_int2(-1, 0);
    a = 0.0f;
    if (na == 1) {
        if (lane < n[0]) {
            v = __ldg(Q + 2 * (size_t)g[0] + lane);
            a = x[0];
        }
    } else if (na == 2) {
        const int j1 = 31 - lane;
        if (lane < n[0]) {
            v = __ldg(Q + 2 * (size_t)g[0] + lane);
            a = x[0];
        } else if (j1 < n[1]) {
            v = __ldg(Q + 2 * (size_t)g[1] + j1);
            a = x[1];
        }
    } else if (na == 3) {
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
    }
}

// Row r with its fetched product (v, a): one entry — the scaled row of B is
// the row of C (sorted, no duplicates); two — five bitonic merge steps;
// three — the full sorting network; more entries (rows of B that are empty
// among them) — the products expanded here, round by round, then sorted.
__device__ __forceinline__ void tiny_process(const NumParams& p, const int2* __restrict__ Q, const TinyRow& r,
                                             int2 v, float a, unsigned long long* err) {
    const int lane = lane_id();
    const unsigned W = (unsigned)p.W;
    const long long na = r.a1 - r.a0;
    int key = 0x7FFFFFFF;  // no product: sorts last
    float val = 0.0f;
    if (na <= TINY_ENT) {
        if ((unsigned)v.x < W) {  // pads and bad columns (-1) add nothing
            key = v.x;
            val = a * __int_as_float(v.y);
        }
        if (na == 1) {
            tiny_emit(p, key, val, false, 1, r.out, r.out_end, err);
        } else if (na == 2) {
#pragma unroll
            for (int j = 16; j > 0; j >>= 1) {
                const int pk = __shfl_xor_sync(FULL, key, j);
                const float pv = __shfl_xor_sync(FULL, val, j);
                if (((lane & j) == 0) ? pk < key : pk > key) {
                    key = pk;
                    val = pv;
                }
            }
            tiny_emit(p, key, val, true, 2, r.out, r.out_end, err);
        } else {
            warp_sort_kv(key, val);
            tiny_emit(p, key, val, true, 4, r.out, r.out_end, err);
        }
        return;
    }
    int base = 0;  // products placed so far (warp-uniform)
    for (long long ec = r.a0; ec < r.a1 && base < 32; ec += 32) {
        const long long e = ec + lane;
        int len = 0;
        long long s = 0;
        unsigned g0 = 0;
        float x = 0.0f;
        if (e < r.a1) {
            const int k = __ldg(p.Ai + e);
            x = p.Ax ? __ldg(p.Ax + e) : 1.0f;
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
        const float aq = __shfl_sync(FULL, x, q);
        if (pj >= 0 && pj < tot) {
            const int2 w = __ldg(Q + 2 * (size_t)gq + (pj - eq));
            if ((unsigned)w.x < W) {
                key = w.x;
                val = aq * __int_as_float(w.y);
            }
        }
        base += tot;
    }
    warp_sort_kv(key, val);
    tiny_emit(p, key, val, true, 32, r.out, r.out_end, err);
}

// Every light row with 1 .. TINY_MAX products (split rows carry negative
// marks in the flops array and are never tiny; with a heavy threshold that
// low, heavy rows stay with the other kernels' blocks), 32-row chunks dealt
// to the warps in turn.  Lane l loads what row l of the chunk needs before
// its rows of B (bounds in A and C, up to TINY_ENT entries of A and their
// rows' descriptions), all rows of the chunk at once; then the chunk's tiny
// rows go through a two-stage pipeline: the next row's gathers are issued
// before the current row is sorted and written.
__global__ void __launch_bounds__(256, 4) k_numeric_tiny(NumParams p) {
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
        // row of chunk lane src, and this lane's product of it
        auto take = [&](int src, TinyRow& t, int2& v, float& a) {
            t.a0 = shfl64(a0, src);
            t.a1 = shfl64(a1, src);
            t.out = shfl64(o0, src);
            t.out_end = shfl64(o1, src);
            unsigned g[TINY_ENT];
            int n[TINY_ENT];
            float x[TINY_ENT];
#pragma unroll
            for (int u = 0; u < TINY_ENT; ++u) {
                g[u] = __shfl_sync(FULL, gl[u], src);
                n[u] = __shfl_sync(FULL, nl[u], src);
                x[u] = __shfl_sync(FULL, xl[u], src);
            }
            tiny_fetch(Q, (int)(t.a1 - t.a0), g, n, x, v, a);
        };
        unsigned rows = __ballot_sync(FULL, tiny);
        if (!rows) continue;
        TinyRow cur;
        int2 v;
        float a;
        take(__ffs(rows) - 1, cur, v, a);
        rows &= rows - 1;
        for (;;) {
            const bool more = rows != 0;  // warp-uniform
            TinyRow nxt{0, 0, 0, 0};
            int2 nv = make_int2(-1, 0);
            float nx = 0.0f;
            if (more) {
                take(__ffs(rows) - 1, nxt, nv, nx);
                rows &= rows - 1;
            }
            tiny_process(p, Q, cur, v, a, err);
            if (!more) break;
            cur = nxt;
            v = nv;
            a = nx;
        }
    }
}

// p.Bq must be the row-aligned copy in pairs (E = 2: rows start at even
// entries), as the wide kernel and the row-group kernels of eight or more
// lanes use it.
cudaError_t launch_numeric_tiny(const NumParams& p, int sms, cudaStream_t st) {
    if (p.nB == 0 || !p.Bq) return cudaSuccess;
    const int grid = persistent_grid((const void*)k_numeric_tiny, 256, 0, sms);
    count_launch();
    k_numeric_tiny<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace ts
