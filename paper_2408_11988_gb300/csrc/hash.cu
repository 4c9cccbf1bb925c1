// Numeric pass with a hash accumulator (paper Sec. III-C: for large d the
// dense SPA spills, so a hash table accumulates each output row).
//
// A warp owns a table of S slots (int32 key, float value; linear probing,
// multiplicative hashing) and a bitmap of d bits.  Every product inserts its
// column into the table (adding the value) and sets the column's bit.  The
// bitmap, read word by word with a warp scan of popcounts, yields the row's
// columns in ascending order; each column's value is then looked up in the
// table and its slot is cleared.  Heavy rows (the CTA schedule) use one table
// of (warps * S) slots and one bitmap for the whole block.  Rows whose
// distinct columns do not fit raise ERR_HASH_FULL instead of being dropped
// silently.  A block row with more distinct columns than the block table
// holds at 75% load (known beforehand from C's row pointers) runs in column
// windows: one walk over its products marks the bitmap only, then for each
// run of bitmap words whose columns fit the table, a walk inserts only the
// columns of that window and the window is read out before the next one.
#include "common.cuh"
#include "kernels.h"

namespace ts {

struct HashParams {
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
    int dw;
    int S;  // slots per warp (power of two)
    const int* perm;
    WsHeader* hdr;
    int cta_class;
    const long long* Cp;
    int* Ci;
    float* Cx;
    long long nnzC;
};

__device__ __forceinline__ unsigned hash_slot(int c, unsigned mask) {
    return ((unsigned)c * 2654435761u) & mask;
}

template <bool VALUES>
struct HashVisit {
    const int* __restrict__ Bi;
    const float* __restrict__ Bx;
    int* keys;
    float* vals;
    unsigned* bm;
    unsigned mask;
    int d;
    unsigned long long* err;
    // 0: bitmap and table; 1: bitmap only; 2: table only, columns [lo, hi)
    int mode = 0, lo = 0, hi = 0;
    __device__ __forceinline__ void insert(int c, float v) {
        if ((unsigned)c >= (unsigned)d) {
            if (mode != 2) atomicOr(err, ERR_B_COL);
            return;
        }
        if (mode == 2) {
            if (c < lo || c >= hi) return;
        } else {
            atomicOr(bm + (c >> 5), 1u << (c & 31));
        }
        if (!VALUES || mode == 1) return;
        unsigned h = hash_slot(c, mask);
        for (unsigned probe = 0; probe <= mask; ++probe) {
            const int k = atomicCAS(keys + h, -1, c);
            if (k == -1 || k == c) {
                atomicAdd(vals + h, v);
                return;
            }
            h = (h + 1) & mask;
        }
        atomicOr(err, ERR_HASH_FULL);
    }
    __device__ __forceinline__ void step4(const long long* j, const float* a, const int*) {
        int c[4];
        float b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = __ldg(Bi + j[u]);
            b[u] = VALUES ? __ldg(Bx + j[u]) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) insert(c[u], a[u] * b[u]);
    }
    __device__ __forceinline__ void step1(long long j, float a, int, bool ok) {
        if (ok) insert(__ldg(Bi + j), VALUES ? a * __ldg(Bx + j) : 0.0f);
    }
};

// Value of column c in the table (read only: slots are reset after the whole
// row is read out, because clearing a slot during lookups would cut the
// probe chains of other columns).
__device__ __forceinline__ float find_slot(const int* keys, const float* vals, unsigned mask, int c,
                                           bool& found) {
    unsigned h = hash_slot(c, mask);
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const int k = keys[h];
        if (k == c) {
            found = true;
            return vals[h];
        }
        if (k == -1) break;
        h = (h + 1) & mask;
    }
    found = false;
    return 0.0f;
}

// Read out the row's columns in ascending order.  With CTA, all warps of the
// block cooperate word-range by word-range (each warp takes a contiguous
// range of bitmap words; ranges are ordered by a block scan).
template <bool VALUES, bool CTA>
__device__ __forceinline__ void hash_emit(int* keys, float* vals, unsigned* bm, unsigned mask, int w0, int w1,
                                          long long out, long long out_end, int* Ci, float* Cx,
                                          int* s_warp_tot, unsigned long long* err) {
    const int lane = lane_id();
    const int nw = CTA ? (blockDim.x >> 5) : 1;
    const int w = CTA ? warp_id() : 0;
    const int per = (w1 - w0 + nw - 1) / nw;
    const int wb = w0 + w * per < w1 ? w0 + w * per : w1, we = wb + per < w1 ? wb + per : w1;
    // count of this warp's range
    long long base = out;
    if (CTA) {
        int cnt = 0;
        for (int x = wb + lane; x < we; x += 32) cnt += __popc(bm[x]);
        cnt = warp_sum(cnt);
        if (lane == 0) s_warp_tot[w] = cnt;
        __syncthreads();
        if (w == 0) {
            const int tot = warp_excl_scan_smem(s_warp_tot, nw);
            (void)tot;
        }
        __syncthreads();
        base = out + s_warp_tot[w];
    }
    for (int x0 = wb; x0 < we; x0 += 32) {
        const int x = x0 + lane;
        unsigned word = x < we ? bm[x] : 0u;
        const int c = __popc(word);
        const int inc = warp_incl_scan(c);
        long long pos = base + inc - c;
        base += __shfl_sync(FULL, inc, 31);
        if (x < we) bm[x] = 0u;
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            const int col = x * 32 + b;
            float v = 0.0f;
            bool found = true;
            if (VALUES) v = find_slot(keys, vals, mask, col, found);
            if (!found) atomicOr(err, ERR_HASH_FULL);
            if (pos < out_end) {
                Ci[pos] = col;
                if (VALUES) Cx[pos] = v;
            } else {
                atomicOr(err, ERR_C_ROW);
            }
            ++pos;
        }
    }
    if (CTA) __syncthreads();
    else __syncwarp();
    if (VALUES) {
        const int t0 = CTA ? threadIdx.x : lane, nt = CTA ? blockDim.x : 32;
        for (unsigned i = t0; i <= mask; i += nt) {
            keys[i] = -1;
            vals[i] = 0.0f;
        }
        if (CTA) __syncthreads();
        else __syncwarp();
    }
}

// The products of entries [a0, a1) of A through visitor vis (the block's
// warps take 32-entry chunks in turn).
template <bool VALUES, bool CTA>
__device__ __forceinline__ void hash_walk(const HashParams& p, long long a0, long long a1, HashVisit<VALUES>& vis,
                                          unsigned long long* err) {
    const int nw = blockDim.x >> 5;
    const long long first = CTA ? a0 + 32LL * warp_id() : a0;
    const long long stride = CTA ? 32LL * nw : 32LL;
    const SegWhole seg{p.Bp, p.nnzB, p.d};
    for (long long e0 = first; e0 < a1; e0 += stride)
        expand_chunk(e0, (int)(a1 - e0 < 32 ? a1 - e0 : 32), p.Ai, VALUES ? p.Ax : nullptr, p.nB, seg,
                     vis, err);
}

// A block row wider than the table (see the top of the file): bitmap walk,
// then per window of bitmap words holding at most `cap` columns a table walk
// restricted to the window and its read-out.  s_win[0..1]: window end and
// its column count, chosen by warp 0.
template <bool VALUES>
__device__ __noinline__ void hash_row_windows(const HashParams& p, long long a0, long long a1, long long out,
                                              long long out_end, int* keys, float* vals, unsigned* bm,
                                              unsigned mask, int* s_warp_tot, int* s_win) {
    unsigned long long* err = &p.hdr->err;
    const unsigned cap = (mask + 1) - (mask + 1) / 4;  // >= 48 columns, more than one word
    HashVisit<VALUES> vis{p.Bi, p.Bx, keys, vals, bm, mask, p.d, err};
    vis.mode = 1;
    hash_walk<VALUES, true>(p, a0, a1, vis, err);
    __syncthreads();
    const int lane = lane_id();
    long long pos = out;
    for (int wlo = 0; wlo < p.dw;) {
        if (warp_id() == 0) {
            int whi = wlo;
            unsigned tot = 0;
            for (;;) {  // extend the window 32 words at a time while its columns fit
                const int x = whi + lane;
                const unsigned c = x < p.dw ? (unsigned)__popc(bm[x]) : 0u;
                const unsigned inc = (unsigned)warp_incl_scan((int)c);
                // inc grows with the lane, so the lanes that fit form a prefix
                const unsigned fit = __ballot_sync(FULL, x < p.dw && tot + inc <= cap);
                const int nfit = __popc(fit);
                if (nfit > 0) tot += __shfl_sync(FULL, inc, nfit - 1);
                whi += nfit;
                if (nfit < 32 || whi >= p.dw) break;
            }
            if (lane == 0) {
                s_win[0] = whi;
                s_win[1] = (int)tot;
            }
        }
        __syncthreads();
        const int whi = s_win[0], cnt = s_win[1];
        vis.mode = 2;
        vis.lo = 32 * wlo;
        vis.hi = 32 * whi;
        hash_walk<VALUES, true>(p, a0, a1, vis, err);
        __syncthreads();  // (also: every thread has read s_win before warp 0 rewrites it)
        hash_emit<VALUES, true>(keys, vals, bm, mask, wlo, whi, pos, out_end, p.Ci, p.Cx, s_warp_tot, err);
        pos += cnt;
        wlo = whi;
    }
    if (threadIdx.x == 0 && pos != out_end) atomicOr(err, ERR_C_ROW);
}

template <bool VALUES, bool CTA>
__device__ __forceinline__ void hash_row(const HashParams& p, int row, int* keys, float* vals, unsigned* bm,
                                         unsigned mask, int* s_warp_tot, int* s_win) {
    unsigned long long* err = &p.hdr->err;
    const long long a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
    const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
    const long long out = clampll(__ldg(p.Cp + row), 0, p.nnzC);
    const long long out_end = clampll(__ldg(p.Cp + row + 1), out, p.nnzC);
    if (VALUES && out_end - out > (long long)(mask + 1) - (long long)(mask + 1) / 4) {
        // more distinct columns than the table holds at 75% load: a block
        // row runs in column windows; a warp row never gets here (warps take
        // only rows with fewer products than 3/4 of their table)
        if (CTA) {
            hash_row_windows<VALUES>(p, a0, a1, out, out_end, keys, vals, bm, mask, s_warp_tot, s_win);
        } else if (lane_id() == 0) {
            atomicOr(err, ERR_HASH_FULL);
        }
        return;
    }
    HashVisit<VALUES> vis{p.Bi, p.Bx, keys, vals, bm, mask, p.d, err};
    hash_walk<VALUES, CTA>(p, a0, a1, vis, err);
    if (CTA) __syncthreads();
    else __syncwarp();
    hash_emit<VALUES, CTA>(keys, vals, bm, mask, 0, p.dw, out, out_end, p.Ci, p.Cx, s_warp_tot, err);
}

template <bool VALUES>
__global__ void __launch_bounds__(1024) k_numeric_hash(HashParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item, s_nheavy, s_nrows;
    __shared__ int s_warp_tot[33];
    __shared__ int s_win[2];
    const int nw = blockDim.x >> 5, warp = warp_id(), tid = threadIdx.x;
    // layout: keys [nw*S] int, vals [nw*S] float, bitmaps [nw*dw] unsigned
    const int totS = nw * p.S;
    int* keys = (int*)smem;
    float* vals = (float*)(smem + sizeof(int) * (size_t)totS);
    unsigned* bms = (unsigned*)(smem + 2 * sizeof(int) * (size_t)totS);
    for (int i = tid; i < totS; i += blockDim.x) {
        keys[i] = -1;
        vals[i] = 0.0f;
    }
    for (int i = tid; i < nw * p.dw; i += blockDim.x) bms[i] = 0u;
    if (tid < 32) {  // one warp; its lanes store the same values
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
        s_nrows = nr;
    }
    __syncthreads();
    const long long nheavy = s_nheavy, nrows = s_nrows;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&p.hdr->heavy_ctr, 1ull);
        __syncthreads();
        const long long h = s_item;
        __syncthreads();
        if (h >= nheavy) break;
        hash_row<VALUES, true>(p, p.perm[h], keys, vals, bms, (unsigned)(totS - 1), s_warp_tot, s_win);
    }
    int* wk = keys + warp * p.S;
    float* wv = vals + warp * p.S;
    unsigned* wb = bms + warp * p.dw;
    for (long long idx = nheavy + (long long)blockIdx.x * nw + warp; idx < nrows;
         idx += (long long)gridDim.x * nw)
        hash_row<VALUES, false>(p, p.perm[idx], wk, wv, wb, (unsigned)(p.S - 1), nullptr, nullptr);
}

size_t numeric_hash_smem(int slots, int warps, bool values) {
    (void)values;
    return (size_t)warps * (size_t)slots * 8;  // bitmap added by the launcher
}

cudaError_t launch_numeric_hash(const DevCsr& A, const DevCsr& B, long long d, int slots, bool values,
                                const Sched& s, const LaunchCfg& cfg, const long long* Cp, int* Ci,
                                float* Cx, long long nnzC, cudaStream_t st) {
    cudaError_t e;
    if (A.nrows == 0) return cudaSuccess;
    int warps = cfg.warps_per_cta;
    // CTA tables must be a power of two: round the warp count down to one
    while (warps & (warps - 1)) --warps;
    const int dw = (int)((d + 31) / 32);
    size_t smem = (size_t)warps * ((size_t)slots * 8 + (size_t)dw * 4);
    while (smem > 200 * 1024 && warps > 1) {
        warps /= 2;
        smem = (size_t)warps * ((size_t)slots * 8 + (size_t)dw * 4);
    }
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(&s.hdr->heavy_ctr, 0, 2 * sizeof(unsigned long long), st))) return e;
    HashParams p;
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
    p.dw = dw;
    p.S = slots;
    p.perm = s.perm;
    p.hdr = s.hdr;
    // warp tables hold 3/4 * slots columns: rows with more products go to the block table
    int cc = cfg.cta_class;
    const int lim = flops_class_host((long long)slots * 3 / 4 + 1);  // warp rows: flops <= 0.75 S
    if (cc > lim) cc = lim;
    p.cta_class = cc;
    p.Cp = Cp;
    p.Ci = Ci;
    p.Cx = Cx;
    p.nnzC = nnzC;
    const void* k = values ? (const void*)k_numeric_hash<true> : (const void*)k_numeric_hash<false>;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    const int grid = persistent_grid(k, 32 * warps, smem, cfg.sms);
    if (values) {
        count_launch();
        k_numeric_hash<true><<<grid, 32 * warps, smem, st>>>(p);
    }
    else {
        count_launch();
        k_numeric_hash<false><<<grid, 32 * warps, smem, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace ts
