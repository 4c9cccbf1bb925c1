// Device pieces of the wide numeric kernels, shared by the single-product
// pass (numeric.cu) and the batched kernels (batched.cu): the row-aligned
// packed copy of B, a shared accumulator with occupancy bits, the walk of a
// chunk of A's entries over it and the read-out of its occupied columns.
#pragma once

#include "common.cuh"
#include "numeric.cuh"

namespace ts {

// ---------------------------------------------------------------------------
// Row-aligned packed copy of B (one column tile, T = 1).  Row k's entries
// start at entry S(k) = E * ceil((Bp[k] + (E-1) k) / E) of the copy, so every
// row begins a group of E entries (one or two 16-byte loads) and
// S(k) + len_k <= S(k+1) holds without a scan over the row lengths.  The
// last group of a row is completed with pad entries (column -1, value 0),
// and a column outside [0, d) (an input error, reported once by the packing
// kernel) is stored as -1 too.  A slot maps a column c to accumulator index
// min((unsigned)c, W): pads and bad columns land in the spare column W,
// which is never read out, so the gather needs no per-entry segment or
// range test.  Groups are numbered with 32 bits (the host checks the copy's
// size).
// ---------------------------------------------------------------------------
// Row k of B as the copy holds it: its first entry s and length len in B
// (clamped like SegWhole) and its first group g0 in the copy.
template <int E>
__device__ __forceinline__ void padded_row(const long long* __restrict__ Bp, long long nnzB, int d, int k,
                                           long long& s, int& len, unsigned& g0) {
    s = clampll(__ldg(Bp + k), 0, nnzB);
    const long long e = clampll(__ldg(Bp + k + 1), s, nnzB);
    len = (int)(e - s < d ? e - s : d);
    g0 = (unsigned)((s + (long long)(E - 1) * k + (E - 1)) / E);
}

template <int E>
__device__ __forceinline__ void padded_seg(const long long* __restrict__ Bp, long long nnzB, int d, int k,
                                           unsigned& g0, int& ng) {
    long long s;
    int len;
    padded_row<E>(Bp, nnzB, d, k, s, len, g0);
    ng = (len + E - 1) / E;
}

// One accumulator shared by several slots (the wide kernels): pads are
// skipped, the value is added with a shared-memory float atomic and the
// column's occupancy bit is set.
struct AddShared {
    float* acc;
    unsigned* bm;
    __device__ __forceinline__ void operator()(int c, unsigned W, float v) const {
        if ((unsigned)c < W) {
            atomicAdd(acc + c, v);
            atomicOr(bm + (c >> 5), 1u << (c & 31));
        }
    }
};


// Marks only (the symbolic count of a row): the column's occupancy bit.
struct AddMark {
    unsigned* bm;
    __device__ __forceinline__ void operator()(int c, unsigned W, float) const {
        if ((unsigned)c < W) atomicOr(bm + (c >> 5), 1u << (c & 31));
    }
};

// ---------------------------------------------------------------------------
// Wide rows (plus-times, one column tile of 256 < W <= 1024 columns: for
// d = 1024 the four 256-column tiles of B side by side, so that A is walked
// once instead of once per tile).  Private accumulators of W floats per row
// group would leave too few rows in flight per SM, and reading a W-wide
// accumulator out costs W/32 steps per row although a row of C holds only
// a few dozen of its W columns.  Here a team -- one warp for a light row,
// the whole block for a heavy row or a part of a split row -- owns ONE
// accumulator of W floats and a bitmap of W/32 occupancy words.  The team's
// slots of 8 lanes take contiguous shares of the item's entries of A and
// walk their segments of B on the row-aligned copy as the row-group kernels
// do (pairs of entries per lane, next segment in flight), but all add into
// the shared accumulator: a shared-memory float reduction for the value and
// an OR of the column's bit.  The read-out visits the occupied columns only:
// output positions are dealt to the lanes 32 at a time, so every store
// writes 32 consecutive entries of C, and lane l finds the column of rank j
// by a search over the words' running counts and a select inside the word.
// ---------------------------------------------------------------------------

// Position of the k-th (0-based) set bit of x (k < popc(x)): binary search
// over halves, quarters, ... of the word by population counts.
__device__ __forceinline__ int select_bit(unsigned x, int k) {
    int pos = 0;
    int c = __popc(x & 0xFFFFu);
    if (k >= c) { k -= c; x >>= 16; pos += 16; }
    c = __popc(x & 0xFFu);
    if (k >= c) { k -= c; x >>= 8; pos += 8; }
    c = __popc(x & 0xFu);
    if (k >= c) { k -= c; x >>= 4; pos += 4; }
    c = __popc(x & 0x3u);
    if (k >= c) { k -= c; x >>= 2; pos += 2; }
    if (k >= (int)(x & 1u)) pos += 1;
    return pos;
}

// Read-out of a shared accumulator acc[0..32*nw) with bitmap bm[0..nw)
// (nw <= 32) into C[out, out_end): positions 32*r + lane for rounds
// r = r0, r0 + rstep, ... (a block team splits the rounds over its warps);
// every emitted column of acc is reset to 0.  Returns the row's count.
// Called with all 32 lanes converged; the caller clears the bitmap after
// every warp of the team has passed.
__device__ __forceinline__ int wide_emit(float* acc, const unsigned* bm, int nw, long long out, long long out_end,
                                         int* Ci, float* Cx, int r0, int rstep, unsigned long long* err) {
    const int lane = lane_id();
    const unsigned word = lane < nw ? bm[lane] : 0u;
    const int cnt = __popc(word);
    const int incl = warp_incl_scan(cnt);
    const int total = __shfl_sync(FULL, incl, 31);
    const long long r = out_end - out;
    const int room = r < (long long)total ? (int)r : total;
    bool over = false;
    for (int base = 32 * r0; base < total; base += 32 * rstep) {
        const int j = base + lane;
        // word of rank j: the number of words whose running count is <= j
        int w = 0;
#pragma unroll
        for (int st = 16; st >= 1; st >>= 1)
            if (__shfl_sync(FULL, incl, w + st - 1) <= j) w += st;
        const unsigned x = __shfl_sync(FULL, word, w);
        const int before = __shfl_sync(FULL, incl - cnt, w);
        if (j < total) {
            const int c = 32 * w + select_bit(x, j - before);
            const float v = acc[c];
            acc[c] = 0.0f;
            if (j < room) {
                Ci[out + j] = c;
                if (Cx) Cx[out + j] = v;
            } else {
                over = true;
            }
        }
    }
    if (over) atomicOr(err, ERR_C_ROW);
    return total;
}

// Segments of one chunk of up to 32 entries of A (lane l: entry l, its
// segment of B in the row-aligned copy as first pair g0 and pairs np, and
// A's value a; np = 0 past the chunk) added into the shared accumulator.
// Groups of four lanes take one segment each, lane gl its pairs gl, gl + 4,
// ...; two steps of eight segments are in flight at once (up to four
// 16-byte loads per lane before any is used).
template <class Add>
__device__ __forceinline__ void wide_chunk_walk(const int4* __restrict__ Q, const Add& add, unsigned W,
                                                unsigned g0, int np, float a, int nvalid) {
    const int lane = lane_id(), grp = lane >> 2, gl = lane & 3;
    for (int s0 = 0; s0 < nvalid; s0 += 16) {
        const int ea = s0 + grp, eb = s0 + 8 + grp;
        const unsigned ga = __shfl_sync(FULL, g0, ea & 31), gb = __shfl_sync(FULL, g0, eb & 31);
        int na = __shfl_sync(FULL, np, ea & 31), nb = __shfl_sync(FULL, np, eb & 31);
        const float xa = __shfl_sync(FULL, a, ea & 31), xb = __shfl_sync(FULL, a, eb & 31);
        if (ea >= nvalid) na = 0;
        if (eb >= nvalid) nb = 0;
        int4 u0 = make_int4(-1, 0, -1, 0), u1 = u0, v0 = u0, v1 = u0;
        if (gl < na) u0 = __ldg(Q + ga + gl);
        if (gl < nb) v0 = __ldg(Q + gb + gl);
        if (gl + 4 < na) u1 = __ldg(Q + ga + gl + 4);
        if (gl + 4 < nb) v1 = __ldg(Q + gb + gl + 4);
        add(u0.x, W, xa * __int_as_float(u0.y));
        add(u0.z, W, xa * __int_as_float(u0.w));
        add(v0.x, W, xb * __int_as_float(v0.y));
        add(v0.z, W, xb * __int_as_float(v0.w));
        add(u1.x, W, xa * __int_as_float(u1.y));
        add(u1.z, W, xa * __int_as_float(u1.w));
        add(v1.x, W, xb * __int_as_float(v1.y));
        add(v1.z, W, xb * __int_as_float(v1.w));
        // rows of B longer than 16 entries
        for (int q = gl + 8; q < na; q += 4) {
            const int4 w = __ldg(Q + ga + q);
            add(w.x, W, xa * __int_as_float(w.y));
            add(w.z, W, xa * __int_as_float(w.w));
        }
        for (int q = gl + 8; q < nb; q += 4) {
            const int4 w = __ldg(Q + gb + q);
            add(w.x, W, xb * __int_as_float(w.y));
            add(w.z, W, xb * __int_as_float(w.w));
        }
    }
}

// Entry e of A for this lane (ok: inside the chunk): its column k (-1 if
// none) and value a.
__device__ __forceinline__ void wide_load_a(const NumParams& p, long long e, bool ok, int& k, float& a) {
    k = -1;
    a = 0.0f;
    if (ok) {
        k = __ldg(p.Ai + e);
        a = p.Ax ? __ldg(p.Ax + e) : 1.0f;
    }
}

// Segment (first pair, pairs) of B's row k in the row-aligned copy (none
// for k = -1; a column of A outside [0, n) is an input error).
__device__ __forceinline__ void wide_seg(const NumParams& p, int k, unsigned& g0, int& np, unsigned long long* err) {
    g0 = 0;
    np = 0;
    if (k < 0) return;
    if (k < p.nB) padded_seg<2>(p.Bp, p.nnzB, p.d, k, g0, np);
    else atomicOr(err, ERR_A_COL);
}

// The default stop test of wide_range: walk every chunk.
struct NeverFull {
    __device__ __forceinline__ bool operator()() const { return false; }
};

// Chunks first, first + stride, ... (< e1) of 32 entries of A walked by
// one warp into the shared accumulator, in three stages: while chunk c is
// walked, the row pointers of B for chunk c + 1 and the entries of A of
// chunk c + 2 are in flight.  After each chunk the warp-uniform test full()
// may end the walk (a symbolic row whose marks hold every column).
template <class Add, class Full = NeverFull>
__device__ __forceinline__ void wide_range(const NumParams& p, const Add& add, long long first, long long e1,
                                           long long stride, unsigned long long* err, const Full& full = Full()) {
    const int lane = lane_id();
    const unsigned W = (unsigned)p.W;
    int k;
    float a;
    wide_load_a(p, first + lane, first + lane < e1, k, a);
    unsigned g0;
    int np;
    wide_seg(p, k, g0, np, err);
    float ca = a;
    wide_load_a(p, first + stride + lane, first + stride + lane < e1, k, a);
    for (long long e = first; e < e1; e += stride) {
        const int nv = e1 - e < 32 ? (int)(e1 - e) : 32;
        unsigned g1;
        int np1;
        wide_seg(p, k, g1, np1, err);  // chunk c + 1
        const float ca1 = a;
        const long long e2 = e + 2 * stride;
        wide_load_a(p, e2 + lane, e2 + lane < e1, k, a);  // chunk c + 2
        wide_chunk_walk(p.Bq, add, W, g0, np, ca, nv);
        if (full()) break;
        g0 = g1;
        np = np1;
        ca = ca1;
    }
}

}  // namespace ts
