// Device building blocks of the TS-SpGEMM kernels (sm_103a).
//
// The product is row-wise Gustavson (paper Sec. III-A, Eq. 1): row i of C is
// the semiring sum over the stored (i,k) of A(i,k) * B(k,:).  On the GPU a row
// is processed by one warp (light rows) or one thread block (heavy rows); the
// products of up to 32 entries of A are flattened across the 32 lanes so that
// every lane handles one (k, j) pair per step regardless of how the rows of B
// vary in length.  Accumulators live in shared memory (paper Sec. III-C: a
// dense accumulator of width d, "SPA", or a hash table).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "kernels.h"
#include "layout.h"

namespace ts {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Row class of f products (layout.h: eighths of an octave).
__device__ __forceinline__ int flops_class(long long f) {
    if (f <= 0) return 0;
    const int lg = 63 - __clzll(f);
    const int sub = lg >= CLASS_SUB_BITS ? (int)((f >> (lg - CLASS_SUB_BITS)) & ((1 << CLASS_SUB_BITS) - 1))
                                         : (int)((f << (CLASS_SUB_BITS - lg)) & ((1 << CLASS_SUB_BITS) - 1));
    const int c = 1 + (lg << CLASS_SUB_BITS) + sub;
    return c < NUM_CLASSES ? c : NUM_CLASSES - 1;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Largest lane q whose (non-decreasing) key is <= p.  Lane 0's key must be <= p.
__device__ __forceinline__ int owner_lane(int key, int p) {
    int q = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        int k = __shfl_sync(FULL, key, q + s);
        if (k <= p) q += s;
    }
    return q;
}

__device__ __forceinline__ long long shfl64(long long v, int src) {
    return (long long)__shfl_sync(FULL, (unsigned long long)v, src);
}

__device__ __forceinline__ long long shfl64_down(long long v, int delta) {
    return (long long)__shfl_down_sync(FULL, (unsigned long long)v, delta);
}

// owner_lane for 64-bit keys.
__device__ __forceinline__ int owner_lane64(long long key, long long p) {
    int q = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        long long k = shfl64(key, q + s);
        if (k <= p) q += s;
    }
    return q;
}

// Ask L2 for the line holding p (no register, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// L2 prefetch of the packed entries [s, s + L) of B (two 128-byte lines
// cover a segment of up to 16 entries).
__device__ __forceinline__ void prefetch_segment(const int2* P, long long s, int L) {
    if (L <= 0) return;
    prefetch_l2(P + s);
    if (L > 8) prefetch_l2(P + s + 16);
}

__device__ __forceinline__ long long clampll(long long v, long long lo, long long hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

// Segment of B's row k that a pass reads: the whole row, or the part of the
// row inside one column tile (tile_ptr holds T+1 offsets per row of B).
// Segments are clamped to [0, nnzB) and to at most `cap` entries (a row of
// B holds at most d distinct columns), so even a malformed row pointer array
// cannot move a gather outside B's arrays.
struct SegWhole {
    const long long* __restrict__ Bp;
    long long nnzB;
    int cap;
    __device__ __forceinline__ void operator()(int k, long long& start, int& len) const {
        long long s = __ldg(Bp + k), e = __ldg(Bp + k + 1);
        s = s < 0 ? 0 : (s > nnzB ? nnzB : s);
        e = e < s ? s : (e > nnzB ? nnzB : e);
        start = s;
        len = (int)(e - s < cap ? e - s : cap);
    }
};

struct SegTile {
    const long long* __restrict__ tp;  // [nB][T+1], already clamped to [0, nnzB]
    int T1;                            // T + 1
    int t;
    int cap;
    __device__ __forceinline__ void operator()(int k, long long& start, int& len) const {
        const long long* r = tp + (long long)k * T1 + t;
        long long s = __ldg(r), e = __ldg(r + 1);
        start = s;
        len = (int)(e > s ? (e - s < cap ? e - s : cap) : 0);
    }
};

// Per-lane view of one chunk of up to 32 entries of A: lane l holds entry
// e0 + l (if l < nvalid): the start and length of its segment of B and its
// value a (1 when A has no values).
struct Chunk {
    long long start;
    int len;
    float a;
};

template <class Seg>
__device__ __forceinline__ Chunk load_chunk(long long e0, int nvalid, const int* __restrict__ Ai,
                                            const float* __restrict__ Ax, int nB, const Seg& seg,
                                            unsigned long long* err) {
    const int lane = lane_id();
    Chunk c{0, 0, 1.0f};
    if (lane < nvalid) {
        const int k = __ldg(Ai + e0 + lane);
        if ((unsigned)k < (unsigned)nB) {
            seg(k, c.start, c.len);
            if (Ax) c.a = __ldg(Ax + e0 + lane);
        } else {
            atomicOr(err, ERR_A_COL);
        }
    }
    return c;
}

// Flattened expansion of a loaded chunk: the products (entry q, position j in
// q's segment of B) are numbered across the 32 entries and lane l takes
// numbers l, l+32, ...; visit.step4/step1(j, a_q, q[, ok]) are called with all
// lanes converged (ok is false for padding lanes).  Steps are issued four at
// a time where possible so that every lane has several gathers in flight.
template <class Visit>
__device__ __forceinline__ void expand_loaded(const Chunk& ch, Visit& visit) {
    const int lane = lane_id();
    const int incl = warp_incl_scan(ch.len);
    const int total = __shfl_sync(FULL, incl, 31);
    const int excl = incl - ch.len;
    const long long shift = ch.start - excl;  // position in B = shift(owner) + p
    int p0 = 0;
    for (; p0 + 128 <= total; p0 += 128) {
        long long j[4];
        float av[4];
        int q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = p0 + 32 * u + lane;
            q[u] = owner_lane(excl, p);
            j[u] = shfl64(shift, q[u]) + p;
            av[u] = __shfl_sync(FULL, ch.a, q[u]);
        }
        visit.step4(j, av, q);
    }
    for (; p0 < total; p0 += 32) {
        const int p = p0 + lane;
        const int q = owner_lane(excl, p);
        const long long j = shfl64(shift, q) + p;
        const float av = __shfl_sync(FULL, ch.a, q);
        visit.step1(j, av, q, p < total);
    }
}

template <class Seg, class Visit>
__device__ __forceinline__ void expand_chunk(long long e0, int nvalid, const int* __restrict__ Ai,
                                             const float* __restrict__ Ax, int nB, const Seg& seg,
                                             Visit& visit, unsigned long long* err) {
    const Chunk ch = load_chunk(e0, nvalid, Ai, Ax, nB, seg, err);
    expand_loaded(ch, visit);
}

// B's entries either as the caller's two arrays or as (column, value bits)
// pairs packed into 8 bytes (one load per product).
struct BSep {
    const int* __restrict__ Bi;
    const float* __restrict__ Bx;
    __device__ __forceinline__ int col(long long j) const { return __ldg(Bi + j); }
    __device__ __forceinline__ void get(long long j, int& c, float& b) const {
        c = __ldg(Bi + j);
        b = Bx ? __ldg(Bx + j) : 0.0f;
    }
};

struct BPacked {
    const int2* __restrict__ P;
    __device__ __forceinline__ int col(long long j) const { return __ldg(&P[j].x); }
    __device__ __forceinline__ void get(long long j, int& c, float& b) const {
        const int2 v = __ldg(P + j);
        c = v.x;
        b = __int_as_float(v.y);
    }
};

// Group distribution of the products of one chunk of up to 32 A entries:
// lanes form 32/G groups of G lanes; a group takes one A entry q and walks
// its segment of B with stride G.  Two entries per group are in flight per
// pass (slots 0 and 1) so that each lane has two independent gathers
// outstanding.  `op` provides fetch(j) -> Item, apply(item, a_q, j, slot) and
// done<G>(q0, q1, nvalid, e0), called once per pass with all 32 lanes
// converged after both entries' segments are complete.
template <int G, class Op>
__device__ __forceinline__ void grouped_loaded(const Chunk& ch, int nvalid, long long e0, Op& op) {
    static_assert(G >= 2 && G <= 32 && (32 % G) == 0, "group size");
    constexpr int NG = 32 / G;
    const int lane = lane_id();
    const int gi = lane / G, gl = lane % G;
    for (int t = 0; t < nvalid; t += 2 * NG) {
        const int q0 = t + gi, q1 = t + NG + gi;  // both <= 31 because 2*NG divides 32
        const long long s0 = shfl64(ch.start, q0), s1 = shfl64(ch.start, q1);
        const int l0 = __shfl_sync(FULL, ch.len, q0), l1 = __shfl_sync(FULL, ch.len, q1);
        const float a0 = __shfl_sync(FULL, ch.a, q0), a1 = __shfl_sync(FULL, ch.a, q1);
        const int lm = l0 > l1 ? l0 : l1;
        for (int r = gl; r < lm; r += G) {
            const bool v0 = r < l0, v1 = r < l1;
            typename Op::Item i0, i1;
            if (v0) i0 = op.fetch(s0 + r);
            if (v1) i1 = op.fetch(s1 + r);
            if (v0) op.apply(i0, a0, s0 + r, 0);
            if (v1) op.apply(i1, a1, s1 + r, 1);
        }
        op.template done<G>(q0, q1, nvalid, e0);
    }
}

template <int G, class Seg, class Op>
__device__ __forceinline__ void grouped_chunk(long long e0, int nvalid, const int* __restrict__ Ai,
                                              const float* __restrict__ Ax, int nB, const Seg& seg,
                                              Op& op, unsigned long long* err) {
    const Chunk ch = load_chunk(e0, nvalid, Ai, Ax, nB, seg, err);
    grouped_loaded<G>(ch, nvalid, e0, op);
}

// Quad distribution of one loaded chunk: a group of four lanes takes one
// entry q and walks its segment [s, s + len) of B in quads of four
// consecutive positions, starting at the multiple of four at or below s;
// lane gl of the group takes quads gl, gl + 4, ...  visit(qb, s, end, a) is
// called once per quad (first position qb); positions outside [s, end) are
// the visitor's to skip.  No lane synchronisation inside.
template <class F>
__device__ __forceinline__ void quads_loaded(const Chunk& ch, int nvalid, F&& visit) {
    const int lane = lane_id(), gi = lane >> 2, gl = lane & 3;
    for (int r = 0; r < nvalid; r += 8) {
        const int q = r + gi;  // <= 31
        const long long s = shfl64(ch.start, q);
        const int L = __shfl_sync(FULL, ch.len, q);
        const float a = __shfl_sync(FULL, ch.a, q);
        const long long base = s & ~3LL, end = s + L;
        const int nq = L > 0 ? (int)((end - base + 3) >> 2) : 0;
        for (int t = gl; t < nq; t += 4) visit(base + 4LL * t, s, end, a);
    }
}

// Products of one chunk in the chosen distribution (G = 1: flattened;
// G = 2: quads, through op.quads).
template <int G, class Op>
__device__ __forceinline__ void expand_any(const Chunk& ch, int nvalid, long long e0, Op& op) {
    if constexpr (G == 2) op.quads(ch, nvalid);
    else if constexpr (G == 1) expand_loaded(ch, op);
    else grouped_loaded<G>(ch, nvalid, e0, op);
}

// A row cut into split work items carries the mark -1 - slot in the flops
// array (only rows with more than SPLIT_ENTRIES entries can be cut).
__device__ __forceinline__ bool is_split_row(const long long* mark, int row, long long alen) {
    return alen > SPLIT_ENTRIES && __ldg(mark + row) < 0;
}

// Software-pipelined walk over the light rows assigned to one warp (rows
// perm[idx0], perm[idx0 + step], ...): while row r is processed, the row
// index, row pointers and first chunk of A of row r+1 are already loaded.
// body.gather(row, a0, a1, chunk0, nvalid0, next_row) gathers one row's
// products (it consumes the first chunk from `chunk0`, loads any further
// chunks itself, and may prefetch for next_row, -1 at the end); then
// body.finish(row) completes the row (read-out), overlapping with the loads
// of the next row's first chunk.
template <class Seg, class Body>
__device__ __forceinline__ void pipelined_rows(const int* __restrict__ perm, long long idx0, long long end,
                                               long long step, const long long* __restrict__ Ap,
                                               long long nnzA, const int* __restrict__ Ai,
                                               const float* __restrict__ Ax, int nB, const Seg& seg,
                                               unsigned long long* err, Body& body,
                                               const long long* split_mark = nullptr) {
    if (idx0 >= end) return;
    int row = __ldg(perm + idx0);
    long long a0 = clampll(__ldg(Ap + row), 0, nnzA);
    long long a1 = clampll(__ldg(Ap + row + 1), a0, nnzA);
    int nv = (int)(a1 - a0 < 32 ? a1 - a0 : 32);
    Chunk ch = load_chunk(a0, nv, Ai, Ax, nB, seg, err);
    for (long long idx = idx0; idx < end; idx += step) {
        // next row's meta data first, so that it is in flight during this row
        const long long nidx = idx + step;
        int nrow = 0;
        long long na0 = 0, na1 = 0;
        if (nidx < end) {
            nrow = __ldg(perm + nidx);
            na0 = clampll(__ldg(Ap + nrow), 0, nnzA);
            na1 = clampll(__ldg(Ap + nrow + 1), na0, nnzA);
        }
        const int nnv = (int)(na1 - na0 < 32 ? na1 - na0 : 32);
        const bool skip = split_mark && is_split_row(split_mark, row, a1 - a0);
        if (!skip) body.gather(row, a0, a1, ch, nv, nidx < end ? nrow : -1);
        // the next row's first chunk is loaded before this row's read-out
        const Chunk nch = load_chunk(na0, nnv, Ai, Ax, nB, seg, err);
        if (!skip) body.finish(row);
        row = nrow;
        a0 = na0;
        a1 = na1;
        nv = nnv;
        ch = nch;
    }
}

// Rows with products: all classes >= 1; heavy: classes >= cta_class.
// Called by all 32 lanes of one warp (every lane gets the counts).
__device__ __forceinline__ void sched_counts(const WsHeader* hdr, int cta_class, long long& nheavy,
                                             long long& nrows) {
    long long nh = 0, nr = 0;
    for (int c = 1 + lane_id(); c < NUM_CLASSES; c += 32) {
        const long long h = hdr->hist[c];
        nr += h;
        if (c >= cta_class) nh += h;
    }
    nheavy = warp_sum(nh);
    nrows = warp_sum(nr);
}

// Fetch the next split item for this block; false when none is left.  On
// true, row/slot/[e0, e1)/nsub describe the item.
struct SplitItem {
    int row;
    int slot;
    long long e0, e1;
    int nsub;
};

__device__ __forceinline__ bool next_split_item(const Sched& s, const long long* __restrict__ Ap, long long nnzA,
                                                long long nitems, long long* s_item, SplitItem& it) {
    if (threadIdx.x == 0) *s_item = (long long)atomicAdd(&s.hdr->item_ctr, 1ull);
    __syncthreads();
    const long long k = *s_item;
    __syncthreads();
    if (k >= nitems) return false;
    const long long code = s.split_items[k];
    it.slot = (int)(code >> 32);
    const long long part = code & 0xFFFFFFFFLL;
    it.row = s.split_rows[it.slot];
    const long long a0 = clampll(__ldg(Ap + it.row), 0, nnzA), a1 = clampll(__ldg(Ap + it.row + 1), a0, nnzA);
    it.nsub = (int)((a1 - a0 + SPLIT_ENTRIES - 1) / SPLIT_ENTRIES);
    it.e0 = a0 + part * SPLIT_ENTRIES;
    it.e1 = it.e0 + SPLIT_ENTRIES < a1 ? it.e0 + SPLIT_ENTRIES : a1;
    return true;
}

// After a block flushed its part of split row `slot` into the staging slot:
// count it and return (to every thread) whether this block was the last.
__device__ __forceinline__ bool split_part_done(const Sched& s, int slot, int nsub, int* s_flag) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *s_flag = (atomicAdd(s.split_done + slot, 1) == nsub - 1) ? 1 : 0;
    __syncthreads();
    const bool last = *s_flag != 0;
    if (last) __threadfence();
    return last;
}

// Exclusive-scan helper for per-word counts held in shared memory by one warp.
// Replaces cnt[0..nw) by exclusive prefix sums; returns the total.
__device__ __forceinline__ int warp_excl_scan_smem(int* cnt, int nw) {
    const int lane = lane_id();
    int carry = 0;
    for (int b = 0; b < nw; b += 32) {
        int v = (b + lane < nw) ? cnt[b + lane] : 0;
        int inc = warp_incl_scan(v);
        if (b + lane < nw) cnt[b + lane] = carry + inc - v;
        carry += __shfl_sync(FULL, inc, 31);
    }
    return carry;
}

}  // namespace ts
