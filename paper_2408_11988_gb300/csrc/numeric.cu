// Numeric pass with a dense accumulator (the paper's SPA, Sec. III-C) of
// width W in shared memory plus one occupancy byte per column.  Row i of C
// (Eq. 1) is produced tile by tile (W columns of B each); inside a tile the
// occupied columns are read out in ascending order, four per lane, which
// also restores the accumulator to zero for the next row.
//
// Products are spread over the lanes in one of two ways (template G):
//   G = 1      flattened: the products of 32 A entries are numbered and lane l
//              takes numbers l, l+32, ... (any mix of B row lengths);
//   G = 4..32  grouped: a group of G lanes takes one A entry and walks its B
//              row with stride G (no per-product owner search; best when B's
//              rows have nearly equal lengths close to G).
// B is read from its two arrays or from a packed (column, value) copy.
#include "common.cuh"
#include "kernels.h"
#include "numeric.cuh"
#include "staged.cuh"
#include "wide.cuh"
#include "rowgroup.cuh"

namespace ts {

template <bool VALUES, class BA>
struct DenseOp {
    BA ba;
    float* acc;
    unsigned char* flg;
    int d;
    int c0;
    int W;
    unsigned long long* err;
    struct Item {
        int c;
        float b;
    };
    __device__ __forceinline__ Item fetch(long long j) const {
        Item it;
        if (VALUES) ba.get(j, it.c, it.b);
        else {
            it.c = ba.col(j);
            it.b = 0.0f;
        }
        return it;
    }
    __device__ __forceinline__ void add(int c, float v) {
        const int lc = c - c0;
        if ((unsigned)c < (unsigned)d && (unsigned)lc < (unsigned)W) {
            flg[lc] = 1;
            if (VALUES) atomicAdd(acc + lc, v);
        } else {
            atomicOr(err, ERR_B_COL);
        }
    }
    __device__ __forceinline__ void apply(const Item& it, float a, long long, int) { add(it.c, a * it.b); }
    template <int G>
    __device__ __forceinline__ void done(int, int, int, long long) {}
    // flattened-mode interface (expand_chunk)
    __device__ __forceinline__ void step4(const long long* j, const float* a, const int*) {
        Item it[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) it[u] = fetch(j[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) add(it[u].c, a[u] * it[u].b);
    }
    __device__ __forceinline__ void step1(long long j, float a, int, bool ok) {
        if (ok) {
            const Item it = fetch(j);
            add(it.c, a * it.b);
        }
    }
    // quads (plus-times, packed B padded by four entries): two 16-byte loads
    // give the four (column, value) pairs of a quad
    __device__ __forceinline__ void quads(const Chunk& ch, int nv) {
        if constexpr (VALUES && std::is_same<BA, BPacked>::value) {
            const int4* P4 = reinterpret_cast<const int4*>(ba.P);
            quads_loaded(ch, nv, [&](long long qb, long long s, long long end, float a) {
                const int4 v0 = __ldg(P4 + (qb >> 1)), v1 = __ldg(P4 + (qb >> 1) + 1);
                const int cs[4] = {v0.x, v0.z, v1.x, v1.z};
                const int bs[4] = {v0.y, v0.w, v1.y, v1.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (qb + u >= s && qb + u < end) add(cs[u], a * __int_as_float(bs[u]));
            });
        }
    }
};

// Warp read-out: lane l looks at columns 4l..4l+3 of each 128-column block.
template <bool VALUES>
__device__ __forceinline__ void warp_emit4(float* acc, unsigned char* flg, int W, int c0, long long& out,
                                           long long out_end, int* Ci, float* Cx,
                                           unsigned long long* err) {
    const int lane = lane_id();
    for (int base = 0; base < W; base += 128) {
        const int cb = base + 4 * lane;
        unsigned f = 0;
        if (cb < W) f = *reinterpret_cast<const unsigned*>(flg + cb) & 0x01010101u;
        const int cnt = __popc(f);
        const int incl = warp_incl_scan(cnt);
        long long pos = out + incl - cnt;
        out += __shfl_sync(FULL, incl, 31);
        if (f) {
            *reinterpret_cast<unsigned*>(flg + cb) = 0u;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (VALUES) {
                v = *reinterpret_cast<const float4*>(acc + cb);
                *reinterpret_cast<float4*>(acc + cb) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (f & (1u << (8 * u))) {
                    if (pos < out_end) {
                        Ci[pos] = c0 + cb + u;
                        if (VALUES) Cx[pos] = vv[u];
                    } else {
                        atomicOr(err, ERR_C_ROW);
                    }
                    ++pos;
                }
            }
        }
    }
}

// Block-wide read-out for a heavy row; wcnt has W/32 + 1 entries.
template <bool VALUES>
__device__ __forceinline__ void cta_emit(float* acc, unsigned char* flg, int W, int c0, long long& out,
                                         long long out_end, int* Ci, float* Cx, int* wcnt,
                                         unsigned long long* err) {
    const int nw = blockDim.x >> 5, warp = warp_id(), lane = lane_id();
    const int words = W >> 5;
    const unsigned lt = lanemask_lt();
    for (int w = warp; w < words; w += nw) {
        const unsigned bal = __ballot_sync(FULL, flg[w * 32 + lane] != 0);
        if (lane == 0) wcnt[w] = __popc(bal);
    }
    __syncthreads();
    if (warp == 0) {
        const int tot = warp_excl_scan_smem(wcnt, words);
        if (lane == 0) wcnt[words] = tot;
    }
    __syncthreads();
    for (int w = warp; w < words; w += nw) {
        const int c = w * 32 + lane;
        const bool f = flg[c] != 0;
        const unsigned bal = __ballot_sync(FULL, f);
        if (f) {
            const long long pos = out + wcnt[w] + __popc(bal & lt);
            if (pos < out_end) {
                Ci[pos] = c0 + c;
                if (VALUES) Cx[pos] = acc[c];
            } else {
                atomicOr(err, ERR_C_ROW);
            }
            flg[c] = 0;
            if (VALUES) acc[c] = 0.0f;
        }
    }
    out += wcnt[words];
    __syncthreads();
}

template <bool VALUES, int G, class BA, bool CTA, class Seg>
__device__ __forceinline__ void numeric_tile(const NumParams& p, const BA& ba, const Seg& seg, long long a0,
                                             long long a1, DenseOp<VALUES, BA>& op) {
    unsigned long long* err = &p.hdr->err;
    const int nw = blockDim.x >> 5;
    const long long first = CTA ? a0 + 32LL * warp_id() : a0;
    const long long stride = CTA ? 32LL * nw : 32LL;
    const float* Ax = VALUES ? p.Ax : nullptr;
    for (long long e0 = first; e0 < a1; e0 += stride) {
        const int nv = (int)(a1 - e0 < 32 ? a1 - e0 : 32);
        const Chunk ch = load_chunk(e0, nv, p.Ai, Ax, p.nB, seg, err);
        expand_any<G>(ch, nv, e0, op);
    }
}

// Heavy row: the whole block works on one row.
template <bool VALUES, int G, class BA>
__device__ __forceinline__ void numeric_row_cta(const NumParams& p, const BA& ba, int row, float* acc,
                                                unsigned char* flg, int* wcnt) {
    unsigned long long* err = &p.hdr->err;
    const long long a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
    const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
    long long out = clampll(__ldg(p.Cp + row), 0, p.nnzC);
    const long long out_end = clampll(__ldg(p.Cp + row + 1), out, p.nnzC);
    for (int t = 0; t < p.T; ++t) {
        DenseOp<VALUES, BA> op{ba, acc, flg, p.d, t * p.W, p.W, err};
        if (p.T == 1) numeric_tile<VALUES, G, BA, true>(p, ba, SegWhole{p.Bp, p.nnzB, p.d}, a0, a1, op);
        else numeric_tile<VALUES, G, BA, true>(p, ba, SegTile{p.tp, p.T + 1, t, p.W}, a0, a1, op);
        __syncthreads();
        cta_emit<VALUES>(acc, flg, p.W, t * p.W, out, out_end, p.Ci, p.Cx, wcnt, err);
    }
    if (out != out_end && threadIdx.x == 0) atomicOr(err, ERR_C_ROW);
}

// One part of a split row: the block accumulates entries [e0, e1) tile by
// tile and adds each tile into the row's staging slot (columns t*W + c).  The
// block finishing the last part reads the row out of the staging slot in
// ascending column order and clears the slot.
template <bool VALUES, int G, class BA>
__device__ __forceinline__ void numeric_split_part(const NumParams& p, const BA& ba, const SplitItem& it,
                                                   float* acc, unsigned char* flg, int* wcnt, int* s_last) {
    unsigned long long* err = &p.hdr->err;
    float* sv = p.s.stg_vals + (size_t)it.slot * p.s.dpad;
    unsigned char* sf = p.s.stg_flags + (size_t)it.slot * p.s.dpad;
    for (int t = 0; t < p.T; ++t) {
        DenseOp<VALUES, BA> op{ba, acc, flg, p.d, t * p.W, p.W, err};
        if (p.T == 1) numeric_tile<VALUES, G, BA, true>(p, ba, SegWhole{p.Bp, p.nnzB, p.d}, it.e0, it.e1, op);
        else numeric_tile<VALUES, G, BA, true>(p, ba, SegTile{p.tp, p.T + 1, t, p.W}, it.e0, it.e1, op);
        __syncthreads();
        for (int c = threadIdx.x; c < p.W; c += blockDim.x) {
            if (flg[c]) {
                if (VALUES) {
                    atomicAdd(sv + t * p.W + c, acc[c]);
                    acc[c] = 0.0f;
                }
                sf[t * p.W + c] = 1;
                flg[c] = 0;
            }
        }
        __syncthreads();
    }
    if (!split_part_done(p.s, it.slot, it.nsub, s_last)) return;
    split_row_readout<VALUES>(p, it, wcnt);
}

// Light row, one warp, driven by pipelined_rows: the first chunk of A (for
// column tile 0) arrives preloaded; the row's output range is requested at
// the start of the gather and used by the read-out.
template <bool VALUES, int G, class BA>
struct NumRowBody {
    const NumParams& p;
    const BA& ba;
    float* acc;
    unsigned char* flg;
    unsigned long long* err;
    long long out, out_end;
    __device__ __forceinline__ void gather(int row, long long a0, long long a1, const Chunk& ch0, int nv0, int) {
        out = clampll(__ldg(p.Cp + row), 0, p.nnzC);
        out_end = clampll(__ldg(p.Cp + row + 1), out, p.nnzC);
        const float* Ax = VALUES ? p.Ax : nullptr;
        for (int t = 0; t < p.T; ++t) {
            DenseOp<VALUES, BA> op{ba, acc, flg, p.d, t * p.W, p.W, err};
            long long e_next = a0;
            if (t == 0) {
                expand_any<G>(ch0, nv0, a0, op);
                e_next = a0 + 32;
            }
            if (p.T == 1) {
                const SegWhole seg{p.Bp, p.nnzB, p.d};
                for (long long e0 = e_next; e0 < a1; e0 += 32) {
                    const int nv = (int)(a1 - e0 < 32 ? a1 - e0 : 32);
                    expand_any<G>(load_chunk(e0, nv, p.Ai, Ax, p.nB, seg, err), nv, e0, op);
                }
            } else {
                const SegTile seg{p.tp, p.T + 1, t, p.W};
                for (long long e0 = e_next; e0 < a1; e0 += 32) {
                    const int nv = (int)(a1 - e0 < 32 ? a1 - e0 : 32);
                    expand_any<G>(load_chunk(e0, nv, p.Ai, Ax, p.nB, seg, err), nv, e0, op);
                }
                if (t + 1 < p.T) {  // the last tile is read out by finish()
                    __syncwarp();
                    warp_emit4<VALUES>(acc, flg, p.W, t * p.W, out, out_end, p.Ci, p.Cx, err);
                    __syncwarp();
                }
            }
        }
    }
    __device__ __forceinline__ void finish(int) {
        __syncwarp();
        warp_emit4<VALUES>(acc, flg, p.W, (p.T - 1) * p.W, out, out_end, p.Ci, p.Cx, err);
        __syncwarp();
        if (out != out_end && lane_id() == 0) atomicOr(err, ERR_C_ROW);
    }
};


// ---------------------------------------------------------------------------
// Light rows in row groups (plus-times, packed B; template RG = lanes per
// row).  A warp takes R = 32/RG consecutive light rows of the schedule at a
// time; the RG lanes of row slot g accumulate row g into their own dense
// accumulator of W floats.  The slot walks the segments B(k,:) of its row's
// entries one after another in quads (RG lanes, four consecutive entries per
// lane, two 16-byte loads of the packed copy of B, padded by four entries):
// the columns of one segment are distinct, so acc[c] += A(i,k) * B(k,c) is a
// plain load and store, and __syncwarp between segments orders the updates
// of one column made by different lanes.  A column no product reached holds
// RG_EMPTY, a signalling-NaN bit pattern: arithmetic never delivers a
// signalling NaN (a NaN result is quiet), so no product or sum carries it and
// no occupancy flags are kept.  The R rows advance in lockstep (consecutive
// rows of the schedule share a flop class, so their lengths are close) and
// are read out together: lane l of a slot takes four columns of every
// 4*RG-column block, so all 32 lanes work in every read-out step.
// ---------------------------------------------------------------------------
// A segment of B as a slot walks it: its first position rounded down to a
// multiple of E (qbase), the positions to skip before the segment (lead),
// the positions covered from qbase (span) and A's value a.  E consecutive
// entries per lane (E = 4: two 16-byte loads; E = 2: one), lane gl taking
// groups gl, gl + RG, ...
struct RgSeg {
    long long qbase;
    int lead, span;
    float a;
};

template <int E>
__device__ __forceinline__ RgSeg rg_seg_of(long long s, int L, float a) {
    RgSeg q;
    q.qbase = s & ~(long long)(E - 1);
    q.lead = (int)(s - q.qbase);
    q.span = L > 0 ? q.lead + L : 0;
    q.a = a;
    return q;
}

// Loads of group q of a segment (entries qbase + E*q ...), if it exists.
template <int E>
__device__ __forceinline__ void rg_fetch(const int4* __restrict__ P4, const RgSeg& sg, int q, int4& v0, int4& v1) {
    if (E * q < sg.span) {
        const long long qb = sg.qbase + (long long)E * q;
        v0 = __ldg(P4 + (qb >> 1));
        if constexpr (E == 4) v1 = __ldg(P4 + (qb >> 1) + 1);
    }
}

// Accumulate group q of a segment from its loaded entries, without branches:
// a position outside the segment, or a column outside the tile (an input
// error, reported through `bad`), is added into the slot's spare column W,
// which is never read out.
template <int E>
__device__ __forceinline__ void rg_apply(float* acc, const RgSeg& sg, int q, const int4& v0, const int4& v1, int Wd,
                                         int W, int c0, bool& bad) {
    const int cs[4] = {v0.x, v0.z, v1.x, v1.z};
    const int bs[4] = {v0.y, v0.w, v1.y, v1.w};
    const int p0 = E * q;
#pragma unroll
    for (int u = 0; u < E; ++u) {
        const bool in_seg = p0 + u >= sg.lead && p0 + u < sg.span;
        const int lc = cs[u] - c0;
        const bool ok = (unsigned)lc < (unsigned)Wd;
        bad |= in_seg && !ok;
        rg_add(acc, in_seg && ok ? lc : W, sg.a * __int_as_float(bs[u]));
    }
}

// A whole segment whose first group (q = gl) is already loaded into v0/v1.
template <int RG, int E>
__device__ __forceinline__ void rg_segment(const int4* __restrict__ P4, float* acc, const RgSeg& sg, int gl,
                                           const int4& v0, const int4& v1, int Wd, int W, int c0, bool& bad) {
    if (E * gl < sg.span) rg_apply<E>(acc, sg, gl, v0, v1, Wd, W, c0, bad);
    for (int q = gl + RG; E * q < sg.span; q += RG) {
        int4 w0 = make_int4(0, 0, 0, 0), w1 = make_int4(0, 0, 0, 0);
        rg_fetch<E>(P4, sg, q, w0, w1);
        rg_apply<E>(acc, sg, q, w0, w1, Wd, W, c0, bad);
    }
}

// Segment of B's row k in the current tile (empty for k = -1; bad k is an
// input error).
template <class Seg>
__device__ __forceinline__ void rg_seg(const NumParams& p, const Seg& seg, int k, bool ok, long long& s, int& L,
                                       unsigned long long* err) {
    s = 0;
    L = 0;
    if (!ok) return;
    if ((unsigned)k < (unsigned)p.nB) seg(k, s, L);
    else atomicOr(err, ERR_A_COL);
}

// Chunks of RG entries of every slot's row for tile t, software-pipelined:
// while chunk c is accumulated, the segments of chunk c+1 (B's row pointers)
// and the entries of chunk c+2 (A's columns and values) are loaded.
template <int RG, class Seg>
__device__ __forceinline__ void rg_tile(const NumParams& p, const Seg& seg, const int4* P4, float* acc, long long a0,
                                        int len, int lmax, int c0, int Wd, unsigned long long* err, bool& bad) {
    constexpr int E = RG == 4 ? 4 : 2;
    const int lane = lane_id(), g = lane / RG, gl = lane % RG;
    int k0, k1;
    float x0, x1;
    rg_load_a(p, a0 + gl, gl < len, k0, x0);
    rg_load_a(p, a0 + RG + gl, RG + gl < len, k1, x1);
    long long s;
    int L;
    rg_seg(p, seg, k0, gl < len, s, L, err);
    // segment pipeline: the next segment's description and first group
    RgSeg nxt = rg_seg_of<E>(shfl64(s, g * RG), __shfl_sync(FULL, L, g * RG), __shfl_sync(FULL, x0, g * RG));
    int4 n0 = make_int4(0, 0, 0, 0), n1 = make_int4(0, 0, 0, 0);
    rg_fetch<E>(P4, nxt, gl, n0, n1);
    for (int e = 0; e < lmax; e += RG) {
        int k2;
        float x2;
        long long ns;
        int nL;
        rg_load_a(p, a0 + e + 2 * RG + gl, e + 2 * RG + gl < len, k2, x2);
        rg_seg(p, seg, k1, e + RG + gl < len, ns, nL, err);
        prefetch_segment(p.Bpk, ns, nL);  // the next chunk's rows of B into L2
        const int nu = lmax - e < RG ? lmax - e : RG;
        for (int u = 0; u < nu; ++u) {
            const RgSeg cur = nxt;
            const int4 c0v = n0, c1v = n1;
            // describe and start loading the segment after this one
            long long s2 = 0;
            int L2 = 0;
            float a2 = 0.0f;
            if (u + 1 < nu) {
                s2 = shfl64(s, g * RG + u + 1);
                L2 = __shfl_sync(FULL, L, g * RG + u + 1);
                a2 = __shfl_sync(FULL, x0, g * RG + u + 1);
            } else {  // first segment of the next chunk (empty past the rows' ends)
                s2 = shfl64(ns, g * RG);
                L2 = __shfl_sync(FULL, nL, g * RG);
                a2 = __shfl_sync(FULL, x1, g * RG);
            }
            nxt = rg_seg_of<E>(s2, L2, a2);
            rg_fetch<E>(P4, nxt, gl, n0, n1);
            rg_segment<RG, E>(P4, acc, cur, gl, c0v, c1v, Wd, p.W, c0, bad);
            __syncwarp();
        }
        s = ns;
        L = nL;
        x0 = x1;
        k1 = k2;
        x1 = x2;
    }
}

// The warp's light rows: row groups idx0, idx0 + step, ... (step = R * warps).
template <int RG>
__device__ __forceinline__ void rg_light_rows(const NumParams& p, float* racc, long long idx0, long long end,
                                              long long step, const long long* mark) {
    constexpr int R = 32 / RG;
    static_assert(RG >= 4 && RG <= 16 && 32 % RG == 0, "lanes per row");
    const int lane = lane_id(), g = lane / RG, gl = lane % RG;
    const int4* P4 = reinterpret_cast<const int4*>(p.Bpk);
    float* acc = racc + g * (p.W + 8);  // W columns, a spare and padding
    unsigned long long* err = &p.hdr->err;
    bool bad = false;
    for (long long idx = idx0; idx < end; idx += step) {
        const long long my = idx + g;
        long long a0 = 0, a1 = 0, out = 0, out_end = 0;
        bool active = false;
        if (my < end) {
            const int row = __ldg(p.perm + my);
            a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
            a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
            if (mark && is_split_row(mark, row, a1 - a0)) {
                a1 = a0;  // taken as split parts
            } else {
                active = true;
                out = clampll(__ldg(p.Cp + row), 0, p.nnzC);
                out_end = clampll(__ldg(p.Cp + row + 1), out, p.nnzC);
            }
        }
        const int len = (int)(a1 - a0);
        const int lmax = (int)__reduce_max_sync(FULL, (unsigned)len);
        for (int t = 0; t < p.T; ++t) {
            const int c0 = t * p.W;
            const int Wd = p.d - c0 < p.W ? p.d - c0 : p.W;
            if (p.T == 1) rg_tile<RG>(p, SegWhole{p.Bp, p.nnzB, p.d}, P4, acc, a0, len, lmax, c0, Wd, err, bad);
            else rg_tile<RG>(p, SegTile{p.tp, p.T + 1, t, p.W}, P4, acc, a0, len, lmax, c0, Wd, err, bad);
            rg_emit<RG>(racc, p.W, c0, out, out_end, p.Ci, p.Cx, err);
            __syncwarp();
        }
        if (active && gl == 0 && out != out_end) atomicOr(err, ERR_C_ROW);
    }
    if (bad) atomicOr(err, ERR_B_COL);
}

// Entries [a0, a0 + len) of A of a slot's row (len = 0 and inactive past the
// schedule's end, or for a split row, whose entries are taken as split parts).
__device__ __forceinline__ void rg_row_bounds(const NumParams& p, int row, const long long* mark, long long& a0,
                                              int& len, bool& active) {
    a0 = 0;
    len = 0;
    active = false;
    if (row < 0) return;
    a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
    const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
    if (mark && is_split_row(mark, row, a1 - a0)) return;
    len = (int)(a1 - a0);
    active = true;
}

// rg_light_rows on the row-aligned copy (T = 1), pipelined across row
// groups: while group idx is gathered, the schedule entry of group idx + 2
// steps and the row bounds of group idx + step are in flight; the next
// group's first two chunks of A and output range load before this group's
// read-out.  A group then starts with only B's row pointers and first groups
// to wait for.
template <int RG>
__device__ __forceinline__ void rgp_light_rows(const NumParams& p, float* racc, long long idx0, long long end,
                                               long long step, const long long* mark) {
    constexpr int E = RG == 4 ? 4 : 2;
    const int lane = lane_id(), g = lane / RG, gl = lane % RG;
    float* acc = racc + g * (p.W + 8);  // W columns, a spare and padding
    unsigned long long* err = &p.hdr->err;
    auto row_at = [&](long long idx) { return idx + g < end ? __ldg(p.perm + idx + g) : -1; };
    int row = row_at(idx0), nrow = row_at(idx0 + step);
    long long a0;
    int len;
    bool active;
    rg_row_bounds(p, row, mark, a0, len, active);
    long long out = 0, out_end = 0;
    if (active) {
        out = clampll(__ldg(p.Cp + row), 0, p.nnzC);
        out_end = clampll(__ldg(p.Cp + row + 1), out, p.nnzC);
    }
    int k0, k1;
    float x0, x1;
    rg_load_a(p, a0 + gl, gl < len, k0, x0);
    rg_load_a(p, a0 + RG + gl, RG + gl < len, k1, x1);
    for (long long idx = idx0; idx < end; idx += step) {
        long long na0;
        int nlen;
        bool nactive;
        rg_row_bounds(p, nrow, mark, na0, nlen, nactive);
        const int nnrow = row_at(idx + 2 * step);
        const int lmax = (int)__reduce_max_sync(FULL, (unsigned)len);
        rgp_tile<RG, E>(p, p.Bq, AddPlain{acc}, a0, len, lmax, err, k0, x0, k1, x1);
        rg_load_a(p, na0 + gl, gl < nlen, k0, x0);
        rg_load_a(p, na0 + RG + gl, RG + gl < nlen, k1, x1);
        long long nout = 0, nout_end = 0;
        if (nactive) {
            nout = clampll(__ldg(p.Cp + nrow), 0, p.nnzC);
            nout_end = clampll(__ldg(p.Cp + nrow + 1), nout, p.nnzC);
        }
        rg_emit<RG>(racc, p.W, 0, out, out_end, p.Ci, p.Cx, err);
        __syncwarp();
        if (active && gl == 0 && out != out_end) atomicOr(err, ERR_C_ROW);
        a0 = na0;
        len = nlen;
        active = nactive;
        out = nout;
        out_end = nout_end;
        nrow = nnrow;
    }
}

// Light rows only, in row groups; R = 32/RG accumulators of W + 8 floats per warp.
// Launched behind k_numeric (which then skips light rows) with programmatic
// dependent launch: its blocks may start while k_numeric's last blocks run.
// Before exiting, each block waits for k_numeric to complete, so that work
// queued after this kernel sees all of C.  PADDED: p.Bq is set (T = 1) and the
// pipelined walk over the row-aligned copy runs (a separate instance keeps
// each walk's registers to itself).
template <int RG, bool PADDED>
__global__ void __launch_bounds__(256, 5) k_numeric_light(NumParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_nheavy, s_nrows;
    constexpr int R = 32 / RG;
    const int nw = blockDim.x >> 5, warp = warp_id(), tid = threadIdx.x;
    float* racc = reinterpret_cast<float*>(smem);
    for (int i = tid; i < nw * R * (p.W + 8); i += blockDim.x) reinterpret_cast<unsigned*>(racc)[i] = RG_EMPTY;
    if (tid < 32) {  // one warp; its lanes store the same values
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        if (p.tiny_max) {  // the tiny rows, last in the class order, run in k_numeric_tiny
            long long t = 0;
            for (int c = 1 + lane_id(); c <= TINY_CLASS && c < p.cta_class; c += 32) t += p.hdr->hist[c];
            nr -= warp_sum(t);
        }
        s_nheavy = nh;
        s_nrows = nr;
    }
    __syncthreads();
    const long long* mark = p.s.stg_vals != nullptr ? p.s.flops : nullptr;
    float* wacc = racc + (size_t)warp * R * (p.W + 8);
    const long long idx0 = s_nheavy + ((long long)blockIdx.x * nw + warp) * R, step = (long long)gridDim.x * nw * R;
    if constexpr (PADDED) rgp_light_rows<RG>(p, wacc, idx0, s_nrows, step, mark);
    else rg_light_rows<RG>(p, wacc, idx0, s_nrows, step, mark);
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Split parts and heavy rows in row groups.  The block's S = warps * 32/RG
// slots share one item (a part of a split row, or a heavy row): each slot
// takes a contiguous share of the item's A entries and accumulates it into
// its own dense accumulator exactly as a light row (no atomics: within a
// slot one segment of B is in flight at a time).  The block then sums the
// S accumulators column by column (a column no slot reached stays
// RG_EMPTY) and resets them, and the sum is read out (heavy row) or added
// into the row's staging slot (split part).
// ---------------------------------------------------------------------------
template <int RG>
__device__ __forceinline__ void rgcta_tile(const NumParams& p, const int4* P4, float* racc, long long e0,
                                           long long e1, int t, bool& bad) {
    constexpr int R = 32 / RG;
    const int S = (blockDim.x >> 5) * R, slot = warp_id() * R + lane_id() / RG;
    const long long n = e1 - e0, q = n / S, r = n % S;
    const long long a0 = e0 + q * slot + (slot < r ? slot : r);
    const int len = (int)(q + (slot < r ? 1 : 0));
    const int lmax = (int)__reduce_max_sync(FULL, (unsigned)len);
    float* acc = racc + (size_t)slot * (p.W + 8);
    const int c0 = t * p.W;
    const int Wd = p.d - c0 < p.W ? p.d - c0 : p.W;
    unsigned long long* err = &p.hdr->err;
    if (p.Bq) {  // T = 1
        const int gl = lane_id() % RG;
        int k0, k1;
        float x0, x1;
        rg_load_a(p, a0 + gl, gl < len, k0, x0);
        rg_load_a(p, a0 + RG + gl, RG + gl < len, k1, x1);
        rgp_tile<RG, RG == 4 ? 4 : 2>(p, p.Bq, AddPlain{acc}, a0, len, lmax, err, k0, x0, k1, x1);
    } else if (p.T == 1) rg_tile<RG>(p, SegWhole{p.Bp, p.nnzB, p.d}, P4, acc, a0, len, lmax, c0, Wd, err, bad);
    else rg_tile<RG>(p, SegTile{p.tp, p.T + 1, t, p.W}, P4, acc, a0, len, lmax, c0, Wd, err, bad);
}

// Split parts, then heavy rows, in row groups (plus-times, padded packed B).
// Shared memory: S accumulators of W + 8 floats (the slots), then W floats
// for the summed tile.  Launched ahead of k_numeric_light, which takes the
// light rows.
template <int RG>
__global__ void __launch_bounds__(256, 5) k_numeric_rgcta(NumParams p) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_wcnt[MAX_DENSE_W / 32 + 1];
    __shared__ long long s_item, s_nheavy;
    __shared__ int s_last;
    constexpr int R = 32 / RG;
    const int tid = threadIdx.x, S = (blockDim.x >> 5) * R, ld = p.W + 8;
    float* racc = reinterpret_cast<float*>(smem);
    float* sum = racc + (size_t)S * ld;
    for (int i = tid; i < S * ld + p.W; i += blockDim.x) reinterpret_cast<unsigned*>(racc)[i] = RG_EMPTY;
    if (tid < 32) {  // one warp; its lanes store the same values
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
    }
    __syncthreads();
    const long long nheavy = s_nheavy;
    const int4* P4 = reinterpret_cast<const int4*>(p.Bpk);
    unsigned long long* err = &p.hdr->err;
    bool bad = false;
    const bool split_ok = p.s.stg_vals != nullptr;
    const long long* mark = split_ok ? p.s.flops : nullptr;
    const long long nitems = split_ok ? min(*(volatile long long*)&p.hdr->scratch[2], p.item_cap) : 0;
    SplitItem it;
    while (next_split_item(p.s, p.Ap, p.nnzA, nitems, &s_item, it)) {
        float* sv = p.s.stg_vals + (size_t)it.slot * p.s.dpad;
        unsigned char* sf = p.s.stg_flags + (size_t)it.slot * p.s.dpad;
        for (int t = 0; t < p.T; ++t) {
            rgcta_tile<RG>(p, P4, racc, it.e0, it.e1, t, bad);
            __syncthreads();
            for (int c = tid; c < p.W; c += blockDim.x) {
                const unsigned x = rgcta_sum(racc, ld, S, c);
                if (x != RG_EMPTY) {
                    atomicAdd(sv + t * p.W + c, __uint_as_float(x));
                    sf[t * p.W + c] = 1;
                }
            }
            __syncthreads();
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
        long long out = clampll(__ldg(p.Cp + row), 0, p.nnzC);
        const long long out_end = clampll(__ldg(p.Cp + row + 1), out, p.nnzC);
        for (int t = 0; t < p.T; ++t) {
            rgcta_tile<RG>(p, P4, racc, a0, a1, t, bad);
            __syncthreads();
            for (int c = tid; c < p.W; c += blockDim.x) sum[c] = __uint_as_float(rgcta_sum(racc, ld, S, c));
            __syncthreads();
            rgcta_emit(sum, p.W, t * p.W, out, out_end, p.Ci, p.Cx, s_wcnt, err);
        }
        if (out != out_end && tid == 0) atomicOr(err, ERR_C_ROW);
    }
    if (bad) atomicOr(err, ERR_B_COL);
}

// A light row as the pipeline holds it: its row id (-1: none), first entry
// of A and length.
struct WideRow {
    int row;
    int len;
    long long a0;
};

__device__ __forceinline__ WideRow wide_row(const NumParams& p, int row) {
    WideRow r{row, 0, 0};
    if (row < 0) return r;
    r.a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
    r.len = (int)(clampll(__ldg(p.Ap + row + 1), r.a0, p.nnzA) - r.a0);
    return r;
}

// The light rows of one warp in natural row order: chunks c, c + step, ...
// of 32 consecutive rows, and in each chunk the rows with products below
// the heavy threshold (split rows carry a negative mark in the flops array
// and heavy rows belong to the blocks).  Rows of C that follow each other
// are then written one after another by the same warp, so that C's lines
// fill while they are in L2, and A is read in order.  The flops of the
// chunk after the current one are loaded ahead.
struct LightRows {
    long long chunk, step, nchunks;
    long long base;
    unsigned mask;
    long long f_next;  // this lane's row of chunk `chunk + step`
    // light and not left to the tiny-row kernel (tiny = 0: none is)
    __device__ __forceinline__ static bool light(long long f, int cc, int tiny) {
        return f > tiny && f > 0 && flops_class(f) < cc;
    }
    __device__ __forceinline__ static long long flops_of(const NumParams& p, long long c, long long nchunks) {
        const long long row = c * 32 + lane_id();
        return (c < nchunks && row < p.nB) ? __ldg(p.s.flops + row) : 0;
    }
    __device__ __forceinline__ void start(const NumParams& p, long long c0, long long st, int cc) {
        step = st;
        nchunks = ((long long)p.nB + 31) / 32;
        chunk = c0;
        base = c0 * 32;
        mask = __ballot_sync(FULL, light(flops_of(p, c0, nchunks), cc, p.tiny_max));
        f_next = flops_of(p, c0 + st, nchunks);
    }
    // next light row of this warp, -1 when none is left (warp-uniform)
    __device__ __forceinline__ int next(const NumParams& p, int cc) {
        while (mask == 0) {
            if (chunk >= nchunks) return -1;
            chunk += step;
            base = chunk * 32;
            mask = __ballot_sync(FULL, light(f_next, cc, p.tiny_max));
            f_next = flops_of(p, chunk + step, nchunks);
        }
        const int b = __ffs(mask) - 1;
        mask &= mask - 1;
        return (int)(base + b);
    }
};

// Persistent kernel: split parts, then heavy rows (team = block: warp w
// walks the item's chunks w, w + warps, ... into its own accumulator and the
// block sums the warps' accumulators into warp 0's),
// then light rows (team = warp, in natural row order, pipelined: while row
// r is walked and read out, the row pointers of B for row r + 1's first
// chunk, the entries of A of row r + 2 and the bounds of row r + 3 are in
// flight).  Shared memory per warp: W + 8 floats of accumulator and
// W/32 + 1 bitmap words (zero between items: every read-out resets what it
// emitted).
__global__ void __launch_bounds__(256, 4) k_numeric_wide(NumParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item, s_nheavy, s_nrows;
    __shared__ int s_last;
    __shared__ int s_wcnt[MAX_DENSE_W / 32 + 1];
    const int nwarps = blockDim.x >> 5, warp = warp_id(), lane = lane_id(), tid = threadIdx.x;
    const int ld = p.W + 8, nw = p.W >> 5, bmw = nw + 1;
    const int per_warp = ld + bmw;  // 4-byte words
    for (int i = tid; i < nwarps * per_warp; i += blockDim.x) reinterpret_cast<unsigned*>(smem)[i] = 0u;
    if (tid < 32) {  // one warp; its lanes store the same values
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
        s_nrows = nr;
    }
    __syncthreads();
    const long long nheavy = s_nheavy, nrows = s_nrows;
    unsigned long long* err = &p.hdr->err;
    const bool split_ok = p.s.stg_vals != nullptr;
    const long long* mark = split_ok ? p.s.flops : nullptr;
    // block teams: every warp walks its chunks into its own accumulator (no
    // contention between warps on the float additions), then the block sums
    // the warps' accumulators column by column
    float* wacc = reinterpret_cast<float*>(smem) + (size_t)warp * per_warp;
    unsigned* wbm = reinterpret_cast<unsigned*>(wacc) + ld;
    const AddShared wadd{wacc, wbm};
    float* acc0 = reinterpret_cast<float*>(smem);  // warp 0's accumulator takes the sum
    unsigned* bm0 = reinterpret_cast<unsigned*>(smem) + ld;
    // column c summed over the warps (and reset in every warp but 0, whose
    // accumulator gets the sum); returns whether any warp reached it
    auto merge_col = [&](int c, float& v) -> bool {
        bool any = false;
        v = 0.0f;
        for (int w = 0; w < nwarps; ++w) {
            float* aw = reinterpret_cast<float*>(smem) + (size_t)w * per_warp;
            const unsigned* bw = reinterpret_cast<const unsigned*>(aw) + ld;
            if ((bw[c >> 5] >> (c & 31)) & 1u) {
                v += aw[c];
                any = true;
                if (w) aw[c] = 0.0f;
            }
        }
        return any;
    };
    auto clear_bitmaps = [&]() {
        for (int i = tid; i < nwarps * nw; i += blockDim.x)
            reinterpret_cast<unsigned*>(smem)[(size_t)(i / nw) * per_warp + ld + (i % nw)] = 0u;
    };
    // parts of split rows: accumulate, then add the occupied columns into the
    // row's staging slot; the block completing a row's last part reads it out
    const long long nitems = split_ok ? min(*(volatile long long*)&p.hdr->scratch[2], p.item_cap) : 0;
    SplitItem it;
    while (next_split_item(p.s, p.Ap, p.nnzA, nitems, &s_item, it)) {
        wide_range(p, wadd, it.e0 + 32LL * warp, it.e1, 32LL * nwarps, err);
        __syncthreads();
        float* sv = p.s.stg_vals + (size_t)it.slot * p.s.dpad;
        unsigned char* sf = p.s.stg_flags + (size_t)it.slot * p.s.dpad;
        for (int c = tid; c < p.W; c += blockDim.x) {
            float v;
            if (merge_col(c, v)) {
                atomicAdd(sv + c, v);
                sf[c] = 1;
                acc0[c] = 0.0f;
            }
        }
        __syncthreads();
        clear_bitmaps();
        __syncthreads();
        if (!split_part_done(p.s, it.slot, it.nsub, &s_last)) continue;
        split_row_readout<true>(p, it, s_wcnt);
    }
    // heavy rows, one per block
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
        const long long out = clampll(__ldg(p.Cp + row), 0, p.nnzC);
        const long long out_end = clampll(__ldg(p.Cp + row + 1), out, p.nnzC);
        wide_range(p, wadd, a0 + 32LL * warp, a1, 32LL * nwarps, err);
        __syncthreads();
        for (int c = tid; c < p.W; c += blockDim.x) {
            float v;
            if (merge_col(c, v)) acc0[c] = v;
        }
        __syncthreads();
        // warp 0's bitmap becomes the union
        for (int i = tid; i < nw; i += blockDim.x) {
            unsigned u = 0;
            for (int w = 0; w < nwarps; ++w) u |= reinterpret_cast<const unsigned*>(smem)[(size_t)w * per_warp + ld + i];
            bm0[i] = u;
        }
        __syncthreads();
        const int tot = wide_emit(acc0, bm0, nw, out, out_end, p.Ci, p.Cx, warp, nwarps, err);
        __syncthreads();
        clear_bitmaps();
        if (tid == 0 && out + tot != out_end) atomicOr(err, ERR_C_ROW);
        __syncthreads();
    }
    // light rows, one per warp, in natural row order
    const unsigned W = (unsigned)p.W;
    const int cc = p.cta_class;
    LightRows q;
    q.start(p, (long long)blockIdx.x * nwarps + warp, (long long)gridDim.x * nwarps, cc);
    // pipeline fill: r0 with its segments, r1 with its entries of A, r2
    WideRow r0 = wide_row(p, q.next(p, cc));
    int k;
    float a;
    wide_load_a(p, r0.a0 + lane, lane < r0.len, k, a);
    unsigned g0;
    int np;
    wide_seg(p, k, g0, np, err);
    float ca = a;
    WideRow r1 = wide_row(p, q.next(p, cc));
    wide_load_a(p, r1.a0 + lane, lane < r1.len, k, a);
    WideRow r2 = wide_row(p, q.next(p, cc));
    while (r0.row >= 0) {
        const WideRow r3 = wide_row(p, q.next(p, cc));
        const long long out = clampll(__ldg(p.Cp + r0.row), 0, p.nnzC);
        const long long out_end = clampll(__ldg(p.Cp + r0.row + 1), out, p.nnzC);
        unsigned g1;
        int np1;
        wide_seg(p, k, g1, np1, err);  // row r + 1: segments of its first chunk
        const float ca1 = a;
        wide_load_a(p, r2.a0 + lane, lane < r2.len, k, a);  // row r + 2: its first chunk of A
        wide_chunk_walk(p.Bq, wadd, W, g0, np, ca, r0.len < 32 ? r0.len : 32);
        if (r0.len > 32) wide_range(p, wadd, r0.a0 + 32, r0.a0 + r0.len, 32, err);  // a long light row
        __syncwarp();
        const int tot = wide_emit(wacc, wbm, nw, out, out_end, p.Ci, p.Cx, 0, 1, err);
        if (lane == 0 && out + tot != out_end) atomicOr(err, ERR_C_ROW);
        __syncwarp();
        if (lane < nw) wbm[lane] = 0u;
        __syncwarp();
        r0 = r1;
        r1 = r2;
        r2 = r3;
        g0 = g1;
        np = np1;
        ca = ca1;
    }
}

size_t numeric_wide_smem(int W, int warps) {
    return (size_t)warps * 4 * (size_t)((W + 8) + (W / 32 + 1));
}

template <bool VALUES, int G, bool PACKED>
__global__ void __launch_bounds__(256, 5) k_numeric(NumParams p) {
    // a light-row kernel launched behind this one may start on SMs this
    // grid frees (the two touch disjoint rows of C)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_wcnt[MAX_DENSE_W / 32 + 1];
    __shared__ long long s_item, s_nheavy, s_nrows;
    const int nw = blockDim.x >> 5, warp = warp_id(), tid = threadIdx.x;
    const int slot = VALUES ? 5 * p.W : p.W;  // bytes per warp: W floats + W flags
    for (int i = tid; i < nw * slot / 4; i += blockDim.x) reinterpret_cast<unsigned*>(smem)[i] = 0u;

    if (tid < 32) {  // one warp; its lanes store the same values
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
        s_nrows = nr;
    }
    __syncthreads();
    const long long nheavy = s_nheavy, nrows = s_nrows;
    using BA = typename std::conditional<PACKED, BPacked, BSep>::type;
    BA ba;
    if constexpr (PACKED) ba = BPacked{p.Bpk};
    else ba = BSep{p.Bi, VALUES ? p.Bx : nullptr};
    // without a staging area (d above the dense staging width) split rows are
    // processed whole like any other row
    const bool split_ok = p.s.stg_vals != nullptr;
    const long long* mark = split_ok ? p.s.flops : nullptr;
    {
        float* acc = reinterpret_cast<float*>(smem);
        unsigned char* flg = smem + (VALUES ? 4 * p.W : 0);
        // parts of split rows first (any block), then whole heavy rows
        const long long nitems = split_ok ? min(*(volatile long long*)&p.hdr->scratch[2], p.item_cap) : 0;
        __shared__ int s_last;
        SplitItem it;
        while (next_split_item(p.s, p.Ap, p.nnzA, nitems, &s_item, it))
            numeric_split_part<VALUES, G, BA>(p, ba, it, acc, flg, s_wcnt, &s_last);
        for (;;) {
            if (tid == 0) s_item = (long long)atomicAdd(&p.hdr->heavy_ctr, 1ull);
            __syncthreads();
            const long long h = s_item;
            __syncthreads();
            if (h >= nheavy) break;
            const int row = p.perm[h];
            if (mark && is_split_row(mark, row, __ldg(p.Ap + row + 1) - __ldg(p.Ap + row))) continue;
            numeric_row_cta<VALUES, G, BA>(p, ba, row, acc, flg, s_wcnt);
        }
    }
    if (p.skip_light) return;
    float* acc = reinterpret_cast<float*>(smem + (size_t)warp * slot);
    unsigned char* flg = smem + (size_t)warp * slot + (VALUES ? 4 * p.W : 0);
    NumRowBody<VALUES, G, BA> body{p, ba, acc, flg, &p.hdr->err, 0, 0};
    const long long idx0 = nheavy + (long long)blockIdx.x * nw + warp;
    const long long step = (long long)gridDim.x * nw;
    const float* Ax = VALUES ? p.Ax : nullptr;
    if (p.T == 1)
        pipelined_rows(p.perm, idx0, nrows, step, p.Ap, p.nnzA, p.Ai, Ax, p.nB, SegWhole{p.Bp, p.nnzB, p.d},
                       &p.hdr->err, body, mark);
    else
        pipelined_rows(p.perm, idx0, nrows, step, p.Ap, p.nnzA, p.Ai, Ax, p.nB,
                       SegTile{p.tp, p.T + 1, 0, p.W}, &p.hdr->err, body, mark);
}

__global__ void k_pack_b(long long nnz, const int* __restrict__ Bi, const float* __restrict__ Bx,
                         int2* __restrict__ P) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < nnz;
         j += (long long)gridDim.x * blockDim.x)
        P[j] = make_int2(__ldg(Bi + j), __float_as_int(__ldg(Bx + j)));
}

// The row-aligned copy (E entries per group): eight lanes per row of B, each
// lane one entry per step (loads and stores of a row are contiguous), pads
// included.
template <int E>
__global__ void __launch_bounds__(256) k_pack_b_rows(int nB, const long long* __restrict__ Bp, long long nnzB,
                                                     const int* __restrict__ Bi, const float* __restrict__ Bx, int d,
                                                     int2* __restrict__ Q, unsigned long long* err) {
    const int gl = threadIdx.x & 7;
    bool bad = false;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 3; k < nB; k += (gridDim.x * blockDim.x) >> 3) {
        long long s;
        int len;
        unsigned g0;
        padded_row<E>(Bp, nnzB, d, k, s, len, g0);
        const int span = (len + E - 1) & ~(E - 1);
        int2* q = Q + (size_t)g0 * E;
        for (int j = gl; j < span; j += 8) {
            int2 v = make_int2(-1, 0);
            if (j < len) {
                const int c = __ldg(Bi + s + j);
                const bool ok = (unsigned)c < (unsigned)d;
                bad |= !ok;
                v = make_int2(ok ? c : -1, __float_as_int(__ldg(Bx + s + j)));
            }
            q[j] = v;
        }
    }
    if (bad) atomicOr(err, ERR_B_COL);
}

// Entries of the row-aligned copy for B (n_B rows, nnzB entries, d columns)
// with groups of E entries: room for S(k) + the row's groups of any row k
// whose length is clamped to d.
static long long padded_b_entries(long long nB, long long nnzB, long long d, int E) {
    return (nnzB + (long long)(E - 1) * nB + d + 2LL * E + E - 1) / E * E;
}

size_t padded_b_bytes(long long nB, long long nnzB, long long d, int E) {
    return 8 * (size_t)padded_b_entries(nB, nnzB, d, E);
}

bool padded_b_fits(long long nB, long long nnzB, long long d, int E) {
    return padded_b_entries(nB, nnzB, d, E) / E < (1LL << 31) && nB < (1LL << 31);
}

cudaError_t launch_pack_b_rows(const DevCsr& B, int E, long long d, int4* Q, unsigned long long* err,
                               cudaStream_t st) {
    if (B.nrows == 0) return cudaSuccess;
    if ((E != 2 && E != 4) || !padded_b_fits(B.nrows, B.nnz, d, E)) return cudaErrorInvalidValue;
    long long blocks = (B.nrows + 31) / 32;  // 32 rows per block of 256 threads
    if (blocks > 152 * 16) blocks = 152 * 16;
    int2* P = reinterpret_cast<int2*>(Q);
    count_launch();
    if (E == 2)
        k_pack_b_rows<2><<<(unsigned)blocks, 256, 0, st>>>((int)B.nrows, B.rowptr, B.nnz, B.col, B.val, (int)d, P, err);
    else
        k_pack_b_rows<4><<<(unsigned)blocks, 256, 0, st>>>((int)B.nrows, B.rowptr, B.nnz, B.col, B.val, (int)d, P, err);
    return cudaGetLastError();
}

cudaError_t launch_pack_b(const DevCsr& B, int2* P, cudaStream_t st) {
    if (B.nnz == 0) return cudaSuccess;
    long long blocks = (B.nnz + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    count_launch();
    k_pack_b<<<(unsigned)blocks, 256, 0, st>>>(B.nnz, B.col, B.val, P);
    return cudaGetLastError();
}

size_t numeric_dense_smem(int W, int warps, bool values) {
    return (size_t)warps * (values ? 5 * (size_t)W : (size_t)W);
}

size_t numeric_light_smem(int W, int warps, int rg) {
    if (rg != 4 && rg != 8 && rg != 16) return 0;
    return (size_t)warps * (32 / rg) * 4 * ((size_t)W + 8);  // W columns, a spare, padding per row
}

size_t numeric_rgcta_smem(int W, int warps, int rg) {
    if (rg != 4 && rg != 8 && rg != 16) return 0;
    return numeric_light_smem(W, warps, rg) + 4 * (size_t)W;  // the slots, then the summed tile
}

template <int RG>
static cudaError_t launch_rgcta(const NumParams& p, int warps, int sms, cudaStream_t st) {
    const void* k = (const void*)k_numeric_rgcta<RG>;
    const size_t smem = numeric_rgcta_smem(p.W, warps, RG);
    cudaError_t e;
    if (smem == 0 || smem > 220 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    const int grid = persistent_grid(k, 32 * warps, smem, sms);
    count_launch();
    k_numeric_rgcta<RG><<<grid, 32 * warps, smem, st>>>(p);
    return cudaGetLastError();
}

static cudaError_t launch_wide(NumParams p, int warps, int sms, cudaStream_t st) {
    const void* k = (const void*)k_numeric_wide;
    const size_t smem = numeric_wide_smem(p.W, warps);
    cudaError_t e;
    if (p.W > 1024 || p.T != 1 || !p.Bq || smem > 220 * 1024) return cudaErrorInvalidValue;
    // rows with at most TINY_MAX products first, in registers
    if ((e = launch_numeric_tiny(p, sms, st))) return e;
    p.tiny_max = TINY_MAX;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    const int grid = persistent_grid(k, 32 * warps, smem, sms);
    count_launch();
    k_numeric_wide<<<grid, 32 * warps, smem, st>>>(p);
    return cudaGetLastError();
}

template <bool VALUES, int G, bool PACKED>
static cudaError_t launch_one(const NumParams& p, int warps, int sms, cudaStream_t st) {
    const void* k = (const void*)k_numeric<VALUES, G, PACKED>;
    const size_t smem = numeric_dense_smem(p.W, warps, VALUES);
    cudaError_t e;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    const int grid = persistent_grid(k, 32 * warps, smem, sms);
    count_launch();
    k_numeric<VALUES, G, PACKED><<<grid, 32 * warps, smem, st>>>(p);
    return cudaGetLastError();
}

template <bool VALUES, bool PACKED>
static cudaError_t launch_g(const NumParams& p, int G, int warps, int sms, cudaStream_t st) {
    switch (G) {
        case 1: return launch_one<VALUES, 1, PACKED>(p, warps, sms, st);
        case 2:
            if constexpr (VALUES && PACKED) return launch_one<VALUES, 2, PACKED>(p, warps, sms, st);
            else return launch_one<VALUES, 1, PACKED>(p, warps, sms, st);
        case 4: return launch_one<VALUES, 4, PACKED>(p, warps, sms, st);
        case 8: return launch_one<VALUES, 8, PACKED>(p, warps, sms, st);
        case 16: return launch_one<VALUES, 16, PACKED>(p, warps, sms, st);
        case 32: return launch_one<VALUES, 32, PACKED>(p, warps, sms, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int RG, bool PADDED>
static cudaError_t launch_light_k(const NumParams& p, int warps, int sms, cudaStream_t st) {
    const void* k = (const void*)k_numeric_light<RG, PADDED>;
    const size_t smem = numeric_light_smem(p.W, warps, RG);
    cudaError_t e;
    if (smem == 0 || smem > 220 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(persistent_grid(k, 32 * warps, smem, sms));
    lc.blockDim = dim3(32 * warps);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    count_launch();
    return cudaLaunchKernelEx(&lc, k_numeric_light<RG, PADDED>, p);
}

template <int RG>
static cudaError_t launch_light(const NumParams& p, int warps, int sms, cudaStream_t st) {
    return p.Bq ? launch_light_k<RG, true>(p, warps, sms, st) : launch_light_k<RG, false>(p, warps, sms, st);
}

cudaError_t launch_numeric_light_rows(const DevCsr& A, const DevCsr& B, long long d, int W, int T,
                                      const long long* tp, const int2* Bpk, const Sched& s, const LaunchCfg& cfg,
                                      const long long* Cp, int* Ci, float* Cx, long long nnzC, cudaStream_t st) {
    if (A.nrows == 0) return cudaSuccess;
    if (!Bpk || W <= 0 || W % 32 || W > MAX_DENSE_W || (long long)W * T < d) return cudaErrorInvalidValue;
    const NumParams p = numeric_params(A, B, d, W, T, tp, Bpk, s, cfg, Cp, Ci, Cx, nnzC);
    switch (cfg.row_lanes) {
        case 4: return launch_light<4>(p, cfg.warps_per_cta, cfg.sms, st);
        case 8: return launch_light<8>(p, cfg.warps_per_cta, cfg.sms, st);
        case 16: return launch_light<16>(p, cfg.warps_per_cta, cfg.sms, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_numeric_dense(const DevCsr& A, const DevCsr& B, long long d, int W, int T,
                                 const long long* tp, bool values, const int2* Bpk, int G,
                                 const Sched& s, const LaunchCfg& cfg, const long long* Cp, int* Ci,
                                 float* Cx, long long nnzC, cudaStream_t st, const int4* Bq) {
    cudaError_t e;
    if (A.nrows == 0) return cudaSuccess;
    if (W <= 0 || W % 32 || W > MAX_DENSE_W || (long long)W * T < d) return cudaErrorInvalidValue;
    if (cfg.warps_per_cta < 1 || cfg.warps_per_cta > 8) return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(&s.hdr->heavy_ctr, 0, 2 * sizeof(unsigned long long), st))) return e;
    NumParams p = numeric_params(A, B, d, W, T, tp, Bpk, s, cfg, Cp, Ci, Cx, nnzC);
    const int w = cfg.warps_per_cta;
    if (Bq && (T != 1 || !values || cfg.row_lanes == 32)) return cudaErrorInvalidValue;
    p.Bq = Bq;
    if (cfg.row_lanes == 1) {  // one shared accumulator per team, on the row-aligned copy
        if (!values || !Bq || T != 1 || W > 1024) return cudaErrorInvalidValue;
        return launch_wide(p, w, cfg.sms, st);
    }
    if (values && (Bpk || Bq) && cfg.row_lanes != 32) {  // row groups need a packed copy
        if (T > 1) {
            // Over several column tiles a segment of B holds only d_tile/d of its
            // row, so the block-wide sum of 32 slot accumulators per item and
            // tile costs more than the item's products: split parts and heavy
            // rows take the flag-and-atomic kernel, light rows the row groups.
            NumParams ph = p;
            ph.skip_light = 1;
            if ((e = launch_g<true, true>(ph, G, w, cfg.sms, st))) return e;
            switch (cfg.row_lanes) {
                case 4: return launch_light<4>(p, w, cfg.sms, st);
                case 8: return launch_light<8>(p, w, cfg.sms, st);
                case 16: return launch_light<16>(p, w, cfg.sms, st);
                default: return cudaErrorInvalidValue;
            }
        }
        if (Bq && cfg.row_lanes != 4) {  // one tile, the copy in pairs (E = 2): tiny rows first, in registers
            if ((e = launch_numeric_tiny(p, cfg.sms, st))) return e;
            p.tiny_max = TINY_MAX;
        }
        switch (cfg.row_lanes) {
            case 4:
                if ((e = launch_rgcta<4>(p, w, cfg.sms, st))) return e;
                return launch_light<4>(p, w, cfg.sms, st);
            case 8:
                if ((e = launch_rgcta<8>(p, w, cfg.sms, st))) return e;
                return launch_light<8>(p, w, cfg.sms, st);
            case 16:
                if ((e = launch_rgcta<16>(p, w, cfg.sms, st))) return e;
                return launch_light<16>(p, w, cfg.sms, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (values) return Bpk ? launch_g<true, true>(p, G, w, cfg.sms, st) : launch_g<true, false>(p, G, w, cfg.sms, st);
    return launch_g<false, false>(p, G, w, cfg.sms, st);
}

}  // namespace ts

// ===========================================================================
// Staged numeric pass: the same dense accumulator and read-out, with B's
// entries gathered into shared memory by cp.async windows (staged.cuh).
// ===========================================================================
namespace ts {

// A window whose copies are in flight, with what to do after it.
struct Pending {
    int buf;
    int m;
    int row;   // -1: no window
    int tile;
    bool last_of_tile;
    bool last_of_row;
    long long out, out_end;
};

template <bool VALUES>
__device__ __forceinline__ void process_window(const StageArea<VALUES ? 8 : 4>& sa, int b, int m, float* acc,
                                               unsigned char* flg, int d, int c0, int W, unsigned long long* err) {
    const int lane = lane_id();
    const unsigned char* own = sa.owner(b);
    const float* av = sa.avals(b);
#pragma unroll 4
    for (int k = 0; k < STAGE_P / 32; ++k) {
        const int s = lane + 32 * k;
        if (s < m) {
            int c;
            float v = 0.0f;
            if (VALUES) {
                const int2 e = reinterpret_cast<const int2*>(sa.payload(b))[s];
                c = e.x;
                v = av[own[s]] * __int_as_float(e.y);
            } else {
                c = reinterpret_cast<const int*>(sa.payload(b))[s];
            }
            const int lc = c - c0;
            if ((unsigned)c < (unsigned)d && (unsigned)lc < (unsigned)W) {
                flg[lc] = 1;
                if (VALUES) atomicAdd(acc + lc, v);
            } else {
                atomicOr(err, ERR_B_COL);
            }
        }
    }
}

// Every window of entries [e0, e1) (this warp's chunks, stride `stride`) of
// tile t accumulated into acc/flg; no read-out.  Used by block rows.
template <bool VALUES, class Seg>
__device__ __forceinline__ void staged_range(const NumParams& p, const StageArea<VALUES ? 8 : 4>& sa, long long e0,
                                             long long e1, long long stride, const Seg& seg, int t, float* acc,
                                             unsigned char* flg) {
    unsigned long long* err = &p.hdr->err;
    const void* src = VALUES ? (const void*)p.Bpk : (const void*)p.Bi;
    const float* Ax = VALUES ? p.Ax : nullptr;
    int buf = 0, pbuf = -1, pm = 0;
    for (long long c = e0; c < e1; c += stride) {
        const int nv = (int)(e1 - c < 32 ? e1 - c : 32);
        const Chunk ch = load_chunk(c, nv, p.Ai, Ax, p.nB, seg, err);
        const ChunkScan cs = scan_chunk(ch);
        for (int p0 = 0; p0 < cs.total; p0 += STAGE_P) {
            const int m = stage_issue(sa, buf, ch, cs, p0, src);
            if (pbuf >= 0) {
                cp_async_wait<1>();
                __syncwarp();
                process_window<VALUES>(sa, pbuf, pm, acc, flg, p.d, t * p.W, p.W, err);
            }
            pbuf = buf;
            pm = m;
            buf ^= 1;
        }
    }
    if (pbuf >= 0) {
        cp_async_wait<0>();
        __syncwarp();
        process_window<VALUES>(sa, pbuf, pm, acc, flg, p.d, t * p.W, p.W, err);
    }
}

template <bool VALUES>
__device__ __forceinline__ void staged_row_cta(const NumParams& p, const StageArea<VALUES ? 8 : 4>& sa, int row,
                                               long long a0, long long a1, float* acc, unsigned char* flg,
                                               int* wcnt) {
    unsigned long long* err = &p.hdr->err;
    long long out = clampll(__ldg(p.Cp + row), 0, p.nnzC);
    const long long out_end = clampll(__ldg(p.Cp + row + 1), out, p.nnzC);
    const long long first = a0 + 32LL * warp_id(), stride = 32LL * (blockDim.x >> 5);
    for (int t = 0; t < p.T; ++t) {
        if (p.T == 1) staged_range<VALUES>(p, sa, first, a1, stride, SegWhole{p.Bp, p.nnzB, p.d}, t, acc, flg);
        else staged_range<VALUES>(p, sa, first, a1, stride, SegTile{p.tp, p.T + 1, t, p.W}, t, acc, flg);
        __syncthreads();
        cta_emit<VALUES>(acc, flg, p.W, t * p.W, out, out_end, p.Ci, p.Cx, wcnt, err);
    }
    if (out != out_end && threadIdx.x == 0) atomicOr(err, ERR_C_ROW);
}

template <bool VALUES>
__device__ __forceinline__ void staged_split_part(const NumParams& p, const StageArea<VALUES ? 8 : 4>& sa,
                                                  const SplitItem& it, float* acc, unsigned char* flg, int* wcnt,
                                                  int* s_last) {
    unsigned long long* err = &p.hdr->err;
    float* sv = p.s.stg_vals + (size_t)it.slot * p.s.dpad;
    unsigned char* sf = p.s.stg_flags + (size_t)it.slot * p.s.dpad;
    const long long first = it.e0 + 32LL * warp_id(), stride = 32LL * (blockDim.x >> 5);
    for (int t = 0; t < p.T; ++t) {
        if (p.T == 1) staged_range<VALUES>(p, sa, first, it.e1, stride, SegWhole{p.Bp, p.nnzB, p.d}, t, acc, flg);
        else staged_range<VALUES>(p, sa, first, it.e1, stride, SegTile{p.tp, p.T + 1, t, p.W}, t, acc, flg);
        __syncthreads();
        for (int c = threadIdx.x; c < p.W; c += blockDim.x) {
            if (flg[c]) {
                if (VALUES) {
                    atomicAdd(sv + t * p.W + c, acc[c]);
                    acc[c] = 0.0f;
                }
                sf[t * p.W + c] = 1;
                flg[c] = 0;
            }
        }
        __syncthreads();
    }
    if (!split_part_done(p.s, it.slot, it.nsub, s_last)) return;
    split_row_readout<VALUES>(p, it, wcnt);
}

// Light rows of one warp: windows of consecutive rows flow through the two
// buffers; a row's read-out happens when its last window has been
// processed, while the next row's first window is already in flight.
template <bool VALUES>
__device__ __forceinline__ void staged_light_rows(const NumParams& p, const StageArea<VALUES ? 8 : 4>& sa,
                                                  float* acc, unsigned char* flg, long long idx0, long long end,
                                                  long long step, const long long* mark) {
    unsigned long long* err = &p.hdr->err;
    const void* src = VALUES ? (const void*)p.Bpk : (const void*)p.Bi;
    const float* Ax = VALUES ? p.Ax : nullptr;
    Pending pend;
    pend.row = -1;
    int buf = 0;
    long long out = 0, out_end = 0;  // read-out cursor of the row being processed
    int cur = -1;
    auto finish_pending = [&](bool all) {
        if (pend.row < 0) return;
        if (all) cp_async_wait<0>();
        else cp_async_wait<1>();
        __syncwarp();
        if (pend.row != cur) {
            cur = pend.row;
            out = pend.out;
            out_end = pend.out_end;
        }
        process_window<VALUES>(sa, pend.buf, pend.m, acc, flg, p.d, pend.tile * p.W, p.W, err);
        if (pend.last_of_tile) {
            __syncwarp();
            warp_emit4<VALUES>(acc, flg, p.W, pend.tile * p.W, out, out_end, p.Ci, p.Cx, err);
            __syncwarp();
            if (pend.last_of_row && out != out_end && lane_id() == 0) atomicOr(err, ERR_C_ROW);
        }
        pend.row = -1;
    };
    int nrow = idx0 < end ? __ldg(p.perm + idx0) : 0;
    for (long long idx = idx0; idx < end; idx += step) {
        const int row = nrow;
        if (idx + step < end) nrow = __ldg(p.perm + idx + step);  // one row ahead
        const long long a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
        const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
        if (mark && is_split_row(mark, row, a1 - a0)) continue;
        const long long o0 = clampll(__ldg(p.Cp + row), 0, p.nnzC);
        const long long o1 = clampll(__ldg(p.Cp + row + 1), o0, p.nnzC);
        for (int t = 0; t < p.T; ++t) {
            for (long long c = a0; c < a1; c += 32) {
                const int nv = (int)(a1 - c < 32 ? a1 - c : 32);
                const Chunk ch = (p.T == 1) ? load_chunk(c, nv, p.Ai, Ax, p.nB, SegWhole{p.Bp, p.nnzB, p.d}, err)
                                            : load_chunk(c, nv, p.Ai, Ax, p.nB, SegTile{p.tp, p.T + 1, t, p.W}, err);
                const ChunkScan cs = scan_chunk(ch);
                const bool last_chunk = c + 32 >= a1;
                int p0 = 0;
                do {  // an empty chunk still issues one (empty) window so that read-outs stay in order
                    const int m = stage_issue(sa, buf, ch, cs, p0, src);
                    const bool last_win = p0 + STAGE_P >= cs.total;
                    finish_pending(false);
                    pend = Pending{buf, m, row, t, last_chunk && last_win, last_chunk && last_win && t + 1 == p.T,
                                   o0, o1};
                    buf ^= 1;
                    p0 += STAGE_P;
                } while (p0 < cs.total);
            }
        }
    }
    finish_pending(true);
}

template <bool VALUES>
__global__ void __launch_bounds__(256, 4) k_numeric_staged(NumParams p) {
    constexpr int E = VALUES ? 8 : 4;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_wcnt[MAX_DENSE_W / 32 + 1];
    __shared__ long long s_item, s_nheavy, s_nrows;
    const int nw = blockDim.x >> 5, warp = warp_id(), tid = threadIdx.x;
    const int slot = VALUES ? 5 * p.W : p.W;
    // layout: [nw][slot] accumulators, then [nw] staging areas
    for (int i = tid; i < nw * slot / 4; i += blockDim.x) reinterpret_cast<unsigned*>(smem)[i] = 0u;
    const StageArea<E> sa{smem + (size_t)nw * slot + (size_t)warp * StageArea<E>::BYTES};
    if (tid < 32) {  // one warp; its lanes store the same values
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
        s_nrows = nr;
    }
    __syncthreads();
    const long long nheavy = s_nheavy, nrows = s_nrows;
    const bool split_ok = p.s.stg_vals != nullptr;
    const long long* mark = split_ok ? p.s.flops : nullptr;
    {
        float* acc = reinterpret_cast<float*>(smem);
        unsigned char* flg = smem + (VALUES ? 4 * p.W : 0);
        const long long nitems = split_ok ? min(*(volatile long long*)&p.hdr->scratch[2], p.item_cap) : 0;
        __shared__ int s_last;
        SplitItem it;
        while (next_split_item(p.s, p.Ap, p.nnzA, nitems, &s_item, it))
            staged_split_part<VALUES>(p, sa, it, acc, flg, s_wcnt, &s_last);
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
            staged_row_cta<VALUES>(p, sa, row, a0, a1, acc, flg, s_wcnt);
        }
    }
    float* acc = reinterpret_cast<float*>(smem + (size_t)warp * slot);
    unsigned char* flg = smem + (size_t)warp * slot + (VALUES ? 4 * p.W : 0);
    staged_light_rows<VALUES>(p, sa, acc, flg, nheavy + (long long)blockIdx.x * nw + warp, nrows,
                              (long long)gridDim.x * nw, mark);
}

size_t numeric_staged_smem(int W, int warps, bool values) {
    return numeric_dense_smem(W, warps, values) +
           (size_t)warps * (values ? StageArea<8>::BYTES : StageArea<4>::BYTES);
}

cudaError_t launch_numeric_staged(const DevCsr& A, const DevCsr& B, long long d, int W, int T,
                                  const long long* tp, bool values, const int2* Bpk, const Sched& s,
                                  const LaunchCfg& cfg, const long long* Cp, int* Ci, float* Cx, long long nnzC,
                                  cudaStream_t st) {
    cudaError_t e;
    if (A.nrows == 0) return cudaSuccess;
    if (W <= 0 || W % 32 || W > MAX_DENSE_W || (long long)W * T < d) return cudaErrorInvalidValue;
    if (cfg.warps_per_cta < 1 || cfg.warps_per_cta > 8) return cudaErrorInvalidValue;
    if (values && !Bpk && B.nnz > 0) return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(&s.hdr->heavy_ctr, 0, 2 * sizeof(unsigned long long), st))) return e;
    NumParams p = numeric_params(A, B, d, W, T, tp, Bpk, s, cfg, Cp, Ci, Cx, nnzC);
    const int warps = cfg.warps_per_cta;
    const size_t smem = numeric_staged_smem(W, warps, values);
    const void* k = values ? (const void*)k_numeric_staged<true> : (const void*)k_numeric_staged<false>;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    const int grid = persistent_grid(k, 32 * warps, smem, cfg.sms);
    void* args[] = {&p};
    count_launch();
    return cudaLaunchKernel(k, dim3(grid), dim3(32 * warps), args, smem, st);
}

}  // namespace ts
