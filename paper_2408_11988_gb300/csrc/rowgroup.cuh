// Device pieces of the row-group numeric kernels (numeric.cu), shared with
// the batched kernels: a slot of RG lanes owns one row and a private dense
// accumulator (empty columns hold RG_EMPTY), walks the row's segments of B on
// the row-aligned copy, and the warp reads its slots out one after another.
#pragma once

#include "common.cuh"
#include "numeric.cuh"
#include "wide.cuh"

namespace ts {

constexpr unsigned RG_EMPTY = 0xFFBADBADu;  // exponent all ones, quiet bit clear
static_assert((RG_EMPTY & 0x7F800000u) == 0x7F800000u && (RG_EMPTY & 0x00400000u) == 0 && (RG_EMPTY & 0x003FFFFFu),
              "RG_EMPTY must be a signalling NaN");

// acc[lc] += v, lc already checked against [0, W) and d.
__device__ __forceinline__ void rg_add(float* acc, int lc, float v) {
    const float old = acc[lc];
    acc[lc] = __float_as_uint(old) == RG_EMPTY ? v : old + v;
}

// Read-out of tile c0 of every slot (all lanes converged): the warp reads
// the slots out one after another, lane l taking column l of every 32-column
// stripe, so that each store instruction writes consecutive positions of one
// row of C (whole sectors) and a stripe's offsets come from one ballot.  A
// slot's output offsets are 32-bit (a row holds at most d entries); a row
// that would pass its end in C stores nothing more and is reported by the
// caller (out != out_end).
template <int RG>
__device__ __forceinline__ void rg_emit(float* racc, int W, int c0, long long& out, long long out_end, int* Ci,
                                        float* Cx, unsigned long long*) {
    constexpr int R = 32 / RG;
    const int lane = lane_id(), g = lane / RG;
    const unsigned lt = lanemask_lt();
#pragma unroll 1
    for (int h = 0; h < R; ++h) {
        const long long o0 = shfl64(out, h * RG), e0 = shfl64(out_end, h * RG);
        const long long r = e0 - o0;
        const int room = r < 0x7FFFFFFFLL ? (int)r : 0x7FFFFFFF;
        int* ci = Ci + o0;
        float* cx = Cx + o0;
        float* acc = racc + h * (W + 8);
        int o = 0;
#pragma unroll 4
        for (int base = 0; base < W; base += 32) {
            const int c = base + lane;
            const unsigned x = __float_as_uint(acc[c]);
            const bool take = x != RG_EMPTY;
            const unsigned bal = __ballot_sync(FULL, take);
            if (take) {
                const int pos = o + __popc(bal & lt);
                if (pos < room) {
                    ci[pos] = c0 + c;
                    cx[pos] = __uint_as_float(x);
                }
                acc[c] = __uint_as_float(RG_EMPTY);
            }
            o += __popc(bal);
        }
        if (g == h) out += o;
    }
}

// Column index and value of entry ei of A (k = -1 past the row's end).
__device__ __forceinline__ void rg_load_a(const NumParams& p, long long ei, bool ok, int& k, float& a) {
    k = -1;
    a = 0.0f;
    if (ok) {
        k = __ldg(p.Ai + ei);
        a = p.Ax ? __ldg(p.Ax + ei) : 1.0f;
    }
}

// Segment (first group, groups) of B's row k for entry k of A (empty when
// !ok; a bad k is an input error).
template <int E>
__device__ __forceinline__ void rgp_seg(const NumParams& p, int k, bool ok, unsigned& g0, int& ng,
                                        unsigned long long* err) {
    g0 = 0;
    ng = 0;
    if (!ok) return;
    if ((unsigned)k < (unsigned)p.nB) padded_seg<E>(p.Bp, p.nnzB, p.d, k, g0, ng);
    else atomicOr(err, ERR_A_COL);
}

// Group g of the copy (E = 2: one 16-byte load; E = 4: two).
template <int E>
__device__ __forceinline__ void rgp_load(const int4* __restrict__ Q, unsigned g, int4& v0, int4& v1) {
    v0 = __ldg(Q + (size_t)g * (E / 2));
    if constexpr (E == 4) v1 = __ldg(Q + (size_t)g * 2 + 1);
}

// How a slot adds a product into its accumulator.  AddPlain: the slot's own
// accumulator (row groups): a column outside [0, W) (a pad) goes to the
// spare column W.  (AddShared, one accumulator shared by several slots, is
// in wide.cuh.)
struct AddPlain {
    float* acc;
    __device__ __forceinline__ void operator()(int c, unsigned W, float v) const {
        rg_add(acc, (unsigned)c < W ? c : (int)W, v);
    }
};

template <int E, class Add>
__device__ __forceinline__ void rgp_apply(const Add& add, const int4& v0, const int4& v1, float a, unsigned W) {
    const int cs[4] = {v0.x, v0.z, v1.x, v1.z};
    const int bs[4] = {v0.y, v0.w, v1.y, v1.w};
#pragma unroll
    for (int u = 0; u < E; ++u) add(cs[u], W, a * __int_as_float(bs[u]));
}

// rg_tile on the row-aligned copy: chunks of RG entries of every slot's row,
// software-pipelined the same way (the next segment's description and first
// group load while the current segment is accumulated).  The caller has
// loaded the first two chunks of A (k0/x0: entry a0 + gl, k1/x1: entry
// a0 + RG + gl, as rg_load_a gives them).
template <int RG, int E, class Add>
__device__ __forceinline__ void rgp_tile(const NumParams& p, const int4* __restrict__ Q, const Add& acc, long long a0,
                                         int len, int lmax, unsigned long long* err, int k0, float x0, int k1,
                                         float x1) {
    const int lane = lane_id(), gl = lane % RG, src0 = (lane / RG) * RG;
    const unsigned W = (unsigned)p.W;
    unsigned g0;
    int n0;
    rgp_seg<E>(p, k0, gl < len, g0, n0, err);
    unsigned ng = __shfl_sync(FULL, g0, src0);
    int nn = __shfl_sync(FULL, n0, src0);
    float na = __shfl_sync(FULL, x0, src0);
    int4 v0 = make_int4(0, 0, 0, 0), v1 = make_int4(0, 0, 0, 0);
    if (gl < nn) rgp_load<E>(Q, ng + gl, v0, v1);
    for (int e = 0; e < lmax; e += RG) {
        int k2;
        float x2;
        unsigned g1;
        int n1;
        rg_load_a(p, a0 + e + 2 * RG + gl, e + 2 * RG + gl < len, k2, x2);
        rgp_seg<E>(p, k1, e + RG + gl < len, g1, n1, err);
        if (n1 > 0) prefetch_l2(Q + (size_t)g1 * (E / 2));  // the next chunk's rows of B into L2
        const int nu = lmax - e < RG ? lmax - e : RG;
        for (int u = 0; u < nu; ++u) {
            const unsigned cg = ng;
            const int cn = nn;
            const float ca = na;
            const int4 c0v = v0, c1v = v1;
            // describe and start loading the segment after this one (the
            // first of the next chunk after the last of this one)
            const bool more = u + 1 < nu;
            const int su = more ? src0 + u + 1 : src0;
            ng = __shfl_sync(FULL, more ? g0 : g1, su);
            nn = __shfl_sync(FULL, more ? n0 : n1, su);
            na = __shfl_sync(FULL, more ? x0 : x1, su);
            if (gl < nn) rgp_load<E>(Q, ng + gl, v0, v1);
            if (gl < cn) {
                rgp_apply<E>(acc, c0v, c1v, ca, W);
                for (int q = gl + RG; q < cn; q += RG) {
                    int4 w0, w1;
                    rgp_load<E>(Q, cg + q, w0, w1);
                    rgp_apply<E>(acc, w0, w1, ca, W);
                }
            }
            __syncwarp();
        }
        g0 = g1;
        n0 = n1;
        x0 = x1;
        k1 = k2;
        x1 = x2;
    }
}

// Column c of the S slots summed (RG_EMPTY if no slot reached it); every
// slot's column is reset.  Called by one thread per column after a barrier.
__device__ __forceinline__ unsigned rgcta_sum(float* racc, int ld, int S, int c) {
    unsigned x = RG_EMPTY;
#pragma unroll 8
    for (int k = 0; k < S; ++k) {
        float* a = racc + (size_t)k * ld + c;
        const unsigned y = __float_as_uint(*a);
        if (y != RG_EMPTY) {
            x = x == RG_EMPTY ? y : __float_as_uint(__uint_as_float(x) + __uint_as_float(y));
            *a = __uint_as_float(RG_EMPTY);
        }
    }
    return x;
}

// Block-wide read-out of a heavy row's tile from the summed columns held in
// sum[0..W) (reset to RG_EMPTY); wcnt has W/32 + 1 entries.
__device__ __forceinline__ void rgcta_emit(float* sum, int W, int c0, long long& out, long long out_end, int* Ci,
                                           float* Cx, int* wcnt, unsigned long long* err) {
    const int nw = blockDim.x >> 5, warp = warp_id(), lane = lane_id();
    const int words = W >> 5;
    const unsigned lt = lanemask_lt();
    for (int w = warp; w < words; w += nw) {
        const unsigned bal = __ballot_sync(FULL, __float_as_uint(sum[w * 32 + lane]) != RG_EMPTY);
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
        const unsigned x = __float_as_uint(sum[c]);
        const bool f = x != RG_EMPTY;
        const unsigned bal = __ballot_sync(FULL, f);
        if (f) {
            const long long pos = out + wcnt[w] + __popc(bal & lt);
            if (pos < out_end) {
                Ci[pos] = c0 + c;
                Cx[pos] = __uint_as_float(x);
            } else {
                atomicOr(err, ERR_C_ROW);
            }
            sum[c] = __uint_as_float(RG_EMPTY);
        }
    }
    out += wcnt[words];
    __syncthreads();
}

}  // namespace ts
