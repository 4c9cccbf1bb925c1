// Pieces shared by the dense-accumulator numeric kernels (numeric.cu and
// numeric_copies.cu): the kernel parameters, their set-up from the launch
// arguments, and the read-out of a split row from its staging slot.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace ts {

constexpr int MAX_DENSE_W = 4096;

struct NumParams {
    const long long* Ap;
    const int* Ai;
    const float* Ax;
    long long nnzA;
    const long long* Bp;
    const int* Bi;
    const float* Bx;
    const int2* Bpk;
    const int4* Bq;  // row-aligned packed copy of B (T = 1, row-group kernels) or nullptr
    long long nnzB;
    int nB;
    int d;
    int W;
    int T;
    const long long* tp;
    const int* perm;
    WsHeader* hdr;
    int cta_class;
    const long long* Cp;
    int* Ci;
    float* Cx;
    long long nnzC;
    Sched s;
    long long item_cap;
    int skip_light;  // 1: split and heavy rows only (light rows run in a kernel of their own)
    int tiny_max;    // wide kernel: light rows with at most this many products run in k_numeric_tiny
};

// Light rows with at most TINY_MAX products go to the tiny-row kernel (one
// product per lane): exactly the flops classes 1 .. TINY_CLASS, the tail of
// the class order, which the row-group light kernel then stops short of.
constexpr int TINY_MAX = 31;
constexpr int TINY_CLASS = 40;  // flops class of 31 products; 32 start class 41

inline NumParams numeric_params(const DevCsr& A, const DevCsr& B, long long d, int W, int T,
                                const long long* tp, const int2* Bpk, const Sched& s, const LaunchCfg& cfg,
                                const long long* Cp, int* Ci, float* Cx, long long nnzC) {
    NumParams p;
    p.Ap = A.rowptr;
    p.Ai = A.col;
    p.Ax = A.val;
    p.nnzA = A.nnz;
    p.Bp = B.rowptr;
    p.Bi = B.col;
    p.Bx = B.val;
    p.Bpk = Bpk;
    p.Bq = nullptr;
    p.nnzB = B.nnz;
    p.nB = (int)B.nrows;
    p.d = (int)d;
    p.W = W;
    p.T = T;
    p.tp = tp;
    p.perm = s.perm;
    p.hdr = s.hdr;
    p.cta_class = cfg.cta_class;
    p.Cp = Cp;
    p.Ci = Ci;
    p.Cx = Cx;
    p.nnzC = nnzC;
    p.s = s;
    p.item_cap = split_item_capacity(A.nnz);
    p.skip_light = 0;
    p.tiny_max = 0;
    return p;
}

// The block that completed the last part of a split row reads the row out of
// its staging slot (values and occupancy flags, all dpad columns) in
// ascending column order and clears the slot; wcnt has dpad/32 + 1 entries.
template <bool VALUES>
__device__ __forceinline__ void split_row_readout(const NumParams& p, const SplitItem& it, int* wcnt) {
    unsigned long long* err = &p.hdr->err;
    float* sv = p.s.stg_vals + (size_t)it.slot * p.s.dpad;
    unsigned char* sf = p.s.stg_flags + (size_t)it.slot * p.s.dpad;
    const int nw = blockDim.x >> 5, warp = warp_id(), lane = lane_id();
    const int words = p.s.dpad >> 5;
    const unsigned lt = lanemask_lt();
    long long out = clampll(__ldg(p.Cp + it.row), 0, p.nnzC);
    const long long out_end = clampll(__ldg(p.Cp + it.row + 1), out, p.nnzC);
    for (int w = warp; w < words; w += nw) {
        const unsigned bal = __ballot_sync(FULL, __ldcg(sf + w * 32 + lane) != 0);
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
        const bool f = __ldcg(sf + c) != 0;
        const unsigned bal = __ballot_sync(FULL, f);
        if (f) {
            const long long pos = out + wcnt[w] + __popc(bal & lt);
            if (pos < out_end) {
                p.Ci[pos] = c;
                if (VALUES) p.Cx[pos] = __ldcg(sv + c);
            } else {
                atomicOr(err, ERR_C_ROW);
            }
            if (VALUES) sv[c] = 0.0f;
            sf[c] = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (out + wcnt[words] != out_end) atomicOr(err, ERR_C_ROW);
        p.s.split_done[it.slot] = 0;
    }
    __syncthreads();
}

}  // namespace ts
