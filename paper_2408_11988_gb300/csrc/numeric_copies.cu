// Numeric pass (plus-times) with per-group copies of the dense accumulator
// and no atomic operations.
//
// The dense accumulator is the paper's SPA (Sec. III-C): W floats per column
// tile.  A warp's lanes form NG = 32/G groups of G lanes and every group owns
// a private copy of the accumulator.  A group walks one segment of B (the
// row B(k,:) of one entry A(i,k), inside the current column tile) at a time,
// G entries of the segment per instruction.  B's rows hold strictly ascending
// columns, so the lanes of one group never touch the same column in one
// instruction, and lanes of different groups touch different copies: the
// update acc[c] += A(i,k) * B(k,c) is a plain load and store.  Between two
// segments the warp synchronises (__syncwarp), which orders one lane's store
// before another lane's load of the same column.  A column that no product
// reached holds PC_EMPTY, a signalling-NaN bit pattern: arithmetic never
// delivers a signalling NaN (a NaN result is quiet), so no product or sum
// carries it and no occupancy flags are kept.
//
// At the end of a row the copies are combined column by column in a fixed
// order (copy 0 first), the reached columns are written to C in ascending
// order and the copies are reset to PC_EMPTY.  Rows taken by a whole block
// (heavy rows, parts of split rows) use one copy set per warp and combine
// all warps' copies the same way, so that no atomic is needed anywhere but
// in the staging of split rows.  Row i of C is the same set of columns with
// the same sums as Eq. (1); only the FP32 summation order differs.
#include "common.cuh"
#include "kernels.h"
#include "numeric.cuh"

namespace ts {

constexpr unsigned PC_EMPTY = 0xFFBADBADu;  // "no product yet": exponent all ones, quiet bit clear
static_assert((PC_EMPTY & 0x7F800000u) == 0x7F800000u && (PC_EMPTY & 0x00400000u) == 0 && (PC_EMPTY & 0x003FFFFFu),
              "PC_EMPTY must be a signalling NaN");

// Segment of B of one entry of A, as a group reads it.
struct PcMeta {
    long long start;
    int len;
    float a;
};
static_assert(sizeof(PcMeta) == 16, "PcMeta is one 16-byte shared-memory word");

// Shared-memory bytes of one warp: NG copies of W floats, then 32 PcMeta.
__host__ __device__ constexpr size_t pc_warp_bytes(int W, int NG) { return (size_t)NG * W * 4 + 32 * 16; }

__device__ __forceinline__ unsigned f2u(float x) { return __float_as_uint(x); }
__device__ __forceinline__ float u2f(unsigned x) { return __uint_as_float(x); }

// acc[c - c0] += v in one copy (cp), no atomic; columns outside [c0, c0+W)
// or [0, d) are input errors.
__device__ __forceinline__ void pc_add(float* cp, int c, float v, int d, int c0, int W,
                                       unsigned long long* err) {
    const int lc = c - c0;
    if ((unsigned)c < (unsigned)d && (unsigned)lc < (unsigned)W) {
        const float old = cp[lc];
        cp[lc] = f2u(old) == PC_EMPTY ? v : old + v;
    } else {
        atomicOr(err, ERR_B_COL);
    }
}

// Accumulate the products of one loaded chunk (up to 32 entries of A; lane q
// holds entry q) into this warp's copies.  Entries are taken in rounds of
// NG * U: group g takes entries r + u*NG + g (u < U), so every lane has U
// gathers in flight.  tab: this warp's 32 PcMeta.
template <int G, int U, class BA>
__device__ __forceinline__ void pc_chunk(const Chunk& ch, int nv, PcMeta* tab, float* cps, const BA& ba, int d,
                                         int c0, int W, unsigned long long* err) {
    constexpr int NG = 32 / G;
    static_assert(32 % (NG * U) == 0, "a round must divide the chunk");
    const int lane = lane_id(), gi = lane / G, gl = lane % G;
    float* cp = cps + gi * W;
    __syncwarp();  // earlier readers of tab are done
    tab[lane] = PcMeta{ch.start, lane < nv ? ch.len : 0, ch.a};
    __syncwarp();
    for (int r = 0; r < nv; r += NG * U) {
        PcMeta m[U];
        int lmax = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            m[u] = tab[r + u * NG + gi];  // index <= 31: r + NG*U <= 32
            lmax = m[u].len > lmax ? m[u].len : lmax;
        }
        lmax = (int)__reduce_max_sync(FULL, (unsigned)lmax);
        for (int base = 0; base < lmax; base += G) {
            const int off = base + gl;
            int c[U];
            float b[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                c[u] = -1;
                b[u] = 0.0f;
                if (off < m[u].len) ba.get(m[u].start + off, c[u], b[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (off < m[u].len) pc_add(cp, c[u], m[u].a * b[u], d, c0, W, err);
                __syncwarp();  // the next segment may hold the same columns
            }
        }
    }
}

// Warp read-out of a light row's tile: lane l combines columns 4l..4l+3 of
// every 128-column block over the NG copies, resets them, and writes the
// reached columns in ascending order from position `out`.
template <int NG>
__device__ __forceinline__ void pc_warp_emit(float* cps, int W, int c0, long long& out, long long out_end,
                                             int* Ci, float* Cx, unsigned long long* err) {
    const int lane = lane_id();
    for (int base = 0; base < W; base += 128) {
        const int cb = base + 4 * lane;
        unsigned v[4] = {PC_EMPTY, PC_EMPTY, PC_EMPTY, PC_EMPTY};
        if (cb < W) {
#pragma unroll
            for (int k = 0; k < NG; ++k) {
                uint4* q = reinterpret_cast<uint4*>(cps + k * W + cb);
                const uint4 x = *q;
                const unsigned xs[4] = {x.x, x.y, x.z, x.w};
                bool any = false;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (xs[i] != PC_EMPTY) {
                        any = true;
                        v[i] = v[i] == PC_EMPTY ? xs[i] : f2u(u2f(v[i]) + u2f(xs[i]));
                    }
                }
                if (any) *q = make_uint4(PC_EMPTY, PC_EMPTY, PC_EMPTY, PC_EMPTY);
            }
        }
        unsigned f = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) f |= (v[i] != PC_EMPTY ? 1u : 0u) << i;
        const int cnt = __popc(f);
        const int incl = warp_incl_scan(cnt);
        long long pos = out + incl - cnt;
        out += __shfl_sync(FULL, incl, 31);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (f & (1u << i)) {
                if (pos < out_end) {
                    Ci[pos] = c0 + cb + i;
                    Cx[pos] = u2f(v[i]);
                } else {
                    atomicOr(err, ERR_C_ROW);
                }
                ++pos;
            }
        }
    }
}

// Block rows: combine the copies of all warps into copy 0 of warp 0 (thread
// per column, fixed order) and reset the others.  Called after __syncthreads.
template <int NG>
__device__ __forceinline__ void pc_cta_merge(unsigned char* smem, size_t wbytes, int W) {
    const int nw = blockDim.x >> 5;
    float* c00 = reinterpret_cast<float*>(smem);
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
        unsigned v = f2u(c00[c]);
        for (int w = 0; w < nw; ++w) {
#pragma unroll
            for (int k = 0; k < NG; ++k) {
                if (w == 0 && k == 0) continue;
                float* cp = reinterpret_cast<float*>(smem + (size_t)w * wbytes) + k * W;
                const unsigned x = f2u(cp[c]);
                if (x != PC_EMPTY) {
                    v = v == PC_EMPTY ? x : f2u(u2f(v) + u2f(x));
                    cp[c] = u2f(PC_EMPTY);
                }
            }
        }
        c00[c] = u2f(v);
    }
}

// Block read-out of the combined copy (c00) into C from `out`, ascending;
// resets c00.  wcnt has W/32 + 1 entries.
__device__ __forceinline__ void pc_cta_emit(float* c00, int W, int c0, long long& out, long long out_end, int* Ci,
                                            float* Cx, int* wcnt, unsigned long long* err) {
    const int nw = blockDim.x >> 5, warp = warp_id(), lane = lane_id();
    const int words = W >> 5;
    const unsigned lt = lanemask_lt();
    for (int w = warp; w < words; w += nw) {
        const unsigned bal = __ballot_sync(FULL, f2u(c00[w * 32 + lane]) != PC_EMPTY);
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
        const unsigned x = f2u(c00[c]);
        const bool f = x != PC_EMPTY;
        const unsigned bal = __ballot_sync(FULL, f);
        if (f) {
            const long long pos = out + wcnt[w] + __popc(bal & lt);
            if (pos < out_end) {
                Ci[pos] = c0 + c;
                Cx[pos] = u2f(x);
            } else {
                atomicOr(err, ERR_C_ROW);
            }
            c00[c] = u2f(PC_EMPTY);
        }
    }
    out += wcnt[words];
    __syncthreads();
}

// Entries [a0, a1) of A for tile t, spread over the block's warps in chunks
// of 32 (warp w takes chunks w, w + nw, ...), each warp into its own copies.
template <int G, int U, class BA, class Seg>
__device__ __forceinline__ void pc_block_range(const NumParams& p, const BA& ba, const Seg& seg, long long a0,
                                               long long a1, int c0, unsigned char* wsm) {
    unsigned long long* err = &p.hdr->err;
    constexpr int NG = 32 / G;
    float* cps = reinterpret_cast<float*>(wsm);
    PcMeta* tab = reinterpret_cast<PcMeta*>(wsm + (size_t)NG * p.W * 4);
    const int nw = blockDim.x >> 5;
    for (long long e0 = a0 + 32LL * warp_id(); e0 < a1; e0 += 32LL * nw) {
        const int nv = (int)(a1 - e0 < 32 ? a1 - e0 : 32);
        const Chunk ch = load_chunk(e0, nv, p.Ai, p.Ax, p.nB, seg, err);
        pc_chunk<G, U>(ch, nv, tab, cps, ba, p.d, c0, p.W, err);
    }
}

template <int G, int U, class BA>
__device__ __forceinline__ void pc_block_tile(const NumParams& p, const BA& ba, int t, long long a0, long long a1,
                                              unsigned char* wsm) {
    if (p.T == 1) pc_block_range<G, U>(p, ba, SegWhole{p.Bp, p.nnzB, p.d}, a0, a1, 0, wsm);
    else pc_block_range<G, U>(p, ba, SegTile{p.tp, p.T + 1, t, p.W}, a0, a1, t * p.W, wsm);
}

// Heavy row: the whole block works on one row.
template <int G, int U, class BA>
__device__ __forceinline__ void pc_row_cta(const NumParams& p, const BA& ba, int row, unsigned char* smem,
                                           size_t wbytes, int* wcnt) {
    unsigned long long* err = &p.hdr->err;
    const long long a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
    const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
    long long out = clampll(__ldg(p.Cp + row), 0, p.nnzC);
    const long long out_end = clampll(__ldg(p.Cp + row + 1), out, p.nnzC);
    for (int t = 0; t < p.T; ++t) {
        pc_block_tile<G, U>(p, ba, t, a0, a1, smem + (size_t)warp_id() * wbytes);
        __syncthreads();
        pc_cta_merge<32 / G>(smem, wbytes, p.W);
        __syncthreads();
        pc_cta_emit(reinterpret_cast<float*>(smem), p.W, t * p.W, out, out_end, p.Ci, p.Cx, wcnt, err);
    }
    if (out != out_end && threadIdx.x == 0) atomicOr(err, ERR_C_ROW);
}

// One part of a split row: combined tile sums are added into the row's
// staging slot; the block completing the last part reads the row out.
template <int G, int U, class BA>
__device__ __forceinline__ void pc_split_part(const NumParams& p, const BA& ba, const SplitItem& it,
                                              unsigned char* smem, size_t wbytes, int* wcnt, int* s_last) {
    float* sv = p.s.stg_vals + (size_t)it.slot * p.s.dpad;
    unsigned char* sf = p.s.stg_flags + (size_t)it.slot * p.s.dpad;
    float* c00 = reinterpret_cast<float*>(smem);
    for (int t = 0; t < p.T; ++t) {
        pc_block_tile<G, U>(p, ba, t, it.e0, it.e1, smem + (size_t)warp_id() * wbytes);
        __syncthreads();
        pc_cta_merge<32 / G>(smem, wbytes, p.W);
        __syncthreads();
        for (int c = threadIdx.x; c < p.W; c += blockDim.x) {
            const unsigned x = f2u(c00[c]);
            if (x != PC_EMPTY) {
                atomicAdd(sv + t * p.W + c, u2f(x));
                sf[t * p.W + c] = 1;
                c00[c] = u2f(PC_EMPTY);
            }
        }
        __syncthreads();
    }
    if (!split_part_done(p.s, it.slot, it.nsub, s_last)) return;
    split_row_readout<true>(p, it, wcnt);
}

// Light row, one warp, driven by pipelined_rows (same contract as the
// flag-based kernel's row body).
template <int G, int U, class BA>
struct PcRowBody {
    const NumParams& p;
    const BA& ba;
    float* cps;
    PcMeta* tab;
    unsigned long long* err;
    long long out, out_end;
    __device__ __forceinline__ void gather(int row, long long a0, long long a1, const Chunk& ch0, int nv0, int) {
        out = clampll(__ldg(p.Cp + row), 0, p.nnzC);
        out_end = clampll(__ldg(p.Cp + row + 1), out, p.nnzC);
        for (int t = 0; t < p.T; ++t) {
            long long e_next = a0;
            if (t == 0) {
                pc_chunk<G, U>(ch0, nv0, tab, cps, ba, p.d, 0, p.W, err);
                e_next = a0 + 32;
            }
            if (p.T == 1) {
                const SegWhole seg{p.Bp, p.nnzB, p.d};
                for (long long e0 = e_next; e0 < a1; e0 += 32) {
                    const int nv = (int)(a1 - e0 < 32 ? a1 - e0 : 32);
                    pc_chunk<G, U>(load_chunk(e0, nv, p.Ai, p.Ax, p.nB, seg, err), nv, tab, cps, ba, p.d, 0, p.W,
                                   err);
                }
            } else {
                const SegTile seg{p.tp, p.T + 1, t, p.W};
                for (long long e0 = e_next; e0 < a1; e0 += 32) {
                    const int nv = (int)(a1 - e0 < 32 ? a1 - e0 : 32);
                    pc_chunk<G, U>(load_chunk(e0, nv, p.Ai, p.Ax, p.nB, seg, err), nv, tab, cps, ba, p.d, t * p.W,
                                   p.W, err);
                }
                if (t + 1 < p.T) {  // the last tile is read out by finish()
                    __syncwarp();
                    pc_warp_emit<32 / G>(cps, p.W, t * p.W, out, out_end, p.Ci, p.Cx, err);
                    __syncwarp();
                }
            }
        }
    }
    __device__ __forceinline__ void finish(int) {
        __syncwarp();
        pc_warp_emit<32 / G>(cps, p.W, (p.T - 1) * p.W, out, out_end, p.Ci, p.Cx, err);
        __syncwarp();
        if (out != out_end && lane_id() == 0) atomicOr(err, ERR_C_ROW);
    }
};

template <int G, int U, bool PACKED>
__global__ void __launch_bounds__(256, (G == 32 ? 3 : 4)) k_numeric_copies(NumParams p) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_wcnt[MAX_DENSE_W / 32 + 1];
    __shared__ long long s_item, s_nheavy, s_nrows;
    __shared__ int s_last;
    constexpr int NG = 32 / G;
    const int nw = blockDim.x >> 5, warp = warp_id(), tid = threadIdx.x;
    const size_t wbytes = pc_warp_bytes(p.W, NG);
    for (size_t i = tid; i < nw * wbytes / 4; i += blockDim.x) reinterpret_cast<unsigned*>(smem)[i] = PC_EMPTY;
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
    else ba = BSep{p.Bi, p.Bx};
    // without a staging area split rows are processed whole like any other row
    const bool split_ok = p.s.stg_vals != nullptr;
    const long long* mark = split_ok ? p.s.flops : nullptr;
    {
        const long long nitems = split_ok ? min(*(volatile long long*)&p.hdr->scratch[2], p.item_cap) : 0;
        SplitItem it;
        while (next_split_item(p.s, p.Ap, p.nnzA, nitems, &s_item, it))
            pc_split_part<G, U, BA>(p, ba, it, smem, wbytes, s_wcnt, &s_last);
        for (;;) {
            if (tid == 0) s_item = (long long)atomicAdd(&p.hdr->heavy_ctr, 1ull);
            __syncthreads();
            const long long h = s_item;
            __syncthreads();
            if (h >= nheavy) break;
            const int row = p.perm[h];
            if (mark && is_split_row(mark, row, __ldg(p.Ap + row + 1) - __ldg(p.Ap + row))) continue;
            pc_row_cta<G, U, BA>(p, ba, row, smem, wbytes, s_wcnt);
        }
    }
    if (p.skip_light) return;
    unsigned char* wsm = smem + (size_t)warp * wbytes;
    PcRowBody<G, U, BA> body{p, ba, reinterpret_cast<float*>(wsm),
                             reinterpret_cast<PcMeta*>(wsm + (size_t)NG * p.W * 4), &p.hdr->err, 0, 0};
    const long long idx0 = nheavy + (long long)blockIdx.x * nw + warp;
    const long long step = (long long)gridDim.x * nw;
    if (p.T == 1)
        pipelined_rows(p.perm, idx0, nrows, step, p.Ap, p.nnzA, p.Ai, p.Ax, p.nB, SegWhole{p.Bp, p.nnzB, p.d},
                       &p.hdr->err, body, mark);
    else
        pipelined_rows(p.perm, idx0, nrows, step, p.Ap, p.nnzA, p.Ai, p.Ax, p.nB,
                       SegTile{p.tp, p.T + 1, 0, p.W}, &p.hdr->err, body, mark);
}

size_t numeric_copies_smem(int W, int G, int warps) {
    if (G != 8 && G != 16 && G != 32) return 0;
    return (size_t)warps * pc_warp_bytes(W, 32 / G);
}

template <int G, bool PACKED>
static cudaError_t launch_pc(const NumParams& p, int warps, int sms, cudaStream_t st) {
    constexpr int U = G == 32 ? 4 : 2;
    const void* k = (const void*)k_numeric_copies<G, U, PACKED>;
    const size_t smem = numeric_copies_smem(p.W, G, warps);
    cudaError_t e;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    const int grid = persistent_grid(k, 32 * warps, smem, sms);
    count_launch();
    k_numeric_copies<G, U, PACKED><<<grid, 32 * warps, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_numeric_copies(const DevCsr& A, const DevCsr& B, long long d, int W, int T,
                                  const long long* tp, const int2* Bpk, int G, const Sched& s,
                                  const LaunchCfg& cfg, const long long* Cp, int* Ci, float* Cx, long long nnzC,
                                  cudaStream_t st, bool skip_light) {
    cudaError_t e;
    if (A.nrows == 0) return cudaSuccess;
    if (W <= 0 || W % 32 || W > MAX_DENSE_W || (long long)W * T < d) return cudaErrorInvalidValue;
    if (cfg.warps_per_cta < 1 || cfg.warps_per_cta > 8) return cudaErrorInvalidValue;
    const size_t smem = numeric_copies_smem(W, G, cfg.warps_per_cta);
    if (smem == 0 || smem > 227 * 1024) return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(&s.hdr->heavy_ctr, 0, 2 * sizeof(unsigned long long), st))) return e;
    NumParams p = numeric_params(A, B, d, W, T, tp, Bpk, s, cfg, Cp, Ci, Cx, nnzC);
    p.skip_light = skip_light ? 1 : 0;
    const int w = cfg.warps_per_cta, sms = cfg.sms;
    switch (G) {
        case 8: return Bpk ? launch_pc<8, true>(p, w, sms, st) : launch_pc<8, false>(p, w, sms, st);
        case 16: return Bpk ? launch_pc<16, true>(p, w, sms, st) : launch_pc<16, false>(p, w, sms, st);
        case 32: return Bpk ? launch_pc<32, true>(p, w, sms, st) : launch_pc<32, false>(p, w, sms, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ts
