// Backward of C = A*B (plus-times) with fixed patterns, for L = <dC, C>:
//   dA(i,k) = sum over j in B_k of dC(i,j) * B(k,j)        (SDDMM on A's pattern)
//   dB(k,j) = sum over i with (i,k) in A of A(i,k) * dC(i,j) (A^T dC on B's pattern)
// Both are computed in one traversal with the forward's schedule: row i of dC
// is scattered into a dense shared-memory row g (width d), then every product
// (k, j) of row i reads g[B.col[j]] once: the dot products for dA are reduced
// across lanes, and the dB terms are added to dB[j] with float atomics.
#include "common.cuh"
#include "kernels.h"

namespace ts {

constexpr int MAX_BWD_D = 8192;

struct BwdParams {
    const long long* Ap;
    const int* Ai;
    const float* Ax;
    long long nnzA;
    const long long* Bp;
    const int* Bi;
    const float* Bx;
    const int2* Bpk;
    long long nnzB;
    int nB;
    int d;
    int dpad;
    const long long* Cp;
    const int* Ci;
    const float* dC;
    long long nnzC;
    float* dA;
    float* dB;
    const int* perm;
    WsHeader* hdr;
    int cta_class;
    Sched s;
    long long item_cap;
    int skip_light;  // 1: split and heavy rows only (light rows run in k_backward_light)
    int tiny;        // 1: light rows of classes <= BWD_TINY_CLASS run in k_backward_tiny
};

// Rows with at most 31 products (flops classes 1 .. 40) are the backward's
// tiny rows when k_backward_tiny runs.
constexpr int BWD_TINY_CLASS = 40;

// Sum of v over the run of equal keys that starts at this lane (keys are
// non-decreasing across lanes); only a run's first lane's result is used.
__device__ __forceinline__ float seg_sum_down(float v, int key) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_down_sync(FULL, v, o);
        const int k = __shfl_down_sync(FULL, key, o);
        if (lane + o < 32 && k == key) v += t;
    }
    return v;
}

template <class BA>
struct BwdOp {
    BA ba;
    const float* g;
    float* sdA;  // flattened mode: 32 partial dot products of this warp's chunk
    float* dA;   // grouped mode: written directly
    float* dB;
    bool want_dA;
    int d;
    unsigned long long* err;
    float part[2];  // grouped mode: this lane's share of the two entries in flight
    struct Item {
        int c;
        float b;
    };
    __device__ __forceinline__ Item fetch(long long j) const {
        Item it;
        ba.get(j, it.c, it.b);
        return it;
    }
    // dB(k,j) += A(i,k) * dC(i,j); returns B(k,j) * dC(i,j) for dA(i,k)
    __device__ __forceinline__ float term(const Item& it, float a, long long j) {
        if ((unsigned)it.c < (unsigned)d) {
            const float gj = g[it.c];
            if (dB) atomicAdd(dB + j, a * gj);
            return it.b * gj;
        }
        atomicOr(err, ERR_B_COL);
        return 0.0f;
    }
    __device__ __forceinline__ void apply(const Item& it, float a, long long j, int slot) {
        part[slot] += term(it, a, j);
    }
    template <int G>
    __device__ __forceinline__ void done(int q0, int q1, int nvalid, long long e0) {
        float t0 = part[0], t1 = part[1];
#pragma unroll
        for (int o = G / 2; o >= 1; o >>= 1) {
            t0 += __shfl_xor_sync(FULL, t0, o);
            t1 += __shfl_xor_sync(FULL, t1, o);
        }
        if (want_dA && (lane_id() % G) == 0) {
            if (q0 < nvalid) dA[e0 + q0] = t0;
            if (q1 < nvalid) dA[e0 + q1] = t1;
        }
        part[0] = part[1] = 0.0f;
    }
    // flattened mode (expand_chunk): segmented lane reduction into sdA
    __device__ __forceinline__ void reduce_into(float contrib, int q, bool ok) {
        if (!want_dA) return;
        const float s = seg_sum_down(contrib, q);
        const int prevq = __shfl_up_sync(FULL, q, 1);
        if (ok && (lane_id() == 0 || prevq != q)) atomicAdd(sdA + q, s);
    }
    __device__ __forceinline__ void step4(const long long* j, const float* a, const int* q) {
        Item it[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) it[u] = fetch(j[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) reduce_into(term(it[u], a[u], j[u]), q[u], true);
    }
    __device__ __forceinline__ void step1(long long j, float a, int q, bool ok) {
        float c = 0.0f;
        if (ok) c = term(fetch(j), a, j);
        reduce_into(c, q, ok);
    }
};

// dC row i scattered into the dense row g (or cleared again).
__device__ __forceinline__ void scatter_dc(const BwdParams& p, long long c0, long long c1, float* g, bool clear,
                                           int tid, int nthr, unsigned long long* err) {
    for (long long e = c0 + tid; e < c1; e += nthr) {
        const int c = __ldg(p.Ci + e);
        if ((unsigned)c < (unsigned)p.d) g[c] = clear ? 0.0f : __ldg(p.dC + e);
        else if (!clear) atomicOr(err, ERR_C_ROW);
    }
}

// Quad mode (G = 2): a group of four lanes takes one entry A(i,k) and walks
// B's row k four consecutive entries per lane, starting at the multiple of
// four at or below the row's first entry, with two 16-byte loads of the
// packed copy (padded by four entries at its end).  The four dB terms of a
// lane go out as one 16-byte float atomic; entries of the quad outside the
// row add 0.  dB must be 16-byte aligned (the launcher checks it).
__device__ __forceinline__ void bwd_quads(const BwdParams& p, const Chunk& ch, int nv, long long e0, const float* g,
                                          unsigned long long* err) {
    const int lane = lane_id(), gi = lane >> 2, gl = lane & 3;
    const int4* P4 = reinterpret_cast<const int4*>(p.Bpk);  // two packed entries per int4
    for (int r = 0; r < nv; r += 8) {
        const int q = r + gi;  // <= 31
        const long long s = shfl64(ch.start, q);
        const int L = __shfl_sync(FULL, ch.len, q);
        const float a = __shfl_sync(FULL, ch.a, q);
        const long long base = s & ~3LL, end = s + L;
        const int nq = L > 0 ? (int)((end - base + 3) >> 2) : 0;
        float part = 0.0f;
        for (int t = gl; t < nq; t += 4) {
            const long long qb = base + 4LL * t;
            const int4 v0 = __ldg(P4 + (qb >> 1)), v1 = __ldg(P4 + (qb >> 1) + 1);
            const int cs[4] = {v0.x, v0.z, v1.x, v1.z};
            const int bs[4] = {v0.y, v0.w, v1.y, v1.w};
            float t4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                t4[u] = 0.0f;
                if (qb + u >= s && qb + u < end) {
                    const int c = cs[u];
                    if ((unsigned)c < (unsigned)p.d) {
                        const float gc = g[c];
                        t4[u] = a * gc;
                        part += __int_as_float(bs[u]) * gc;
                    } else {
                        atomicOr(err, ERR_B_COL);
                    }
                }
            }
            if (p.dB) {
                if (qb + 4 <= p.nnzB) {
                    atomicAdd(reinterpret_cast<float4*>(p.dB + qb), make_float4(t4[0], t4[1], t4[2], t4[3]));
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (qb + u >= s && qb + u < end) atomicAdd(p.dB + qb + u, t4[u]);
                }
            }
        }
        part += __shfl_xor_sync(FULL, part, 1);
        part += __shfl_xor_sync(FULL, part, 2);
        if (p.dA && gl == 0 && q < nv) p.dA[e0 + q] = part;
    }
}

// Products of one chunk, with the flattened-mode dA write-back.
template <int G, class BA>
__device__ __forceinline__ void bwd_chunk(const BwdParams& p, const Chunk& ch, int nv, long long e0, BwdOp<BA>& op,
                                          float* sdA) {
    if constexpr (G == 2) {
        bwd_quads(p, ch, nv, e0, op.g, op.err);
    } else if constexpr (G == 1) {
        expand_loaded(ch, op);
        __syncwarp();
        if (p.dA) {
            const int lane = lane_id();
            if (lane < nv) p.dA[e0 + lane] = sdA[lane];
            sdA[lane] = 0.0f;
            __syncwarp();
        }
    } else {
        grouped_loaded<G>(ch, nv, e0, op);
    }
}

// Heavy row or one part [a0, a1) of a split row: the whole block works on it.
// The parts of a split row are independent: each writes dA of its own
// entries and adds its dB terms.
template <int G, class BA>
__device__ __forceinline__ void backward_range_cta(const BwdParams& p, const BA& ba, int row, long long a0,
                                                   long long a1, float* g, float* sdA) {
    unsigned long long* err = &p.hdr->err;
    const long long c0 = clampll(__ldg(p.Cp + row), 0, p.nnzC);
    const long long c1 = clampll(__ldg(p.Cp + row + 1), c0, p.nnzC);
    scatter_dc(p, c0, c1, g, false, threadIdx.x, blockDim.x, err);
    __syncthreads();
    const int nw = blockDim.x >> 5;
    const SegWhole seg{p.Bp, p.nnzB, p.d};
    BwdOp<BA> op{ba, g, sdA, p.dA, p.dB, p.dA != nullptr, p.d, err, {0.0f, 0.0f}};
    for (long long e0 = a0 + 32LL * warp_id(); e0 < a1; e0 += 32LL * nw) {
        const int nv = (int)(a1 - e0 < 32 ? a1 - e0 : 32);
        bwd_chunk<G>(p, load_chunk(e0, nv, p.Ai, p.Ax, p.nB, seg, err), nv, e0, op, sdA);
    }
    __syncthreads();
    scatter_dc(p, c0, c1, g, true, threadIdx.x, blockDim.x, err);
    __syncthreads();
}

// Light row, one warp, driven by pipelined_rows; the next row's range in C
// is requested one row ahead.
template <int G, class BA>
struct BwdRowBody {
    const BwdParams& p;
    const BA& ba;
    float* g;
    float* sdA;
    unsigned long long* err;
    int pref_row;
    long long pc0, pc1;
    long long c0, c1;
    __device__ __forceinline__ void gather(int row, long long a0, long long a1, const Chunk& ch0, int nv0,
                                           int next_row) {
        if (pref_row == row) {
            c0 = pc0;
            c1 = pc1;
        } else {
            c0 = clampll(__ldg(p.Cp + row), 0, p.nnzC);
            c1 = clampll(__ldg(p.Cp + row + 1), c0, p.nnzC);
        }
        if (next_row >= 0) {
            pc0 = clampll(__ldg(p.Cp + next_row), 0, p.nnzC);
            pc1 = clampll(__ldg(p.Cp + next_row + 1), pc0, p.nnzC);
            pref_row = next_row;
        }
        scatter_dc(p, c0, c1, g, false, lane_id(), 32, err);
        __syncwarp();
        const SegWhole seg{p.Bp, p.nnzB, p.d};
        BwdOp<BA> op{ba, g, sdA, p.dA, p.dB, p.dA != nullptr, p.d, err, {0.0f, 0.0f}};
        bwd_chunk<G>(p, ch0, nv0, a0, op, sdA);
        for (long long e0 = a0 + 32; e0 < a1; e0 += 32) {
            const int nv = (int)(a1 - e0 < 32 ? a1 - e0 : 32);
            bwd_chunk<G>(p, load_chunk(e0, nv, p.Ai, p.Ax, p.nB, seg, err), nv, e0, op, sdA);
        }
    }
    __device__ __forceinline__ void finish(int) {
        __syncwarp();
        scatter_dc(p, c0, c1, g, true, lane_id(), 32, err);
        __syncwarp();
    }
};

// ---------------------------------------------------------------------------
// Light rows of the backward in row groups (packed B, 16-byte aligned dB):
// R = 32/RG rows of the schedule per warp in lockstep, RG lanes per row.  A
// slot scatters its row of dC into its own dense row g (W = dpad floats),
// then walks the segments B(k,:) of its row's entries two entries per lane
// (one 16-byte load of the packed copy, starting at the even position at or
// below the segment's first entry): each entry (k, j) reads g[col] once, adds
// A(i,k) * dC(i,col) into dB with one 8-byte float atomic per lane (an entry
// of the pair outside the segment adds 0; the last pair of B takes scalar
// atomics) and B(k,j) * dC(i,col) into the entry's dA sum, reduced over the
// slot's lanes.  g is only read while the segments are walked, so segments
// need no ordering among themselves.  Launched behind k_backward with
// programmatic dependent launch; waits for that grid before exiting.
// ---------------------------------------------------------------------------
// A segment of B as a slot walks it in pairs: first position rounded down to
// even (qbase), positions before the segment (lead), positions covered from
// qbase (span), A's value a.
struct BrgSeg {
    long long qbase;
    int lead, span;
    float a;
};

__device__ __forceinline__ BrgSeg brg_seg_of(long long s, int L, float a) {
    BrgSeg q;
    q.qbase = s & ~1LL;
    q.lead = (int)(s - q.qbase);
    q.span = L > 0 ? q.lead + L : 0;
    q.a = a;
    return q;
}

__device__ __forceinline__ void brg_fetch(const int4* __restrict__ P4, const BrgSeg& sg, int q, int4& v) {
    if (2 * q < sg.span) v = __ldg(P4 + ((sg.qbase >> 1) + q));
}

// Pair q of a segment (entries qbase + 2q, + 2q + 1): dB terms out, dA part back.
__device__ __forceinline__ float brg_apply(const BwdParams& p, const BrgSeg& sg, int q, const int4& v, const float* g,
                                           unsigned long long* err) {
    const int cs[2] = {v.x, v.z};
    const int bs[2] = {v.y, v.w};
    float t2[2] = {0.0f, 0.0f};
    float part = 0.0f;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int pos = 2 * q + u;
        if (pos >= sg.lead && pos < sg.span) {
            const int c = cs[u];
            if ((unsigned)c < (unsigned)p.d) {
                const float gc = g[c];
                t2[u] = sg.a * gc;
                part += __int_as_float(bs[u]) * gc;
            } else {
                atomicOr(err, ERR_B_COL);
            }
        }
    }
    if (p.dB) {
        const long long qb = sg.qbase + 2LL * q;
        if (qb + 2 <= p.nnzB) {
            atomicAdd(reinterpret_cast<float2*>(p.dB + qb), make_float2(t2[0], t2[1]));
        } else {
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (2 * q + u >= sg.lead && 2 * q + u < sg.span) atomicAdd(p.dB + qb + u, t2[u]);
        }
    }
    return part;
}

// Entry ei of A: column k (-1 past the row) and value.
__device__ __forceinline__ void brg_load_a(const BwdParams& p, long long ei, bool ok, int& k, float& a) {
    k = -1;
    a = 0.0f;
    if (ok) {
        k = __ldg(p.Ai + ei);
        a = __ldg(p.Ax + ei);
    }
}

__device__ __forceinline__ void brg_seg(const BwdParams& p, int k, bool ok, long long& s, int& L,
                                        unsigned long long* err) {
    s = 0;
    L = 0;
    if (!ok) return;
    if ((unsigned)k < (unsigned)p.nB) SegWhole{p.Bp, p.nnzB, p.d}(k, s, L);
    else atomicOr(err, ERR_A_COL);
}

template <int RG>
__global__ void __launch_bounds__(256, 5) k_backward_light(BwdParams p) {
    extern __shared__ __align__(16) float fsm[];
    __shared__ long long s_nheavy, s_nrows;
    constexpr int R = 32 / RG;
    const int nw = blockDim.x >> 5, warp = warp_id(), lane = lane_id(), tid = threadIdx.x;
    const int g = lane / RG, gl = lane % RG;
    for (int i = tid; i < nw * R * p.dpad; i += blockDim.x) fsm[i] = 0.0f;
    if (tid < 32) {  // one warp; its lanes store the same values
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
        s_nrows = nr;
    }
    __syncthreads();
    float* gr = fsm + (size_t)(warp * R + g) * p.dpad;
    unsigned long long* err = &p.hdr->err;
    const int4* P4 = reinterpret_cast<const int4*>(p.Bpk);
    const long long* mark = p.s.flops;
    const long long end = s_nrows, step = (long long)gridDim.x * nw * R;
    for (long long idx = s_nheavy + ((long long)blockIdx.x * nw + warp) * R; idx < end; idx += step) {
        const long long my = idx + g;
        long long a0 = 0, a1 = 0, c0 = 0, c1 = 0;
        if (my < end) {
            const int row = __ldg(p.perm + my);
            a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
            a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
            if (is_split_row(mark, row, a1 - a0)) {
                a1 = a0;  // done by split parts
            } else {
                c0 = clampll(__ldg(p.Cp + row), 0, p.nnzC);
                c1 = clampll(__ldg(p.Cp + row + 1), c0, p.nnzC);
            }
        }
        const int len = (int)(a1 - a0);
        // first two chunks of A while dC is scattered
        int k0, k1;
        float x0, x1;
        brg_load_a(p, a0 + gl, gl < len, k0, x0);
        brg_load_a(p, a0 + RG + gl, RG + gl < len, k1, x1);
        // the row of dC into the dense row, eight entries per lane in flight
        // (the row is read once, from DRAM: a chain of single loads would
        // wait out one memory latency per entry)
        for (long long e = c0 + gl; e < c1; e += 8 * RG) {
            int cc[8];
            float vv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const long long eu = e + u * RG;
                cc[u] = eu < c1 ? __ldg(p.Ci + eu) : 0;
                vv[u] = eu < c1 ? __ldg(p.dC + eu) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (e + u * RG < c1) {
                    if ((unsigned)cc[u] < (unsigned)p.d) gr[cc[u]] = vv[u];
                    else atomicOr(err, ERR_C_ROW);
                }
            }
        }
        long long sg;
        int L;
        brg_seg(p, k0, gl < len, sg, L, err);
        __syncwarp();
        const int lmax = (int)__reduce_max_sync(FULL, (unsigned)len);
        BrgSeg nxt = brg_seg_of(shfl64(sg, g * RG), __shfl_sync(FULL, L, g * RG), __shfl_sync(FULL, x0, g * RG));
        int4 nv = make_int4(0, 0, 0, 0);
        brg_fetch(P4, nxt, gl, nv);
        for (int e = 0; e < lmax; e += RG) {
            int k2;
            float x2;
            long long ns;
            int nL;
            brg_load_a(p, a0 + e + 2 * RG + gl, e + 2 * RG + gl < len, k2, x2);
            brg_seg(p, k1, e + RG + gl < len, ns, nL, err);
            const int nu = lmax - e < RG ? lmax - e : RG;
            float mine = 0.0f;  // dA of entry e + gl of this slot's row
            for (int u = 0; u < nu; ++u) {
                const BrgSeg cur = nxt;
                const int4 cv = nv;
                long long s2;
                int L2;
                float a2;
                if (u + 1 < nu) {
                    s2 = shfl64(sg, g * RG + u + 1);
                    L2 = __shfl_sync(FULL, L, g * RG + u + 1);
                    a2 = __shfl_sync(FULL, x0, g * RG + u + 1);
                } else {
                    s2 = shfl64(ns, g * RG);
                    L2 = __shfl_sync(FULL, nL, g * RG);
                    a2 = __shfl_sync(FULL, x1, g * RG);
                }
                nxt = brg_seg_of(s2, L2, a2);
                brg_fetch(P4, nxt, gl, nv);
                float part = 0.0f;
                if (2 * gl < cur.span) part = brg_apply(p, cur, gl, cv, gr, err);
                for (int q = gl + RG; 2 * q < cur.span; q += RG) {
                    int4 w = make_int4(0, 0, 0, 0);
                    brg_fetch(P4, cur, q, w);
                    part += brg_apply(p, cur, q, w, gr, err);
                }
#pragma unroll
                for (int o = RG / 2; o >= 1; o >>= 1) part += __shfl_xor_sync(FULL, part, o, RG);
                if (gl == u) mine = part;
            }
            if (p.dA && e + gl < len) p.dA[a0 + e + gl] = mine;
            sg = ns;
            L = nL;
            x0 = x1;
            k1 = k2;
            x1 = x2;
        }
        __syncwarp();
        // clear the whole dense row with 16-byte stores (dpad is a multiple
        // of 32, rows 16-byte aligned): cheaper than revisiting the row's
        // entries of C
        for (int c = 4 * gl; c < p.dpad; c += 4 * RG) *reinterpret_cast<float4*>(gr + c) = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// HEAVY: split parts and heavy rows only (light rows run in k_backward_light);
// without the light-row walk the kernel fits six blocks per SM, and more
// resident warps hide more of its gather latency (300 -> 272 us at scale 20).
template <int G, bool PACKED, bool HEAVY>
__global__ void __launch_bounds__(256, HEAVY ? 6 : 5) k_backward(BwdParams p) {
    // a light-row kernel launched behind this one may start on SMs this grid
    // frees (the two handle disjoint rows; dB is only added to atomically)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(16) float fsm[];
    __shared__ long long s_item, s_nheavy, s_nrows;
    const int nw = blockDim.x >> 5, warp = warp_id(), tid = threadIdx.x;
    // layout: [nw][dpad] dense dC rows, then [nw][32] dA partials
    for (int i = tid; i < nw * (p.dpad + 32); i += blockDim.x) fsm[i] = 0.0f;
    if (tid < 32) {  // one warp; its lanes store the same values
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
        s_nrows = nr;
    }
    __syncthreads();
    const long long nheavy = s_nheavy, nrows = s_nrows;
    float* sdA = fsm + (size_t)nw * p.dpad + 32 * warp;
    using BA = typename std::conditional<PACKED, BPacked, BSep>::type;
    BA ba;
    if constexpr (PACKED) ba = BPacked{p.Bpk};
    else ba = BSep{p.Bi, p.Bx};
    const long long* mark = p.s.flops;
    {
        const long long nitems = min(*(volatile long long*)&p.hdr->scratch[2], p.item_cap);
        SplitItem it;
        while (next_split_item(p.s, p.Ap, p.nnzA, nitems, &s_item, it))
            backward_range_cta<G, BA>(p, ba, it.row, it.e0, it.e1, fsm, sdA);
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
        if (is_split_row(mark, row, a1 - a0)) continue;
        backward_range_cta<G, BA>(p, ba, row, a0, a1, fsm, sdA);
    }
    if constexpr (!HEAVY) {
        // light rows in the class order (highest first: the tiny rows, when
        // k_backward_tiny takes them, are the last ones)
        long long nlight_end = nrows;
        if (p.tiny) {
            long long t = 0;
            for (int c = 1 + lane_id(); c <= BWD_TINY_CLASS && c < p.cta_class; c += 32) t += p.hdr->hist[c];
            nlight_end -= warp_sum(t);
        }
        float* g = fsm + (size_t)warp * p.dpad;
        BwdRowBody<G, BA> body{p, ba, g, sdA, &p.hdr->err, -1, 0, 0, 0, 0};
        pipelined_rows(p.perm, nheavy + (long long)blockIdx.x * nw + warp, nlight_end, (long long)gridDim.x * nw,
                       p.Ap, p.nnzA, p.Ai, p.Ax, p.nB, SegWhole{p.Bp, p.nnzB, p.d}, &p.hdr->err, body, mark);
    }
}

// Tiny light rows (at most 31 products) in registers: lane j holds entry j
// of row i of C (column and dC value; the row has at most as many entries as
// products), and the row's products are placed one per lane (lane j: the
// product of number j over the row's entries of A, like an expansion of
// Eq. 1).  A product (k, col) finds dC(i, col) by a binary search of the
// sorted row of C over the lanes; it adds A(i,k) * dC(i, col) to dB with a
// float atomic and B(k, col) * dC(i, col) to dA(i,k), the products of one
// entry (neighbouring lanes) summed into their first lane.  32-row chunks
// are dealt to the warps in turn.  Used where the light rows would each
// take a warp pass over a dense row of d floats (d above the row-group
// range).
template <bool PACKED>
__global__ void __launch_bounds__(256) k_backward_tiny(BwdParams p) {
    const int lane = lane_id();
    unsigned long long* err = &p.hdr->err;
    const long long nchunks = ((long long)p.nB + 31) / 32;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const SegWhole seg{p.Bp, p.nnzB, p.d};
    for (long long c = gw; c < nchunks; c += nwarps) {
        const long long r = c * 32 + lane;
        const long long f = r < p.nB ? __ldg(p.s.flops + r) : 0;
        const int cls = flops_class(f);
        const bool tiny = f >= 1 && cls <= BWD_TINY_CLASS && cls < p.cta_class;
        long long a0 = 0, a1 = 0, o0 = 0, o1 = 0;
        if (tiny) {
            a0 = clampll(__ldg(p.Ap + r), 0, p.nnzA);
            a1 = clampll(__ldg(p.Ap + r + 1), a0, p.nnzA);
            o0 = clampll(__ldg(p.Cp + r), 0, p.nnzC);
            o1 = clampll(__ldg(p.Cp + r + 1), o0, p.nnzC);
        }
        unsigned rows = __ballot_sync(FULL, tiny);
        while (rows) {
            const int src = __ffs(rows) - 1;
            rows &= rows - 1;
            const long long b0 = shfl64(a0, src), b1 = shfl64(a1, src);
            const long long q0 = shfl64(o0, src), q1 = shfl64(o1, src);
            // the row of C, one entry per lane (sorted columns; none: INT_MAX)
            int cc = 0x7FFFFFFF;
            float dv = 0.0f;
            if (lane < q1 - q0) {
                cc = __ldg(p.Ci + q0 + lane);
                dv = __ldg(p.dC + q0 + lane);
            }
            if (q1 - q0 > 32 && lane == 0) atomicOr(err, ERR_C_ROW);
            int base = 0;  // products placed so far (warp-uniform)
            for (long long ec = b0; ec < b1 && base < 32; ec += 32) {
                const long long e = ec + lane;
                int len = 0;
                long long st = 0;
                float a = 0.0f;
                if (e < b1) {
                    const int k = __ldg(p.Ai + e);
                    a = __ldg(p.Ax + e);
                    if ((unsigned)k < (unsigned)p.nB) seg(k, st, len);
                    else atomicOr(err, ERR_A_COL);
                }
                const int incl = warp_incl_scan(len), excl = incl - len;
                const int tot = __shfl_sync(FULL, incl, 31);
                const int pj = lane - base;
                const int q = owner_lane(excl, pj < 0 ? 0 : pj);  // entry ec + q of A
                const long long sq = shfl64(st, q);
                const int eq = __shfl_sync(FULL, excl, q);
                const float aq = __shfl_sync(FULL, a, q);
                const bool ent = pj >= 0 && pj < tot;
                int col = 0x7FFFFFFF;
                float b = 0.0f;
                const long long j = sq + (pj - eq);  // the product's entry of B
                if (ent) {
                    if constexpr (PACKED) {
                        const int2 v = __ldg(p.Bpk + j);
                        col = v.x;
                        b = __int_as_float(v.y);
                    } else {
                        col = __ldg(p.Bi + j);
                        b = __ldg(p.Bx + j);
                    }
                }
                // dC(i, col): the last lane of the row of C whose column is <= col
                const int at = owner_lane(cc, col);
                const float g = __shfl_sync(FULL, dv, at);
                const bool found = __shfl_sync(FULL, cc, at) == col;
                float part = 0.0f;
                if (ent) {
                    if (found && (unsigned)col < (unsigned)p.d) {
                        if (p.dB) atomicAdd(p.dB + j, aq * g);
                        part = b * g;
                    } else {
                        atomicOr(err, (unsigned)col < (unsigned)p.d ? ERR_C_ROW : ERR_B_COL);
                    }
                }
                // dA of entry ec + q: its products are neighbouring lanes
                const int key = ent ? q : -1 - lane;
                part = seg_sum_down(part, key);
                const int prevq = __shfl_up_sync(FULL, key, 1);
                if (ent && p.dA && (lane == 0 || prevq != key)) p.dA[ec + q] = part;
                base += tot;
            }
        }
    }
}

size_t backward_smem(long long d, int warps) {
    const long long dpad = (d + 31) / 32 * 32;
    return sizeof(float) * (size_t)warps * (size_t)(dpad + 32);
}

template <int G, bool PACKED>
static const void* bwd_kernel(bool heavy_only) {
    return heavy_only ? (const void*)k_backward<G, PACKED, true> : (const void*)k_backward<G, PACKED, false>;
}

cudaError_t launch_backward(const DevCsr& A, const DevCsr& B, long long d, const long long* Cp,
                            const int* Ci, long long nnzC, const float* dC, float* dA, float* dB,
                            const int2* Bpk, const Sched& s, const LaunchCfg& cfg, cudaStream_t st) {
    cudaError_t e;
    if (d > MAX_BWD_D) return cudaErrorInvalidValue;
    if (dA && A.nnz && (e = cudaMemsetAsync(dA, 0, sizeof(float) * A.nnz, st))) return e;
    if (dB && B.nnz && (e = cudaMemsetAsync(dB, 0, sizeof(float) * B.nnz, st))) return e;
    if (A.nrows == 0 || (!dA && !dB)) return cudaSuccess;
    if ((e = cudaMemsetAsync(&s.hdr->heavy_ctr, 0, 2 * sizeof(unsigned long long), st))) return e;
    BwdParams p;
    p.Ap = A.rowptr;
    p.Ai = A.col;
    p.Ax = A.val;
    p.nnzA = A.nnz;
    p.Bp = B.rowptr;
    p.Bi = B.col;
    p.Bx = B.val;
    p.Bpk = Bpk;
    p.nnzB = B.nnz;
    p.nB = (int)B.nrows;
    p.d = (int)d;
    p.dpad = (int)((d + 31) / 32 * 32);
    p.Cp = Cp;
    p.Ci = Ci;
    p.dC = dC;
    p.nnzC = nnzC;
    p.dA = dA;
    p.dB = dB;
    p.perm = s.perm;
    p.hdr = s.hdr;
    p.cta_class = cfg.cta_class;
    p.s = s;
    p.item_cap = split_item_capacity(A.nnz);
    p.skip_light = 0;
    p.tiny = 0;
    int warps = cfg.warps_per_cta;
    if (warps > 8) return cudaErrorInvalidValue;
    size_t smem = backward_smem(d, warps);
    while (smem > 200 * 1024 && warps > 1) {
        warps /= 2;
        smem = backward_smem(d, warps);
    }
    const bool pk = Bpk != nullptr;
    // light rows in row groups of eight lanes (pairs): packed B, aligned dB
    constexpr int BRG = 8;
    const size_t lsmem = sizeof(float) * (size_t)p.dpad * (32 / BRG) * warps;
    const bool rg = cfg.row_lanes != 32 && pk && !(dB && (reinterpret_cast<uintptr_t>(dB) & 15)) && p.dpad <= 512 &&
                    lsmem <= 200 * 1024;
    if (rg) p.skip_light = 1;
    // without the row-group kernel, tiny light rows run in registers (one
    // warp per light row forced: the classic walk for every row)
    if (!rg && cfg.row_lanes != 32 && d > 256) {
        p.tiny = 1;
        const void* kt = pk ? (const void*)k_backward_tiny<true> : (const void*)k_backward_tiny<false>;
        void* targs[] = {&p};
        count_launch();
        if ((e = cudaLaunchKernel(kt, dim3(persistent_grid(kt, 256, 0, cfg.sms)), dim3(256), targs, 0, st)))
            return e;
    }
    const void* k;
    switch (cfg.group) {
        case 2:  // quads: packed B and a 16-byte aligned dB only
            if (!pk || (dB && (reinterpret_cast<uintptr_t>(dB) & 15))) return cudaErrorInvalidValue;
            k = bwd_kernel<2, true>(rg);
            break;
        case 1: k = pk ? bwd_kernel<1, true>(rg) : bwd_kernel<1, false>(rg); break;
        case 4: k = pk ? bwd_kernel<4, true>(rg) : bwd_kernel<4, false>(rg); break;
        case 8: k = pk ? bwd_kernel<8, true>(rg) : bwd_kernel<8, false>(rg); break;
        case 16: k = pk ? bwd_kernel<16, true>(rg) : bwd_kernel<16, false>(rg); break;
        case 32: k = pk ? bwd_kernel<32, true>(rg) : bwd_kernel<32, false>(rg); break;
        default: return cudaErrorInvalidValue;
    }
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    const int grid = persistent_grid(k, 32 * warps, smem, cfg.sms);
    void* args[] = {&p};
    count_launch();
    if ((e = cudaLaunchKernel(k, dim3(grid), dim3(32 * warps), args, smem, st))) return e;
    if (!rg) return cudaSuccess;
    const void* kl = (const void*)k_backward_light<BRG>;
    if (lsmem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(kl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem)))
        return e;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(persistent_grid(kl, 32 * warps, lsmem, cfg.sms));
    lc.blockDim = dim3(32 * warps);
    lc.dynamicSmemBytes = lsmem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    count_launch();
    return cudaLaunchKernelEx(&lc, k_backward_light<BRG>, p);
}

}  // namespace ts
