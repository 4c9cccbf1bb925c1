// Batched TS-SpGEMM: many independent products C_b = A_b * B_b of uneven
// shapes, each phase one launch over all instances, graph capturable.
//
// The kernels read every instance's own arrays through a device table of
// instance descriptors (InstDesc): there is no copy of the instances into a
// common product and no copy of the results back.  The rows of all
// instances are numbered one after another (instance b owns rows
// row_off_b .. row_off_b + n_b - 1); a kernel finds a row's instance by a
// binary search over the table.  Each descriptor carries that instance's
// own tuning: its accumulator width W_b (one column tile of the instance's
// 32-column-padded d_b), its accumulator kind (the shared accumulator with
// occupancy bits, or the dense-B form for a dense enough B_b) and its
// heavy-row threshold.
//
// Forward (four launches): prepare (row flops, the row-aligned packed copy
// of each B_b and, for dense-B instances, the dense copy; rows at or above
// their instance's threshold go on the heavy list), symbolic (row counts
// into each C_b's row pointers: heavy rows one block each from the list,
// light rows one warp each in row order), scan (one block per instance),
// numeric (as the symbolic pass, writing each C_b).  Backward (two
// launches): the gradients are cleared, then dA by rows and dB by float
// atomics.  Nothing waits on another block: the only coordination is
// atomic counters over the heavy list.
#include "common.cuh"
#include "denseb.cuh"
#include "kernels.h"
#include "numeric.cuh"
#include "rowgroup.cuh"
#include "wide.cuh"

namespace ts {

// Instance of global row g (the last instance whose first row is <= g; an
// instance without rows shares its first row with the next one).
__device__ __forceinline__ int inst_of(const InstDesc* __restrict__ inst, int count, long long g) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&inst[mid].row_off) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The single-product parameters the shared walks read, for instance I.
__device__ __forceinline__ NumParams inst_params(const InstDesc& I) {
    NumParams p{};
    p.Ap = I.A_rowptr;
    p.Ai = I.A_col;
    p.Ax = I.A_val;
    p.nnzA = I.annz;
    p.Bp = I.B_rowptr;
    p.Bi = I.B_col;
    p.Bx = I.B_val;
    p.Bq = I.Bq;
    p.nnzB = I.bnnz;
    p.nB = (int)I.n;
    p.d = (int)I.d;
    p.W = I.W;
    p.T = 1;
    return p;
}

// Instance of 32-row chunk c (the last instance whose first chunk is <= c).
__device__ __forceinline__ int inst_of_chunk(const InstDesc* __restrict__ inst, int count, long long c) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&inst[mid].chunk_off) <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// This warp's next 32-row chunk from queue q: chunks are dealt c0, c0 + 1,
// ... in order as warps ask for them (>= the caller's end when none is
// left), so a warp that drew heavy chunks takes fewer of them.
__device__ __forceinline__ long long bat_next_chunk(unsigned long long* q, long long c0) {
    unsigned long long t = 0;
    if (lane_id() == 0) t = atomicAdd(q, 1ull);
    return c0 + (long long)__shfl_sync(FULL, t, 0);
}

// Products of row k of B for the flops (its length, at most d).
__device__ __forceinline__ long long bat_brow_len(const InstDesc& I, int k) {
    const long long s = clampll(__ldg(I.B_rowptr + k), 0, I.bnnz);
    const long long e = clampll(__ldg(I.B_rowptr + k + 1), s, I.bnnz);
    return e - s < I.d ? e - s : I.d;
}

// ---------------------------------------------------------------------------
// prepare: one warp per 32-row chunk of one instance (chunks dealt from a
// queue), lane l owning row i0 + l of A_b and of B_b.
//  * flops: the entries of the chunk's rows of A with at most PREP_SHORT
//    entries are numbered across the rows and read 32 at a time, four
//    rounds in flight (coalesced); each entry's B row length goes to its row
//    by a segmented sum over the lanes.  A longer row is then summed by the
//    whole warp, eight loads per lane in flight.  Rows at or above their
//    instance's threshold go on the heavy list.
//  * the chunk's rows of B are copied into the row-aligned packed copy the
//    same way (entries numbered across the rows, pads as column -1), and for
//    a dense-B instance into its dense copy and pattern bits, cleared first.
// ---------------------------------------------------------------------------
constexpr int PREP_SHORT = 256;

__global__ void __launch_bounds__(256) k_bat_prepare(const InstDesc* __restrict__ inst, int count, long long c0,
                                                     long long c1, long long* __restrict__ flops,
                                                     int* __restrict__ heavy, BatchCtl* ctl) {
    __shared__ long long s_f[8][32];
    const int lane = lane_id(), warp = warp_id();
    long long* wf = s_f[warp];
    wf[lane] = 0;
    __syncwarp();
    bool bad_a = false, bad_b = false;
    for (long long c = bat_next_chunk(&ctl->l_prep, c0); c < c1; c = bat_next_chunk(&ctl->l_prep, c0)) {
        const InstDesc& I = inst[inst_of_chunk(inst, count, c)];
        const long long i0 = (c - I.chunk_off) * 32;
        const long long i = i0 + lane;
        const bool act = i < I.n;
        long long a0 = 0, a1 = 0;
        if (act) {
            a0 = clampll(__ldg(I.A_rowptr + i), 0, I.annz);
            a1 = clampll(__ldg(I.A_rowptr + i + 1), a0, I.annz);
        }
        // short rows, numbered across the chunk
        const int slen = a1 - a0 <= PREP_SHORT ? (int)(a1 - a0) : 0;
        const int incl = warp_incl_scan(slen), excl = incl - slen;
        const int total = __shfl_sync(FULL, incl, 31);
        const long long shift = a0 - excl;  // entry of number p in row q: shift(q) + p
        for (int p0 = 0; p0 < total; p0 += 128) {
            int q[4], k[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = p0 + 32 * u + lane;
                q[u] = owner_lane(excl, p);
                const long long e = shfl64(shift, q[u]) + p;
                k[u] = p < total ? __ldg(I.A_col + e) : -1;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = p0 + 32 * u + lane;
                long long v = 0;
                if (p < total) {
                    if ((unsigned)k[u] < (unsigned)I.n) v = bat_brow_len(I, k[u]);
                    else bad_a = true;
                }
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {  // sum over this lane's run of equal q, from this lane on
                    const long long t = shfl64_down(v, o);
                    const int qo = __shfl_down_sync(FULL, q[u], o);
                    if (lane + o < 32 && qo == q[u]) v += t;
                }
                const int qp = __shfl_up_sync(FULL, q[u], 1);
                if (p < total && (lane == 0 || qp != q[u])) wf[q[u]] += v;  // one lane per row and round
                __syncwarp();
            }
        }
        long long f = wf[lane];
        wf[lane] = 0;
        // long rows, one at a time by the whole warp
        unsigned longs = __ballot_sync(FULL, a1 - a0 > PREP_SHORT);
        while (longs) {
            const int src = __ffs(longs) - 1;
            longs &= longs - 1;
            const long long la0 = shfl64(a0, src), la1 = shfl64(a1, src);
            long long sum = 0;
            for (long long e = la0 + lane; e < la1; e += 256) {
                int k[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) k[u] = e + 32 * u < la1 ? __ldg(I.A_col + e + 32 * u) : 0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (e + 32 * u < la1) {
                        if ((unsigned)k[u] < (unsigned)I.n) sum += bat_brow_len(I, k[u]);
                        else bad_a = true;
                    }
                }
            }
            sum = warp_sum(sum);
            if (lane == src) f = sum;
        }
        if (act) {
            flops[I.row_off + i] = f;
            if (f > 0 && f >= I.heavy_min) heavy[atomicAdd(&ctl->nheavy, 1ull)] = (int)(I.row_off + i);
        }
        // the chunk's rows of B into the copies
        long long bs = 0;
        int blen = 0;
        unsigned g0 = 0;
        if (act) padded_row<2>(I.B_rowptr, I.bnnz, (int)I.d, (int)i, bs, blen, g0);
        const bool dense = I.accum == BAT_DENSE_B && I.Bd;
        if (dense) {  // cleared before the entries land
            const long long nr = I.n - i0 < 32 ? I.n - i0 : 32;
            float4* r4 = reinterpret_cast<float4*>(I.Bd + (size_t)i0 * I.Wd);
            for (long long x = lane; x < nr * (I.Wd >> 2); x += 32) r4[x] = make_float4(0.f, 0.f, 0.f, 0.f);
            unsigned* bw = I.Bbits + (size_t)i0 * (I.Wd >> 5);
            for (long long x = lane; x < nr * (I.Wd >> 5); x += 32) bw[x] = 0u;
            __syncwarp();
        }
        const int span = (blen + 1) & ~1;
        const int bincl = warp_incl_scan(span), bexcl = bincl - span;
        const int btotal = __shfl_sync(FULL, bincl, 31);
        int2* Q = reinterpret_cast<int2*>(I.Bq);
        for (int p0 = 0; p0 < btotal; p0 += 128) {
            int q[4], j[4], cc[4];
            unsigned gq[4];
            bool ent[4];
            float xx[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = p0 + 32 * u + lane;
                q[u] = owner_lane(bexcl, p);
                j[u] = p - __shfl_sync(FULL, bexcl, q[u]);
                gq[u] = __shfl_sync(FULL, g0, q[u]);
                const long long sq = shfl64(bs, q[u]);
                const int lq = __shfl_sync(FULL, blen, q[u]);
                ent[u] = p < btotal && j[u] < lq;  // an entry of B (else a pad)
                cc[u] = ent[u] ? __ldg(I.B_col + sq + j[u]) : -1;
                xx[u] = ent[u] && I.B_val ? __ldg(I.B_val + sq + j[u]) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = p0 + 32 * u + lane;
                if (p >= btotal) continue;
                int2 v = make_int2(-1, 0);  // pad
                const int c = cc[u];
                if (ent[u]) {
                    if ((unsigned)c < (unsigned)I.d) {
                        v = make_int2(c, __float_as_int(xx[u]));
                        if (dense) {
                            const long long row = i0 + q[u];
                            I.Bd[(size_t)row * I.Wd + c] = xx[u];
                            atomicOr(I.Bbits + (size_t)row * (I.Wd >> 5) + (c >> 5), 1u << (c & 31));
                        }
                    } else {
                        bad_b = true;
                    }
                }
                Q[2 * (size_t)gq[u] + j[u]] = v;
            }
        }
    }
    if (bad_a) atomicOr(&ctl->err, ERR_A_COL);
    if (bad_b) atomicOr(&ctl->err, ERR_B_COL);
}

// Ascending bitonic sort of one key per lane across the warp, carrying val.
__device__ __forceinline__ void warp_sort_asc(int& key, int& val) {
    const int lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int pk = __shfl_xor_sync(FULL, key, j), pv = __shfl_xor_sync(FULL, val, j);
            const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
            if (keep_min ? pk < key : pk > key) {
                key = pk;
                val = pv;
            }
        }
    }
}

// Light rows of one 32-row chunk of instance I, sorted by products
// (heaviest first) so that the four rows a warp takes side by side have
// nearly equal lengths: returns the count L; sorted position t of the warp
// holds row base + srt (lanes >= L hold no row).
__device__ __forceinline__ int chunk_light_sorted(const InstDesc& I, const long long* __restrict__ flops,
                                                  long long i0, int& srt) {
    const int lane = lane_id();
    const long long i = i0 + lane;
    const long long f = i < I.n ? __ldg(flops + I.row_off + i) : 0;
    const bool light = f > 0 && f < I.heavy_min;
    int key = light ? -(int)(f < (1LL << 30) ? f : (1LL << 30)) : 0x7FFFFFFF;
    srt = lane;
    warp_sort_asc(key, srt);
    return __popc(__ballot_sync(FULL, light));
}

// This slot's row of the group at sorted position t of a chunk (eight
// lanes per slot, four slots; i = -1 past the chunk's L light rows): its
// first entry of A and length, and with want_out its range in C_b.
struct BatRow {
    long long i, a0, out, out_end;
    int len;
};

__device__ __forceinline__ BatRow bat_row(const InstDesc& I, long long i0, int srt, int L, int t, bool want_out) {
    const int pos = t + (lane_id() >> 3);
    const int r = __shfl_sync(FULL, srt, pos & 31);
    BatRow b{-1, 0, 0, 0, 0};
    if (pos < L) {
        b.i = i0 + r;
        b.a0 = clampll(__ldg(I.A_rowptr + b.i), 0, I.annz);
        b.len = (int)(clampll(__ldg(I.A_rowptr + b.i + 1), b.a0, I.annz) - b.a0);
        if (want_out) {
            b.out = clampll(__ldg(I.C_rowptr + b.i), 0, I.cap);
            b.out_end = clampll(__ldg(I.C_rowptr + b.i + 1), b.out, I.cap);
        }
    }
    return b;
}

// Whether global row g (lane's row of a 32-row chunk) is a light row: it
// has products and fewer than its instance's threshold.
__device__ __forceinline__ bool bat_light(const InstDesc* inst, int count, const long long* flops, long long g,
                                          long long g1, int& b) {
    b = 0;
    if (g >= g1) return false;
    const long long f = __ldg(flops + g);
    if (f <= 0) return false;
    b = inst_of(inst, count, g);
    return f < __ldg(&inst[b].heavy_min);
}

// Byte marks (symbolic light rows): column c of the slot's row is reached.
// Lanes that reach the same column store the same byte, so no atomic is
// needed.
struct AddByte {
    unsigned char* m;
    __device__ __forceinline__ void operator()(int c, unsigned W, float) const {
        if ((unsigned)c < W) m[c] = 1;
    }
};

// ---------------------------------------------------------------------------
// symbolic: row counts into each C_b's row pointers (C_b.rowptr[i + 1])
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bat_symbolic(const InstDesc* __restrict__ inst, int count, long long c0,
                                                      long long c1, const long long* __restrict__ flops,
                                                      const int* __restrict__ heavy, BatchCtl* ctl, int Wmax) {
    __shared__ __align__(16) unsigned char s_hb[1024];  // the block's byte marks (heavy rows)
    // four slots of byte marks per warp (light rows), Wmax + 32 bytes each
    // (the pad puts the slots' words on different banks)
    extern __shared__ __align__(16) unsigned char s_marks[];
    __shared__ long long s_item;
    const int nwarps = blockDim.x >> 5, warp = warp_id(), lane = lane_id(), tid = threadIdx.x;
    const int mstride = Wmax + 32;
    for (int x = tid; x < 1024 / 4; x += blockDim.x) reinterpret_cast<unsigned*>(s_hb)[x] = 0u;
    for (int x = tid; x < nwarps * 4 * mstride / 4; x += blockDim.x) reinterpret_cast<unsigned*>(s_marks)[x] = 0u;
    __syncthreads();
    unsigned long long* err = &ctl->err;
    const long long nheavy = (long long)ctl->nheavy;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&ctl->q_sym, 1ull);
        __syncthreads();
        const long long h = s_item;
        __syncthreads();
        if (h >= nheavy) break;
        const long long g = heavy[h];
        const InstDesc& I = inst[inst_of(inst, count, g)];
        const long long i = g - I.row_off;
        const NumParams p = inst_params(I);
        const long long a0 = clampll(I.A_rowptr[i], 0, I.annz), a1 = clampll(I.A_rowptr[i + 1], a0, I.annz);
        // the warps take the row's chunks in turn, each stopping once the
        // marks hold all d columns (the count is then d whatever products
        // remain); a warp reads marks other warps may still be storing, which
        // can only delay its stop
        const int nw4 = I.W >> 2;  // words of marks
        const long long d = I.d;
        auto full = [&]() {
            int cnt = 0;
            for (int x = lane; x < nw4; x += 32) cnt += __popc(reinterpret_cast<const volatile unsigned*>(s_hb)[x]);
            return warp_sum(cnt) >= d;
        };
        wide_range(p, AddByte{s_hb}, a0 + 32LL * warp, a1, 32LL * nwarps, err, full);
        __syncthreads();
        if (warp == 0) {
            int cnt = 0;
            for (int x = lane; x < nw4; x += 32) {  // bytes are 0 or 1
                cnt += __popc(reinterpret_cast<unsigned*>(s_hb)[x]);
                reinterpret_cast<unsigned*>(s_hb)[x] = 0u;
            }
            cnt = warp_sum(cnt);
            if (lane == 0) I.C_rowptr[i + 1] = cnt;
        }
        __syncthreads();
    }
    // light rows in row groups: four rows per warp (eight lanes each, the
    // chunk's rows sorted by products), each marking its own bytes
    const int lanes = lane & 7, slot = lane >> 3;
    unsigned char* mym = s_marks + (size_t)(warp * 4 + slot) * mstride;
    for (long long c = bat_next_chunk(&ctl->l_sym, c0); c < c1; c = bat_next_chunk(&ctl->l_sym, c0)) {
        const InstDesc& I = inst[inst_of_chunk(inst, count, c)];
        const long long i0 = (c - I.chunk_off) * 32;
        {
            const long long i = i0 + lane;
            if (i < I.n && __ldg(flops + I.row_off + i) <= 0) I.C_rowptr[i + 1] = 0;
        }
        int srt;
        const int L = chunk_light_sorted(I, flops, i0, srt);
        const NumParams p = inst_params(I);
        const int nw = I.W >> 5;
        // pipelined over the chunk's groups: the next group's row bounds load
        // before this group's walk, its first entries of A before the count
        BatRow cur = bat_row(I, i0, srt, L, 0, false);
        int k0, k1;
        float x0, x1;
        rg_load_a(p, cur.a0 + lanes, lanes < cur.len, k0, x0);
        rg_load_a(p, cur.a0 + 8 + lanes, 8 + lanes < cur.len, k1, x1);
        for (int t = 0; t < L; t += 4) {
            const BatRow nxt = bat_row(I, i0, srt, L, t + 4, false);
            const int lmax = (int)__reduce_max_sync(FULL, (unsigned)cur.len);
            rgp_tile<8, 2>(p, I.Bq, AddByte{mym}, cur.a0, cur.len, lmax, err, k0, x0, k1, x1);
            rg_load_a(p, nxt.a0 + lanes, lanes < nxt.len, k0, x0);
            rg_load_a(p, nxt.a0 + 8 + lanes, 8 + lanes < nxt.len, k1, x1);
            __syncwarp();
            int cnt = 0;
            unsigned* mw = reinterpret_cast<unsigned*>(mym);
            for (int w = lanes; w < nw * 8; w += 8) {  // bytes are 0 or 1
                cnt += __popc(mw[w]);
                mw[w] = 0u;
            }
            cnt += __shfl_xor_sync(FULL, cnt, 1);
            cnt += __shfl_xor_sync(FULL, cnt, 2);
            cnt += __shfl_xor_sync(FULL, cnt, 4);
            if (cur.i >= 0 && lanes == 0) I.C_rowptr[cur.i + 1] = cnt;
            __syncwarp();
            cur = nxt;
        }
    }
}

// ---------------------------------------------------------------------------
// scan: one block of 1024 threads per instance, in place over C_b.rowptr
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_bat_scan(const InstDesc* __restrict__ inst, BatchCtl* ctl) {
    __shared__ long long s_w[32];
    __shared__ long long s_carry;
    const InstDesc& I = inst[blockIdx.x];
    long long* rp = I.C_rowptr;
    const int tid = threadIdx.x, lane = lane_id(), warp = warp_id();
    if (tid == 0) {
        s_carry = 0;
        rp[0] = 0;
    }
    __syncthreads();
    constexpr int ITEMS = 4;
    for (long long base = 1; base <= I.n; base += 1024LL * ITEMS) {
        long long v[ITEMS];
        long long t = 0;
#pragma unroll
        for (int u = 0; u < ITEMS; ++u) {
            const long long x = base + (long long)tid * ITEMS + u;
            v[u] = x <= I.n ? rp[x] : 0;
            t += v[u];
            v[u] = t;  // running sum inside the thread
        }
        const long long wi = warp_incl_scan(t);
        if (lane == 31) s_w[warp] = wi;
        __syncthreads();
        if (warp == 0) {
            const long long y = warp_incl_scan(s_w[lane]);
            s_w[lane] = y;
        }
        __syncthreads();
        const long long before = s_carry + (warp ? s_w[warp - 1] : 0) + wi - t;
#pragma unroll
        for (int u = 0; u < ITEMS; ++u) {
            const long long x = base + (long long)tid * ITEMS + u;
            if (x <= I.n) rp[x] = before + v[u];
        }
        __syncthreads();
        if (tid == 0) s_carry += s_w[31];
        __syncthreads();
    }
    if (tid == 0 && s_carry > I.cap) atomicOr(&ctl->err, ERR_CAPACITY);
}

// ---------------------------------------------------------------------------
// numeric
// ---------------------------------------------------------------------------
// Row i of a dense-B instance: the warp (team: the block, its warps taking
// the row's chunks in turn and summing their partial rows) holds V columns
// per lane in registers.  A copy wider than 32 V columns (Wd = 256 with
// V = 4) is walked in bands of 32 V columns, each written out in turn, so
// that no lane holds more than four columns.
template <int V>
__device__ __forceinline__ void bat_dense_row(const NumParams& p, const InstDesc& I, long long i, long long a0,
                                              long long a1, bool team, float* s_rows, unsigned* s_mask,
                                              unsigned long long* err) {
    const int nwarps = blockDim.x >> 5;
    const bool writer = !team || warp_id() == 0;
    const long long out = clampll(I.C_rowptr[i], 0, I.cap);
    const long long out_end = clampll(I.C_rowptr[i + 1], out, I.cap);
    long long pos = out;
    for (int cb = 0; cb < I.Wd; cb += 32 * V) {
        float acc[V];
        unsigned m = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0.0f;
        if (team) {
            dense_accumulate<V>(p, I.Bd, I.Bbits, I.Wd, a0 + 32LL * warp_id(), a1, 32LL * nwarps, acc, m, err, cb);
            dense_block_sum<V>(acc, m, s_rows, s_mask);
        } else {
            dense_accumulate<V>(p, I.Bd, I.Bbits, I.Wd, a0, a1, 32, acc, m, err, cb);
        }
        if (writer) pos += dense_emit<V>(acc, m, pos, out_end, I.C_col, I.C_val, cb);
    }
    if (writer && lane_id() == 0 && pos != out_end) atomicOr(err, ERR_C_ROW);
}

__device__ __forceinline__ void bat_dense_any(const NumParams& p, const InstDesc& I, long long i, long long a0,
                                              long long a1, bool team, float* s_rows, unsigned* s_mask,
                                              unsigned long long* err) {
    switch (I.Wd) {
        case 32: bat_dense_row<1>(p, I, i, a0, a1, team, s_rows, s_mask, err); break;
        case 64: bat_dense_row<2>(p, I, i, a0, a1, team, s_rows, s_mask, err); break;
        default: bat_dense_row<4>(p, I, i, a0, a1, team, s_rows, s_mask, err); break;  // 128, 256
    }
}

// Words of shared memory per warp in the numeric kernel: a shared
// accumulator of Wmax + 8 floats and Wmax/32 + 1 bitmap words, or, for
// plus-times with Wmax <= 256, four row-group accumulators of Wmax + 8.
__host__ __device__ inline int bat_per_warp(int Wmax, bool values) {
    const int wide = (Wmax + 8) + Wmax / 32 + 1;
    const int rg = 4 * (Wmax + 8);
    return (values && Wmax <= 256 && rg > wide) ? rg : wide;
}

// Heavy rows (one block each, per-warp shared accumulators summed by the
// block, or the dense-B form), then light rows (one warp each, in row
// order).  Dynamic shared memory per warp: Wmax + 8 floats of accumulator
// and Wmax/32 + 1 bitmap words.
__global__ void __launch_bounds__(256, 3) k_bat_numeric(const InstDesc* __restrict__ inst, int count, long long c0,
                                                        long long c1, const long long* __restrict__ flops,
                                                        const int* __restrict__ heavy, BatchCtl* ctl, int Wmax,
                                                        bool values) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float s_rows[8 * 128];  // dense-B partial rows (V <= 4)
    __shared__ unsigned s_mask[8 * 32];
    __shared__ long long s_item;
    const int nwarps = blockDim.x >> 5, warp = warp_id(), lane = lane_id(), tid = threadIdx.x;
    const int ld = Wmax + 8;
    const int per_warp = bat_per_warp(Wmax, values);  // 4-byte words
    // plus-times with every width <= 256: row groups (accumulators start
    // RG_EMPTY; 32 slots of Wmax + 8, then a summed row of Wmax for heavy
    // rows); otherwise per-warp shared accumulators (start at 0)
    const bool rg = values && Wmax <= 256;
    for (int x = tid; x < nwarps * per_warp + (rg ? Wmax : 0); x += blockDim.x)
        reinterpret_cast<unsigned*>(smem)[x] = rg ? RG_EMPTY : 0u;
    __shared__ int s_wcnt[256 / 32 + 1];
    __syncthreads();
    unsigned long long* err = &ctl->err;
    float* wacc = reinterpret_cast<float*>(smem) + (size_t)warp * per_warp;
    unsigned* wbm = reinterpret_cast<unsigned*>(wacc) + ld;
    const AddShared wadd{wacc, wbm};
    float* acc0 = reinterpret_cast<float*>(smem);
    unsigned* bm0 = reinterpret_cast<unsigned*>(smem) + ld;
    const long long nheavy = (long long)ctl->nheavy;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&ctl->q_num, 1ull);
        __syncthreads();
        const long long h = s_item;
        __syncthreads();
        if (h >= nheavy) break;
        const long long g = heavy[h];
        const InstDesc& I = inst[inst_of(inst, count, g)];
        const long long i = g - I.row_off;
        const NumParams p = inst_params(I);
        const long long a0 = clampll(I.A_rowptr[i], 0, I.annz), a1 = clampll(I.A_rowptr[i + 1], a0, I.annz);
        if (I.accum == BAT_DENSE_B && I.Bd && I.C_val) {
            bat_dense_any(p, I, i, a0, a1, true, s_rows, s_mask, err);
            __syncthreads();
            continue;
        }
        if (rg) {
            // 32 slots of eight lanes, each a contiguous share of the row's
            // entries on its own accumulator; the block sums the slots
            const int S = nwarps * 4, sl = warp * 4 + (lane >> 3), gl = lane & 7;
            const long long n = a1 - a0, q = n / S, r = n % S;
            const long long s0 = a0 + q * sl + (sl < r ? sl : r);
            const int len = (int)(q + (sl < r ? 1 : 0));
            const int lmax = (int)__reduce_max_sync(FULL, (unsigned)len);
            float* sacc = reinterpret_cast<float*>(smem) + (size_t)sl * ld;
            float* sum = reinterpret_cast<float*>(smem) + (size_t)nwarps * per_warp;
            int k0, k1;
            float x0, x1;
            rg_load_a(p, s0 + gl, gl < len, k0, x0);
            rg_load_a(p, s0 + 8 + gl, 8 + gl < len, k1, x1);
            rgp_tile<8, 2>(p, I.Bq, AddPlain{sacc}, s0, len, lmax, err, k0, x0, k1, x1);
            __syncthreads();
            for (int c = tid; c < I.W; c += blockDim.x) sum[c] = __uint_as_float(rgcta_sum(sacc - (size_t)sl * ld, ld, S, c));
            if (gl == 0) sacc[I.W] = __uint_as_float(RG_EMPTY);  // the spare column (pads)
            __syncthreads();
            long long out = clampll(I.C_rowptr[i], 0, I.cap);
            const long long out_end = clampll(I.C_rowptr[i + 1], out, I.cap);
            rgcta_emit(sum, I.W, 0, out, out_end, I.C_col, I.C_val, s_wcnt, err);
            if (tid == 0 && out != out_end) atomicOr(err, ERR_C_ROW);
            continue;
        }
        wide_range(p, wadd, a0 + 32LL * warp, a1, 32LL * nwarps, err);
        __syncthreads();
        const int nw = I.W >> 5;
        for (int c = tid; c < I.W; c += blockDim.x) {  // the warps' columns summed into warp 0's
            float v = 0.0f;
            bool any = false;
            for (int w = 0; w < nwarps; ++w) {
                float* aw = reinterpret_cast<float*>(smem) + (size_t)w * per_warp;
                const unsigned* bw = reinterpret_cast<const unsigned*>(aw) + ld;
                if ((bw[c >> 5] >> (c & 31)) & 1u) {
                    v += aw[c];
                    any = true;
                    if (w) aw[c] = 0.0f;
                }
            }
            if (any) acc0[c] = v;
        }
        __syncthreads();
        for (int x = tid; x < nw; x += blockDim.x) {
            unsigned u = 0;
            for (int w = 0; w < nwarps; ++w) u |= reinterpret_cast<const unsigned*>(smem)[(size_t)w * per_warp + ld + x];
            bm0[x] = u;
        }
        __syncthreads();
        const long long out = clampll(I.C_rowptr[i], 0, I.cap);
        const long long out_end = clampll(I.C_rowptr[i + 1], out, I.cap);
        const int tot = wide_emit(acc0, bm0, nw, out, out_end, I.C_col, I.C_val, warp, nwarps, err);
        __syncthreads();
        for (int x = tid; x < nwarps * nw; x += blockDim.x)
            reinterpret_cast<unsigned*>(smem)[(size_t)(x / nw) * per_warp + ld + (x % nw)] = 0u;
        if (tid == 0 && out + tot != out_end) atomicOr(err, ERR_C_ROW);
        __syncthreads();
    }
    // light rows, by 32-row chunks of one instance.  Plus-times with every
    // width <= 256: four rows per warp in row groups (eight lanes, private
    // accumulators that start RG_EMPTY, rows sorted by products); dense-B
    // instances one row per warp in registers; otherwise one row per warp on
    // the warp's shared accumulator.
    const int lanes = lane & 7, slot = lane >> 3;
    for (long long c = bat_next_chunk(&ctl->l_num, c0); c < c1; c = bat_next_chunk(&ctl->l_num, c0)) {
        const InstDesc& I = inst[inst_of_chunk(inst, count, c)];
        const long long i0 = (c - I.chunk_off) * 32;
        const NumParams p = inst_params(I);
        const bool dense = I.accum == BAT_DENSE_B && I.Bd && I.C_val;
        if (rg && !dense) {
            int srt;
            const int L = chunk_light_sorted(I, flops, i0, srt);
            const int Wi = I.W;
            float* myacc = wacc + (size_t)slot * (Wi + 8);
            for (int t = 0; t < L; t += 4) {
                const BatRow cur = bat_row(I, i0, srt, L, t, true);
                const int lmax = (int)__reduce_max_sync(FULL, (unsigned)cur.len);
                int k0, k1;
                float x0, x1;
                rg_load_a(p, cur.a0 + lanes, lanes < cur.len, k0, x0);
                rg_load_a(p, cur.a0 + 8 + lanes, 8 + lanes < cur.len, k1, x1);
                rgp_tile<8, 2>(p, I.Bq, AddPlain{myacc}, cur.a0, cur.len, lmax, err, k0, x0, k1, x1);
                long long out = cur.out;
                rg_emit<8>(wacc, Wi, 0, out, cur.out_end, I.C_col, I.C_val, err);
                // the spare column (pads) back to empty, for the next rows
                if (lanes == 0) myacc[Wi] = __uint_as_float(RG_EMPTY);
                if (cur.i >= 0 && lanes == 0 && out != cur.out_end) atomicOr(err, ERR_C_ROW);
                __syncwarp();
            }
            continue;
        }
        const long long g = I.row_off + i0 + lane;
        const long long f = i0 + lane < I.n ? __ldg(flops + g) : 0;
        unsigned rows = __ballot_sync(FULL, f > 0 && f < I.heavy_min);
        while (rows) {
            const int src = __ffs(rows) - 1;
            rows &= rows - 1;
            const long long i = i0 + src;
            const long long a0 = clampll(I.A_rowptr[i], 0, I.annz), a1 = clampll(I.A_rowptr[i + 1], a0, I.annz);
            if (dense) {
                bat_dense_any(p, I, i, a0, a1, false, nullptr, nullptr, err);
                continue;
            }
            wide_range(p, wadd, a0, a1, 32, err);
            __syncwarp();
            const long long out = clampll(I.C_rowptr[i], 0, I.cap);
            const long long out_end = clampll(I.C_rowptr[i + 1], out, I.cap);
            const int tot = wide_emit(wacc, wbm, I.W >> 5, out, out_end, I.C_col, I.C_val, 0, 1, err);
            if (lane == 0 && out + tot != out_end) atomicOr(err, ERR_C_ROW);
            __syncwarp();
            if (lane < (I.W >> 5)) wbm[lane] = 0u;
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// backward: dA(i,k) = sum_j dC(i,j) B(k,j) on A's pattern, dB(k,j) += A(i,k)
// dC(i,j) on B's pattern.  Row i's dC is scattered into a dense shared row;
// groups of four lanes take two entries of A at a time (their segments of B
// on the row-aligned copy, 16-byte loads), reduce dA within the group and
// add the dB terms with float atomics.  A row's entries go in chunks through
// a three-stage pipeline (entries of A, then B's row pointers, then the
// walk), as in the forward's wide rows.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bat_zero_grads(const InstDesc* __restrict__ inst) {
    const InstDesc& I = inst[blockIdx.y];
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
    if (I.dA)
        for (long long e = t0; e < I.annz; e += st) I.dA[e] = 0.0f;
    if (I.dB)
        for (long long e = t0; e < I.bnnz; e += st) I.dB[e] = 0.0f;
}

// Both terms of one 16-byte group of the row-aligned copy (entries j and
// j + 1 of B): dB(k, .) += a * dC(i, col) with float atomics, and the dA
// part B(k, .) * dC(i, col) returned.  Pads carry column -1 and add nothing.
__device__ __forceinline__ float bat_bwd_group(const InstDesc& I, const float* gr, const int4& v, float a,
                                               long long j, unsigned W) {
    float part = 0.0f;
    if ((unsigned)v.x < W) {
        const float g = gr[v.x];
        part = __int_as_float(v.y) * g;
        if (I.dB) atomicAdd(I.dB + j, a * g);
    }
    if ((unsigned)v.z < W) {
        const float g = gr[v.z];
        part = fmaf(__int_as_float(v.w), g, part);
        if (I.dB) atomicAdd(I.dB + j + 1, a * g);
    }
    return part;
}

// The segments of up to 32 entries of A held by the lanes (lane l: entry
// e0 + l, the first group g0 and groups ng of its row of B in the row-aligned
// copy, B's index s of that row's first entry, A's value a) against the
// dense dC row gr.  Groups of four lanes take two segments at a time, lane
// gl their groups gl, gl + 4 (four 16-byte loads in flight before any is
// used); the dA sum of each segment is reduced over its four lanes.
__device__ __forceinline__ void bat_bwd_walk(const InstDesc& I, const float* gr, unsigned g0, int ng, long long s,
                                             float a, int nv, long long e0) {
    const int lane = lane_id(), grp = lane >> 2, gl = lane & 3;
    const unsigned W = (unsigned)I.W;
    const int4* Q = reinterpret_cast<const int4*>(I.Bq);
    const int4 none = make_int4(-1, 0, -1, 0);
    for (int s0 = 0; s0 < nv; s0 += 16) {
        const int ea = s0 + grp, eb = s0 + 8 + grp;
        const unsigned ga = __shfl_sync(FULL, g0, ea & 31), gb = __shfl_sync(FULL, g0, eb & 31);
        int na = __shfl_sync(FULL, ng, ea & 31), nb = __shfl_sync(FULL, ng, eb & 31);
        const long long sa = shfl64(s, ea & 31), sb = shfl64(s, eb & 31);
        const float xa = __shfl_sync(FULL, a, ea & 31), xb = __shfl_sync(FULL, a, eb & 31);
        if (ea >= nv) na = 0;
        if (eb >= nv) nb = 0;
        const int nm = na > nb ? na : nb;
        float pa = 0.0f, pb = 0.0f;
        for (int q = gl; q < nm; q += 8) {
            int4 u0 = none, u1 = none, v0 = none, v1 = none;
            if (q < na) u0 = __ldg(Q + ga + q);
            if (q < nb) v0 = __ldg(Q + gb + q);
            if (q + 4 < na) u1 = __ldg(Q + ga + q + 4);
            if (q + 4 < nb) v1 = __ldg(Q + gb + q + 4);
            pa += bat_bwd_group(I, gr, u0, xa, sa + 2LL * q, W);
            pb += bat_bwd_group(I, gr, v0, xb, sb + 2LL * q, W);
            pa += bat_bwd_group(I, gr, u1, xa, sa + 2LL * (q + 4), W);
            pb += bat_bwd_group(I, gr, v1, xb, sb + 2LL * (q + 4), W);
        }
        pa += __shfl_xor_sync(FULL, pa, 1);
        pb += __shfl_xor_sync(FULL, pb, 1);
        pa += __shfl_xor_sync(FULL, pa, 2);
        pb += __shfl_xor_sync(FULL, pb, 2);
        if (gl == 0 && I.dA) {
            if (ea < nv) I.dA[e0 + ea] = pa;
            if (eb < nv) I.dA[e0 + eb] = pb;
        }
    }
}

// Entry e of A for this lane (ok: inside the chunk) and its row of B in the
// row-aligned copy (ng = 0 when none; a column outside [0, n) is an input
// error).
__device__ __forceinline__ void bat_bwd_entry(const InstDesc& I, long long e, bool ok, int& k, float& a) {
    k = -1;
    a = 0.0f;
    if (ok) {
        k = __ldg(I.A_col + e);
        a = __ldg(I.A_val + e);
    }
}

__device__ __forceinline__ void bat_bwd_seg(const InstDesc& I, int k, unsigned& g0, int& ng, long long& s,
                                            unsigned long long* err) {
    g0 = 0;
    ng = 0;
    s = 0;
    if (k < 0) return;
    if (k < I.n) {
        int len;
        padded_row<2>(I.B_rowptr, I.bnnz, (int)I.d, k, s, len, g0);
        ng = (len + 1) >> 1;
    } else {
        atomicOr(err, ERR_A_COL);
    }
}

// Entries [first, e1) of A's row i, in chunks of cs <= 32 entries at first,
// first + stride, ..., against the dense dC row gr, in three stages: while
// chunk c is walked, the row pointers of B for chunk c + 1 and the entries
// of A of chunk c + 2 are in flight.
__device__ __forceinline__ void bat_bwd_range(const InstDesc& I, const float* gr, long long first, long long e1,
                                              long long stride, int cs, unsigned long long* err) {
    const int lane = lane_id();
    const bool mine = lane < cs;
    int k;
    float a;
    bat_bwd_entry(I, first + lane, mine && first + lane < e1, k, a);
    unsigned g0;
    int ng;
    long long s;
    bat_bwd_seg(I, k, g0, ng, s, err);
    float ca = a;
    bat_bwd_entry(I, first + stride + lane, mine && first + stride + lane < e1, k, a);
    for (long long e = first; e < e1; e += stride) {
        const int nv = e1 - e < cs ? (int)(e1 - e) : cs;
        unsigned g1;
        int ng1;
        long long s1;
        bat_bwd_seg(I, k, g1, ng1, s1, err);  // chunk c + 1
        const float ca1 = a;
        const long long e2 = e + 2 * stride;
        bat_bwd_entry(I, e2 + lane, mine && e2 + lane < e1, k, a);  // chunk c + 2
        bat_bwd_walk(I, gr, g0, ng, s, ca, nv, e);
        g0 = g1;
        ng = ng1;
        s = s1;
        ca = ca1;
    }
}

// Row i of dC scattered into the dense row (or cleared from it) by nt
// threads from t0, four entries per thread in flight.
__device__ __forceinline__ void bat_scatter_dc(const InstDesc& I, long long i, float* row, int t0, int nt,
                                               bool clear) {
    const long long c0 = clampll(I.C_rowptr[i], 0, I.cap), c1 = clampll(I.C_rowptr[i + 1], c0, I.cap);
    for (long long x = c0 + t0; x < c1; x += 4LL * nt) {
        int cc[4];
        float vv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long xu = x + (long long)u * nt;
            cc[u] = xu < c1 ? __ldg(I.C_col + xu) : -1;
            vv[u] = (xu < c1 && !clear) ? __ldg(I.dC + xu) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if ((unsigned)cc[u] < (unsigned)I.W) row[cc[u]] = vv[u];
    }
}

__global__ void __launch_bounds__(256, 4) k_bat_backward(const InstDesc* __restrict__ inst, int count, long long g0,
                                                         long long g1, const long long* __restrict__ flops,
                                                         const int* __restrict__ heavy, BatchCtl* ctl, int Wmax) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;
    const int nwarps = blockDim.x >> 5, warp = warp_id(), lane = lane_id(), tid = threadIdx.x;
    for (int x = tid; x < nwarps * Wmax; x += blockDim.x) reinterpret_cast<float*>(smem)[x] = 0.0f;
    __syncthreads();
    unsigned long long* err = &ctl->err;
    float* wrow = reinterpret_cast<float*>(smem) + (size_t)warp * Wmax;
    float* trow = reinterpret_cast<float*>(smem);  // the block's row (warp 0's)
    const long long nheavy = (long long)ctl->nheavy;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&ctl->q_bwd, 1ull);
        __syncthreads();
        const long long h = s_item;
        __syncthreads();
        if (h >= nheavy) break;
        const long long g = heavy[h];
        const InstDesc& I = inst[inst_of(inst, count, g)];
        const long long i = g - I.row_off;
        if (!I.dC) continue;
        bat_scatter_dc(I, i, trow, tid, blockDim.x, false);
        __syncthreads();
        const long long a0 = clampll(I.A_rowptr[i], 0, I.annz), a1 = clampll(I.A_rowptr[i + 1], a0, I.annz);
        // chunks of 16 entries when the row has too few for every warp to
        // take two chunks of 32
        const int cs = a1 - a0 >= 64LL * nwarps ? 32 : 16;
        bat_bwd_range(I, trow, a0 + (long long)cs * warp, a1, (long long)cs * nwarps, cs, err);
        __syncthreads();
        bat_scatter_dc(I, i, trow, tid, blockDim.x, true);
        __syncthreads();
    }
    const long long nchunks = (g1 - g0 + 31) / 32;
    for (long long ch = bat_next_chunk(&ctl->l_bwd, 0); ch < nchunks; ch = bat_next_chunk(&ctl->l_bwd, 0)) {
        const long long g = g0 + ch * 32 + lane;
        int b;
        unsigned rows = __ballot_sync(FULL, bat_light(inst, count, flops, g, g1, b));
        while (rows) {
            const int src = __ffs(rows) - 1;
            rows &= rows - 1;
            const InstDesc& I = inst[__shfl_sync(FULL, b, src)];
            if (!I.dC) continue;
            const long long i = g0 + ch * 32 + src - I.row_off;
            bat_scatter_dc(I, i, wrow, lane, 32, false);
            __syncwarp();
            const long long a0 = clampll(I.A_rowptr[i], 0, I.annz), a1 = clampll(I.A_rowptr[i + 1], a0, I.annz);
            bat_bwd_range(I, wrow, a0, a1, 32, 32, err);
            __syncwarp();
            bat_scatter_dc(I, i, wrow, lane, 32, true);
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// bounds: sum over the rows of min(d_b, flops_i); block per instance
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_batch_bounds(const InstDesc* __restrict__ inst, const long long* flops,
                                                      long long* bound) {
    const InstDesc& I = inst[blockIdx.x];
    long long s = 0;
    for (long long i = threadIdx.x; i < I.n; i += blockDim.x) {
        const long long f = flops[I.row_off + i];
        s += f < I.d ? f : I.d;
    }
    s = warp_sum(s);
    __shared__ long long red[8];
    if (lane_id() == 0) red[warp_id()] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        bound[blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_bat_prepare(const InstDesc* inst, int count, long long c0, long long c1, long long* flops,
                               int* heavy, BatchCtl* ctl, int sms, cudaStream_t st) {
    if (c1 <= c0) return cudaSuccess;
    long long grid = persistent_grid((const void*)k_bat_prepare, 256, 0, sms);
    if (grid > (c1 - c0 + 7) / 8) grid = (c1 - c0 + 7) / 8;
    count_launch();
    k_bat_prepare<<<(unsigned)grid, 256, 0, st>>>(inst, count, c0, c1, flops, heavy, ctl);
    return cudaGetLastError();
}

cudaError_t launch_bat_symbolic(const InstDesc* inst, int count, long long c0, long long c1, long long,
                                const long long* flops, const int* heavy, BatchCtl* ctl, int Wmax, int sms,
                                cudaStream_t st) {
    if (c1 <= c0) return cudaSuccess;
    if (Wmax < 32 || Wmax > 1024 || (Wmax & 31)) return cudaErrorInvalidValue;
    const size_t smem = 8 * 4 * (size_t)(Wmax + 32);
    const int grid = persistent_grid((const void*)k_bat_symbolic, 256, smem, sms);
    count_launch();
    k_bat_symbolic<<<grid, 256, smem, st>>>(inst, count, c0, c1, flops, heavy, ctl, Wmax);
    return cudaGetLastError();
}

cudaError_t launch_bat_scan(const InstDesc* inst, int count, BatchCtl* ctl, cudaStream_t st) {
    if (count < 1) return cudaSuccess;
    count_launch();
    k_bat_scan<<<count, 1024, 0, st>>>(inst, ctl);
    return cudaGetLastError();
}

cudaError_t launch_bat_numeric(const InstDesc* inst, int count, long long c0, long long c1, long long values,
                               const long long* flops, const int* heavy, BatchCtl* ctl, int Wmax, int sms,
                               cudaStream_t st) {
    if (c1 <= c0) return cudaSuccess;
    if (Wmax < 32 || Wmax > 1024 || (Wmax & 31)) return cudaErrorInvalidValue;
    const size_t smem = 4 * (8 * (size_t)bat_per_warp(Wmax, values != 0) + (values && Wmax <= 256 ? Wmax : 0));
    cudaError_t e;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute((const void*)k_bat_numeric, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    const int grid = persistent_grid((const void*)k_bat_numeric, 256, smem, sms);
    count_launch();
    k_bat_numeric<<<grid, 256, smem, st>>>(inst, count, c0, c1, flops, heavy, ctl, Wmax, values != 0);
    return cudaGetLastError();
}

cudaError_t launch_bat_backward(const InstDesc* inst, int count, long long g0, long long g1, long long max_work,
                                const long long* flops, const int* heavy, BatchCtl* ctl, int Wmax, int sms,
                                cudaStream_t st) {
    if (g1 <= g0 || count < 1) return cudaSuccess;
    if (Wmax < 32 || Wmax > 1024 || (Wmax & 31)) return cudaErrorInvalidValue;
    long long gx = (max_work + 255) / 256;
    if (gx < 1) gx = 1;
    if (gx > 64) gx = 64;
    count_launch();
    k_bat_zero_grads<<<dim3((unsigned)gx, count), 256, 0, st>>>(inst);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    const size_t smem = 8 * 4 * (size_t)Wmax;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute((const void*)k_bat_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    const int grid = persistent_grid((const void*)k_bat_backward, 256, smem, sms);
    count_launch();
    k_bat_backward<<<grid, 256, smem, st>>>(inst, count, g0, g1, flops, heavy, ctl, Wmax);
    return cudaGetLastError();
}

cudaError_t launch_batch_bounds(const InstDesc* inst, int count, const long long* flops, long long* bound,
                                cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    count_launch();
    k_batch_bounds<<<count, 256, 0, st>>>(inst, flops, bound);
    return cudaGetLastError();
}

}  // namespace ts
