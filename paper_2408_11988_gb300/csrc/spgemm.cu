// Forward TS-SpGEMM kernels: row flops, row binning, symbolic pass, scan,
// column-tile split and the dense-accumulator numeric pass (paper Sec. III-A,
// Eq. 1; accumulator per Sec. III-C).
#include <atomic>
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace ts {

// ---------------------------------------------------------------------------
// Row flops: flops_i = sum over stored (i,k) of nnz(B_k) (paper Sec. II-A:
// flops = number of multiplications).  Rows of at most SHORT_ROW entries are
// summed by the warp that holds them (32 rows per warp, their entries read
// together).  Longer rows are cut into chunks of LONG_CHUNK
// entries, queued as (row, chunk) items, and each chunk is summed by one
// warp and added to its row with an atomic, so a row with very many entries
// is spread over many warps.
// ---------------------------------------------------------------------------
constexpr int SHORT_ROW = 256;
constexpr int LONG_CHUNK = 256;

// Row lengths of B clamped as SegWhole clamps them, as one int32 array: the
// flops pass then reads one 4-byte word per entry of A from an array that
// stays in L2 instead of two 8-byte row pointers.
__global__ void __launch_bounds__(256) k_row_len(long long nB, SegWhole segB, int* __restrict__ blen) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nB;
         k += (long long)gridDim.x * blockDim.x) {
        long long s0;
        int len;
        segB((int)k, s0, len);
        blen[k] = len;
    }
}

struct SegLen {
    const int* __restrict__ blen;
    __device__ __forceinline__ void operator()(int k, long long& start, int& len) const {
        start = 0;
        len = __ldg(blen + k);
    }
};

template <class Seg>
__global__ void __launch_bounds__(256) k_flops_rows(long long n, const long long* __restrict__ Ap,
                                                    const int* __restrict__ Ai, long long nnzA,
                                                    Seg segB, int nB, long long* __restrict__ flops,
                                                    long long* __restrict__ items, long long item_cap,
                                                    WsHeader* hdr) {
    __shared__ long long s_f[256];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = lane_id();
    unsigned long long* err = &hdr->err;
    long long nchunks = 0;
    long long a0 = 0;
    int len = 0;  // entries of this lane's row summed here (short rows)
    if (i < n) {
        a0 = clampll(__ldg(Ap + i), 0, nnzA);
        const long long a1 = clampll(__ldg(Ap + i + 1), a0, nnzA);
        if (a1 - a0 <= SHORT_ROW) len = (int)(a1 - a0);
        else nchunks = (a1 - a0 + LONG_CHUNK - 1) / LONG_CHUNK;
    }
    long long* wf = s_f + (threadIdx.x & ~31);
    wf[lane] = 0;
    __syncwarp();
    // The short rows of the warp's 32 rows hold consecutive entries of A: they
    // are numbered across the rows and read 32 at a time (coalesced); each
    // entry's B row length goes to its row by a segmented sum over the lanes
    // (the row of entry p is the last lane whose first number is <= p).
    const int incl = warp_incl_scan(len), excl = incl - len;
    const int total = __shfl_sync(FULL, incl, 31);
    const long long shift = a0 - excl;  // entry of number p in row q: shift(q) + p
    for (int p0 = 0; p0 < total; p0 += 32) {
        const int p = p0 + lane;
        const int q = owner_lane(excl, p);
        const long long e = shfl64(shift, q) + p;
        long long v = 0;
        if (p < total) {
            const int k = __ldg(Ai + e);
            if ((unsigned)k < (unsigned)nB) {
                long long s0;
                int l;
                segB(k, s0, l);
                v = l;
            } else {
                atomicOr(err, ERR_A_COL);
            }
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {  // sum over this lane's run of equal q, from this lane on
            const long long t = shfl64_down(v, o);
            const int qo = __shfl_down_sync(FULL, q, o);
            if (lane + o < 32 && qo == q) v += t;
        }
        const int qp = __shfl_up_sync(FULL, q, 1);
        if (p < total && (lane == 0 || qp != q)) wf[q] += v;  // one lane per row and step
        __syncwarp();
    }
    if (i < n) flops[i] = nchunks ? 0 : wf[lane];
    // reserve item slots: one atomic per warp
    long long cincl = warp_incl_scan(nchunks);
    const long long tot = __shfl_sync(FULL, cincl, 31);
    long long base = 0;
    if (tot > 0) {
        if (lane == 31) base = (long long)atomicAdd((unsigned long long*)&hdr->scratch[0], (unsigned long long)tot);
        base = __shfl_sync(FULL, base, 31);
    }
    for (long long c = 0; c < nchunks; ++c) {
        const long long slot = base + cincl - nchunks + c;
        if (slot < item_cap) items[slot] = (i << 24) | c;
        else atomicOr(err, ERR_CAPACITY);
    }
}

template <class Seg>
__global__ void __launch_bounds__(256) k_flops_chunks(const long long* __restrict__ Ap,
                                                      const int* __restrict__ Ai, long long nnzA,
                                                      Seg segB, int nB, long long* flops,
                                                      const long long* __restrict__ items,
                                                      long long item_cap, WsHeader* hdr) {
    const long long nitems_raw = *(volatile long long*)&hdr->scratch[0];
    const long long nitems = nitems_raw < item_cap ? nitems_raw : item_cap;
    const int lane = lane_id();
    unsigned long long* err = &hdr->err;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long it = gw; it < nitems; it += nwarps) {
        const long long item = items[it];
        const long long row = item >> 24, c = item & 0xFFFFFF;
        const long long a0 = clampll(__ldg(Ap + row), 0, nnzA);
        const long long a1 = clampll(__ldg(Ap + row + 1), a0, nnzA);
        const long long e0 = a0 + c * LONG_CHUNK;
        const long long e1 = e0 + LONG_CHUNK < a1 ? e0 + LONG_CHUNK : a1;
        long long f = 0;
#pragma unroll
        for (int u = 0; u < LONG_CHUNK / 32; ++u) {
            const long long e = e0 + u * 32 + lane;
            if (e < e1) {
                const int k = __ldg(Ai + e);
                if ((unsigned)k < (unsigned)nB) {
                    long long s0;
                    int len;
                    segB(k, s0, len);
                    f += len;
                } else {
                    atomicOr(err, ERR_A_COL);
                }
            }
        }
        f = warp_sum(f);
        if (lane == 0 && f) atomicAdd((unsigned long long*)(flops + row), (unsigned long long)f);
    }
}

// Room for the (row, chunk) items: rows longer than SHORT_ROW are at most
// nnzA / (SHORT_ROW + 1), and their chunks add at most nnzA / LONG_CHUNK.
long long flops_item_capacity(long long n, long long nnzA) {
    long long rows = nnzA / (SHORT_ROW + 1) + 1;
    if (rows > n) rows = n;
    return rows + nnzA / LONG_CHUNK + 1;
}

// Class histogram of the rows (class 0 = no products); rows without products
// get their output count (0) right away.
__global__ void __launch_bounds__(256) k_classify(long long n, const long long* __restrict__ flops,
                                                  long long* Cp_next, WsHeader* hdr) {
    __shared__ unsigned s_hist[NUM_CLASSES];
    for (int c = threadIdx.x; c < NUM_CLASSES; c += blockDim.x) s_hist[c] = 0;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = flops_class(flops[i]);
        atomicAdd(&s_hist[c], 1u);
        if (c == 0 && Cp_next) Cp_next[i] = 0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < NUM_CLASSES; c += blockDim.x)
        if (s_hist[c]) atomicAdd((unsigned long long*)&hdr->hist[c], (unsigned long long)s_hist[c]);
}

// perm = rows with products, heaviest class first (order inside a class is
// arbitrary).  Each block ranks its rows per class in shared memory and
// reserves one range per class with a single global atomic.
constexpr int SCATTER_ROWS = 8;  // rows per thread
__global__ void __launch_bounds__(256) k_scatter(long long n, const long long* __restrict__ flops,
                                                 int* __restrict__ perm, WsHeader* hdr) {
    __shared__ unsigned s_cnt[NUM_CLASSES];
    __shared__ long long s_start[NUM_CLASSES];
    __shared__ long long s_base[NUM_CLASSES];
    const int tid = threadIdx.x;
    for (int c = tid; c < NUM_CLASSES; c += blockDim.x) s_cnt[c] = 0;
    if (tid < 32) {  // start of class c = rows of the classes above it (warp scan, highest class first)
        long long run = 0;
        for (int top = NUM_CLASSES - 1; top >= 1; top -= 32) {
            const int c = top - tid;
            const long long h = c >= 1 ? hdr->hist[c] : 0;
            const long long incl = warp_incl_scan(h);
            if (c >= 1) s_start[c] = run + incl - h;
            run += __shfl_sync(FULL, incl, 31);
        }
        if (tid == 0) s_start[0] = run;
    }
    __syncthreads();
    const long long base = (long long)blockIdx.x * blockDim.x * SCATTER_ROWS;
    int cls[SCATTER_ROWS];
    unsigned rank[SCATTER_ROWS];
#pragma unroll
    for (int u = 0; u < SCATTER_ROWS; ++u) {
        const long long i = base + (long long)u * blockDim.x + tid;
        cls[u] = 0;
        if (i < n) {
            cls[u] = flops_class(flops[i]);
            if (cls[u] > 0) rank[u] = atomicAdd(&s_cnt[cls[u]], 1u);
        }
    }
    __syncthreads();
    for (int c = tid; c < NUM_CLASSES; c += blockDim.x)
        s_base[c] = (c > 0 && s_cnt[c])
                        ? (long long)atomicAdd((unsigned long long*)&hdr->cursor[c], (unsigned long long)s_cnt[c])
                        : 0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < SCATTER_ROWS; ++u) {
        const long long i = base + (long long)u * blockDim.x + tid;
        if (i < n && cls[u] > 0) perm[s_start[cls[u]] + s_base[cls[u]] + rank[u]] = (int)i;
    }
}

cudaError_t launch_row_flops(const DevCsr& A, const DevCsr& B, const Sched& s, cudaStream_t st) {
    const long long n = A.nrows;
    cudaError_t e;
    if ((e = cudaMemsetAsync(s.hdr, 0, sizeof(WsHeader), st))) return e;
    if (n == 0) return cudaSuccess;
    const SegWhole segB{B.rowptr, B.nnz, (int)B.ncols};
    const long long cap = flops_item_capacity(n, A.nnz);
    const unsigned rb = (unsigned)((n + 255) / 256);
    if (s.blen && B.nrows > 0) {
        long long lb = (B.nrows + 255) / 256;
        if (lb > 152 * 16) lb = 152 * 16;
        count_launch();
        k_row_len<<<(unsigned)lb, 256, 0, st>>>(B.nrows, segB, s.blen);
        const SegLen sl{s.blen};
        count_launch();
        k_flops_rows<<<rb, 256, 0, st>>>(n, A.rowptr, A.col, A.nnz, sl, (int)B.nrows, s.flops, s.items, cap, s.hdr);
        count_launch();
        k_flops_chunks<<<152 * 8, 256, 0, st>>>(A.rowptr, A.col, A.nnz, sl, (int)B.nrows, s.flops, s.items, cap,
                                                s.hdr);
    } else {
        count_launch();
        k_flops_rows<<<rb, 256, 0, st>>>(n, A.rowptr, A.col, A.nnz, segB, (int)B.nrows, s.flops, s.items, cap,
                                         s.hdr);
        count_launch();
        k_flops_chunks<<<152 * 8, 256, 0, st>>>(A.rowptr, A.col, A.nnz, segB, (int)B.nrows, s.flops, s.items,
                                                cap, s.hdr);
    }
    return cudaGetLastError();
}

cudaError_t launch_reclassify(long long n, const Sched& s, long long* Cp_next, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(s.hdr->hist, 0, sizeof(long long) * 2 * NUM_CLASSES, st))) return e;
    if (n == 0) return cudaSuccess;
    long long cb = (n + 255) / 256;
    if (cb > 152 * 16) cb = 152 * 16;
    count_launch();
    k_classify<<<(unsigned)cb, 256, 0, st>>>(n, s.flops, Cp_next, s.hdr);
    const long long sb = (n + 256LL * SCATTER_ROWS - 1) / (256LL * SCATTER_ROWS);
    count_launch();
    k_scatter<<<(unsigned)sb, 256, 0, st>>>(n, s.flops, s.perm, s.hdr);
    return cudaGetLastError();
}

cudaError_t launch_row_schedule(const DevCsr& A, const DevCsr& B, const Sched& s, long long* Cp,
                                cudaStream_t st) {
    cudaError_t e;
    if ((e = launch_row_flops(A, B, s, st))) return e;
    return launch_reclassify(A.nrows, s, Cp ? Cp + 1 : nullptr, st);
}

// ---------------------------------------------------------------------------
// Split rows: a row with more than SPLIT_ENTRIES entries of A (and some
// products) gets a slot u < MAX_SPLIT_ROWS and ceil(len / SPLIT_ENTRIES)
// work items (u, part) that any block may take, so that one very heavy row
// is spread over many SMs instead of forming the tail of the pass.  The
// row's flops entry becomes the mark -1 - u, and its staging slot is cleared.
// ---------------------------------------------------------------------------
long long split_item_capacity(long long nnzA) { return nnzA / SPLIT_ENTRIES + MAX_SPLIT_ROWS + 1; }

__global__ void __launch_bounds__(256) k_split_rows(long long n, const long long* __restrict__ Ap, long long nnzA,
                                                    long long* flops, Sched s, long long item_cap) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long a0 = clampll(Ap[i], 0, nnzA), a1 = clampll(Ap[i + 1], a0, nnzA);
    const long long alen = a1 - a0;
    if (alen <= SPLIT_ENTRIES || flops[i] <= 0) return;
    const long long u = (long long)atomicAdd((unsigned long long*)&s.hdr->scratch[1], 1ull);
    if (u >= MAX_SPLIT_ROWS) return;  // out of slots: the row runs whole
    const long long nsub = (alen + SPLIT_ENTRIES - 1) / SPLIT_ENTRIES;
    const long long base = (long long)atomicAdd((unsigned long long*)&s.hdr->scratch[2], (unsigned long long)nsub);
    if (base + nsub > item_cap) {
        atomicOr(&s.hdr->err, ERR_CAPACITY);
        return;
    }
    for (int w = 0; w < s.dw; ++w) s.stg_bits[u * s.dw + w] = 0u;
    if (s.stg_vals) {
        float4* v = reinterpret_cast<float4*>(s.stg_vals + u * s.dpad);
        unsigned* f = reinterpret_cast<unsigned*>(s.stg_flags + u * s.dpad);
        for (int c = 0; c < s.dpad / 4; ++c) {
            v[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            f[c] = 0u;
        }
    }
    s.split_rows[u] = (int)i;
    s.split_done[u] = 0;
    for (long long q = 0; q < nsub; ++q) s.split_items[base + q] = (u << 32) | q;
    flops[i] = -1 - u;
}


// ---------------------------------------------------------------------------
// Symbolic pass: nnz(C_i) = number of distinct columns over the rows B_k,
// k in A_i (Eq. 1 on patterns).  The columns of a row are collected in one
// occupancy byte per column (FL, for d up to SYM_FLAG_MAX_D) or one bit per
// column (wide d) per warp, shared by the whole block for heavy rows; the
// count is a population count.  Byte marks are plain stores of the value 1:
// lanes that mark the same column at the same time store the same value, so
// no atomic is needed; bits are set with shared-memory atomicOr.
// ---------------------------------------------------------------------------
constexpr int SYM_FLAG_MAX_D = 4096;

template <bool FL>
struct SymVisit {
    const int* __restrict__ Bi;
    unsigned* bm;  // bitmap words, or (FL) dpad occupancy bytes
    int d;
    unsigned long long* err;
    long long nnzB;
    struct Item {
        int c;
    };
    __device__ __forceinline__ Item fetch(long long j) const { return Item{__ldg(Bi + j)}; }
    __device__ __forceinline__ void apply(const Item& it, float, long long, int) { mark(it.c); }
    template <int G>
    __device__ __forceinline__ void done(int, int, int, long long) {}
    __device__ __forceinline__ void mark(int c) {
        if ((unsigned)c < (unsigned)d) {
            if (FL) reinterpret_cast<unsigned char*>(bm)[c] = 1;
            else atomicOr(bm + (c >> 5), 1u << (c & 31));
        } else {
            atomicOr(err, ERR_B_COL);
        }
    }
    __device__ __forceinline__ void step4(const long long* j, const float*, const int*) {
        int c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = __ldg(Bi + j[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) mark(c[u]);
    }
    __device__ __forceinline__ void step1(long long j, float, int, bool ok) {
        if (ok) mark(__ldg(Bi + j));
    }
    // quads: one 16-byte load of four columns (Bi is 16-byte aligned), or
    // single loads for a quad that reaches past the end of B
    __device__ __forceinline__ void quads(const Chunk& ch, int nv) {
        quads_loaded(ch, nv, [&](long long qb, long long s, long long end, float) {
            int c[4];
            if (qb + 4 <= nnzB) {
                const int4 v = __ldg(reinterpret_cast<const int4*>(Bi + qb));
                c[0] = v.x;
                c[1] = v.y;
                c[2] = v.z;
                c[3] = v.w;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) c[u] = qb + u < end ? __ldg(Bi + qb + u) : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (qb + u >= s && qb + u < end) mark(c[u]);
        });
    }
};

struct SymParams {
    const long long* Ap;
    const int* Ai;
    long long nnzA;
    SegWhole segB;
    const int* Bi;
    int nB;
    int d;
    int dw;    // bitmap words per row (d/32 rounded up)
    int slot;  // shared-memory words per warp: dw, or (FL) dw * 8 for the bytes
    const int* perm;
    WsHeader* hdr;
    int cta_class;
    long long* Cp_next;
    Sched s;
    long long item_cap;
    int skip_light;  // 1: split and heavy rows only (light rows run in k_symbolic_light)
    int tiny;        // 1: light rows of classes <= SYM_TINY_CLASS are counted by k_symbolic_tiny
};

// Rows with at most 31 products (flops classes 1 .. 40, eighths of an
// octave) are the symbolic pass's tiny rows when k_symbolic_tiny runs.
constexpr int SYM_TINY_CLASS = 40;
static_assert(SYM_TINY_CLASS < NUM_CLASSES, "tiny classes");

// Count of the marks in words [w0, dw*8 or dw) of a warp's or block's
// marks, stride `step`, clearing them.
template <bool FL>
__device__ __forceinline__ int count_and_clear(unsigned* bm, int dw, int w0, int step) {
    int c = 0;
    const int words = FL ? 8 * dw : dw;  // FL: bytes are 0 or 1, four per word
    for (int w = w0; w < words; w += step) {
        c += __popc(bm[w]);
        bm[w] = 0u;
    }
    return c;
}

template <int G, bool FL, class Seg>
__device__ __forceinline__ void sym_chunk(const SymParams& p, long long e0, int nv, SymVisit<FL>& vis,
                                          unsigned long long* err) {
    if constexpr (G == 1) expand_chunk(e0, nv, p.Ai, (const float*)nullptr, p.nB, p.segB, vis, err);
    else if constexpr (G == 2) vis.quads(load_chunk(e0, nv, p.Ai, (const float*)nullptr, p.nB, p.segB, err), nv);
    else grouped_chunk<G>(e0, nv, p.Ai, (const float*)nullptr, p.nB, p.segB, vis, err);
}

// Light row of the symbolic pass, driven by pipelined_rows.
template <int G, bool FL>
struct SymRowBody {
    const SymParams& p;
    unsigned* bm;
    unsigned long long* err;
    __device__ __forceinline__ void gather(int, long long a0, long long a1, const Chunk& ch0, int nv0, int) {
        SymVisit<FL> vis{p.Bi, bm, p.d, err, p.segB.nnzB};
        expand_any<G>(ch0, nv0, a0, vis);
        for (long long e0 = a0 + 32; e0 < a1; e0 += 32) {
            const int nv = (int)(a1 - e0 < 32 ? a1 - e0 : 32);
            expand_any<G>(load_chunk(e0, nv, p.Ai, (const float*)nullptr, p.nB, p.segB, err), nv, e0, vis);
        }
    }
    __device__ __forceinline__ void finish(int row) {
        __syncwarp();
        const int c = warp_sum(count_and_clear<FL>(bm, p.dw, lane_id(), 32));
        if (lane_id() == 0) p.Cp_next[row] = c;
        __syncwarp();
    }
};

// Marks set so far in the block's marks (all lanes of the calling warp get
// the count; marks other warps are still setting may be missed, which only
// delays the test below).
template <bool FL>
__device__ __forceinline__ int count_marks_warp(const unsigned* bm, int dw) {
    const int words = FL ? 8 * dw : dw;
    int c = 0;
    for (int w = lane_id(); w < words; w += 32) c += __popc(((const volatile unsigned*)bm)[w]);
    return warp_sum(c);
}

// A warp's chunks [first, a1) (stride 32 * warps) of a heavy row or split
// part, marked into the block's marks.  Once all d columns are marked the
// row's count is d whatever the remaining products, so the block stops: after
// each of its chunks a warp counts the marks and raises *full when they
// reach d, and every warp reads *full before its next chunk.  (Columns of B
// in the skipped products are not range-checked here; the numeric pass checks
// every entry of B.)
template <int G, bool FL>
__device__ __forceinline__ void sym_range(const SymParams& p, long long first, long long a1, long long stride,
                                          SymVisit<FL>& vis, volatile int* full, unsigned long long* err) {
    const bool test = p.dw <= 32;  // counting costs a pass over the marks: d <= 1024 only
    for (long long e0 = first; e0 < a1; e0 += stride) {
        if (*full) break;
        sym_chunk<G, FL, SegWhole>(p, e0, (int)(a1 - e0 < 32 ? a1 - e0 : 32), vis, err);
        if (test && count_marks_warp<FL>(vis.bm, p.dw) >= p.d && lane_id() == 0) *full = 1;
    }
}

// Block total of per-thread counts (all threads get it).
__device__ __forceinline__ int block_sum(int c, int* s_red) {
    const int nw = blockDim.x >> 5, warp = warp_id(), lane = lane_id();
    c = warp_sum(c);
    if (lane == 0) s_red[warp] = c;
    __syncthreads();
    int v = lane < nw ? s_red[lane] : 0;
    v = warp_sum(v);
    __syncthreads();
    return v;
}

// Tiny rows (light, at most 31 products) counted in registers: a row of one
// entry of A has as many columns as its row of B (flops_i itself); a longer
// one has its rows of B's columns placed one per lane, sorted (two rows: one
// bitonic merge of the first row and the second reversed at the top lanes;
// more: the full network) and the distinct ones counted.  32-row chunks are
// dealt to the warps in turn; the one-entry rows of a chunk are counted lane
// by lane.  Called when d is too wide for the row-group light kernel, where
// each light row costs a pass over d/4 words of byte marks.
__device__ __forceinline__ void warp_sort_keys(int& key) {
    const int lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int pk = __shfl_xor_sync(FULL, key, j);
            const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
            if (keep_min ? pk < key : pk > key) key = pk;
        }
    }
}

__global__ void __launch_bounds__(256) k_symbolic_tiny(SymParams p) {
    const int lane = lane_id();
    unsigned long long* err = &p.hdr->err;
    const long long* flops = p.s.flops;
    const long long nchunks = ((long long)p.nB + 31) / 32;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long c = gw; c < nchunks; c += nwarps) {
        const long long r = c * 32 + lane;
        const long long f = r < p.nB ? __ldg(flops + r) : 0;
        const int cls = flops_class(f);
        const bool tiny = f >= 1 && cls <= SYM_TINY_CLASS && cls < p.cta_class;
        long long a0 = 0, a1 = 0;
        if (tiny) {
            a0 = clampll(__ldg(p.Ap + r), 0, p.nnzA);
            a1 = clampll(__ldg(p.Ap + r + 1), a0, p.nnzA);
            if (a1 - a0 == 1) p.Cp_next[r] = f;  // one row of B: its columns, all distinct
        }
        unsigned rows = __ballot_sync(FULL, tiny && a1 - a0 > 1);
        while (rows) {
            const int src = __ffs(rows) - 1;
            rows &= rows - 1;
            const long long b0 = shfl64(a0, src), b1 = shfl64(a1, src);
            int key = 0x7FFFFFFF;  // no column: sorts last
            if (b1 - b0 == 2) {
                long long s0, s1;
                int n0, n1;
                const int k0 = __ldg(p.Ai + b0), k1 = __ldg(p.Ai + b0 + 1);
                n0 = n1 = 0;
                s0 = s1 = 0;
                if ((unsigned)k0 < (unsigned)p.nB) p.segB(k0, s0, n0);
                else if (lane == 0) atomicOr(err, ERR_A_COL);
                if ((unsigned)k1 < (unsigned)p.nB) p.segB(k1, s1, n1);
                else if (lane == 0) atomicOr(err, ERR_A_COL);
                if (n0 + n1 <= 32) {
                    const int j1 = 31 - lane;  // the second row, reversed, at the top lanes
                    int col = -1;
                    if (lane < n0) col = __ldg(p.Bi + s0 + lane);
                    else if (j1 < n1) col = __ldg(p.Bi + s1 + j1);
                    if ((unsigned)col < (unsigned)p.d) key = col;
                    else if (col != -1) atomicOr(err, ERR_B_COL);
#pragma unroll
                    for (int j = 16; j > 0; j >>= 1) {
                        const int pk = __shfl_xor_sync(FULL, key, j);
                        if (((lane & j) == 0) ? pk < key : pk > key) key = pk;
                    }
                    const int prev = __shfl_up_sync(FULL, key, 1);
                    const unsigned heads = __ballot_sync(FULL, key != 0x7FFFFFFF && (lane == 0 || prev != key));
                    if (lane == 0) p.Cp_next[c * 32 + src] = __popc(heads);
                    continue;
                }
            }
            int base = 0;  // columns placed so far (warp-uniform)
            for (long long ec = b0; ec < b1 && base < 32; ec += 32) {
                const long long e = ec + lane;
                int len = 0;
                long long st = 0;
                if (e < b1) {
                    const int k = __ldg(p.Ai + e);
                    if ((unsigned)k < (unsigned)p.nB) p.segB(k, st, len);
                    else atomicOr(err, ERR_A_COL);
                }
                const int incl = warp_incl_scan(len), excl = incl - len;
                const int tot = __shfl_sync(FULL, incl, 31);
                const int pj = lane - base;
                const int q = owner_lane(excl, pj < 0 ? 0 : pj);
                const long long sq = shfl64(st, q);
                const int eq = __shfl_sync(FULL, excl, q);
                if (pj >= 0 && pj < tot) {
                    const int col = __ldg(p.Bi + sq + (pj - eq));
                    if ((unsigned)col < (unsigned)p.d) key = col;
                    else atomicOr(err, ERR_B_COL);
                }
                base += tot;
            }
            warp_sort_keys(key);
            const int prev = __shfl_up_sync(FULL, key, 1);
            const unsigned heads = __ballot_sync(FULL, key != 0x7FFFFFFF && (lane == 0 || prev != key));
            if (lane == 0) p.Cp_next[c * 32 + src] = __popc(heads);
        }
    }
}

template <int G, bool FL>
__global__ void __launch_bounds__(256, 8) k_symbolic(SymParams p) {
    // a light-row kernel launched behind this one may start on SMs this grid
    // frees (the two count disjoint rows)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(16) unsigned smem_u[];
    __shared__ long long s_item, s_nheavy, s_nrows;
    __shared__ int s_red[32];
    __shared__ int s_full;  // the current item's marks hold all d columns
    const int nw = blockDim.x >> 5, warp = warp_id(), lane = lane_id(), tid = threadIdx.x;
    for (int i = tid; i < nw * p.slot; i += blockDim.x) smem_u[i] = 0;
    if (tid == 0) s_full = 0;
    if (tid < 32) {  // one warp; its lanes store the same values
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
        s_nrows = nr;
    }
    __syncthreads();
    const long long nheavy = s_nheavy, nrows = s_nrows;
    unsigned long long* err = &p.hdr->err;
    const long long* mark = p.s.flops;

    // split rows: parts of very long rows, any block; partial bitmaps are OR-ed
    // into the row's staging slot and the last part counts the row
    {
        const long long nitems = min(*(volatile long long*)&p.hdr->scratch[2], p.item_cap);
        __shared__ int s_last;
        SplitItem it;
        while (next_split_item(p.s, p.Ap, p.nnzA, nitems, &s_item, it)) {
            SymVisit<FL> vis{p.Bi, smem_u, p.d, err, p.segB.nnzB};
            sym_range<G, FL>(p, it.e0 + 32LL * warp, it.e1, 32LL * nw, vis, &s_full, err);
            __syncthreads();
            if (tid == 0) s_full = 0;  // read again only after the next barrier
            unsigned* stg = p.s.stg_bits + (size_t)it.slot * p.dw;
            if (FL) {  // bytes -> bitmap words by ballot, one word per warp step
                const unsigned char* fb = reinterpret_cast<const unsigned char*>(smem_u);
                for (int w = warp; w < p.dw; w += nw) {
                    const unsigned v = __ballot_sync(FULL, fb[w * 32 + lane] != 0);
                    if (lane == 0 && v) atomicOr(stg + w, v);
                }
                __syncthreads();
                for (int w = tid; w < 8 * p.dw; w += blockDim.x) smem_u[w] = 0u;
            } else {
                for (int w = tid; w < p.dw; w += blockDim.x) {
                    const unsigned v = smem_u[w];
                    if (v) {
                        atomicOr(stg + w, v);
                        smem_u[w] = 0u;
                    }
                }
            }
            if (split_part_done(p.s, it.slot, it.nsub, &s_last)) {
                int c = 0;
                for (int w = tid; w < p.dw; w += blockDim.x) {
                    c += __popc(__ldcg(stg + w));
                    stg[w] = 0u;
                }
                c = block_sum(c, s_red);
                if (tid == 0) {
                    p.Cp_next[it.row] = c;
                    p.s.split_done[it.slot] = 0;
                }
                __syncthreads();
            }
        }
    }

    // heavy rows: one block per row, dynamic
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
        SymVisit<FL> vis{p.Bi, smem_u, p.d, err, p.segB.nnzB};
        sym_range<G, FL>(p, a0 + 32LL * warp, a1, 32LL * nw, vis, &s_full, err);
        __syncthreads();
        if (tid == 0) s_full = 0;  // read again only after the next barrier
        const int c = block_sum(count_and_clear<FL>(smem_u, p.dw, tid, blockDim.x), s_red);
        if (tid == 0) p.Cp_next[row] = c;
    }

    // light rows: one warp per row, static round robin over the class order
    // (highest first: the tiny rows, when k_symbolic_tiny counts them, are
    // the last ones)
    if (p.skip_light) return;
    long long nlight_end = nrows;
    if (p.tiny) {
        long long t = 0;
        for (int c = 1 + lane; c <= SYM_TINY_CLASS && c < p.cta_class; c += 32) t += p.hdr->hist[c];
        nlight_end -= warp_sum(t);
    }
    unsigned* bm = smem_u + warp * p.slot;
    SymRowBody<G, FL> body{p, bm, err};
    pipelined_rows(p.perm, nheavy + (long long)blockIdx.x * nw + warp, nlight_end, (long long)gridDim.x * nw,
                   p.Ap, p.nnzA, p.Ai, (const float*)nullptr, p.nB, p.segB, err, body, mark);
}


// Light rows of the symbolic pass in row groups (byte marks, B.col 16-byte
// aligned): R = 32/RG rows of the schedule per warp in lockstep, RG lanes per
// row, each row with its own dpad occupancy bytes.  A slot walks the
// segments B(k,:) of its row's entries in quads (one 16-byte load of four
// columns, single loads for a quad that reaches past the end of B).  Marks
// are plain byte stores of the value 1, so segments need no ordering among
// themselves; two segments are loaded before either is marked.  The count of
// a row is a popcount over its bytes, summed over the slot's lanes.
// Launched behind k_symbolic with programmatic dependent launch; waits for
// that grid before exiting.
__device__ __forceinline__ void symrg_quad(const int* __restrict__ Bi, long long nnzB, long long qb, long long s,
                                           long long end, int c[4]) {
    if (qb + 4 <= nnzB) {
        const int4 v = __ldg(reinterpret_cast<const int4*>(Bi + qb));
        c[0] = v.x;
        c[1] = v.y;
        c[2] = v.z;
        c[3] = v.w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = qb + u < end ? __ldg(Bi + qb + u) : -1;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (qb + u < s || qb + u >= end) c[u] = -1;
}

__device__ __forceinline__ void symrg_mark(unsigned char* fl, const int c[4], int d, unsigned long long* err) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if (c[u] >= 0) {
            if (c[u] < d) fl[c[u]] = 1;
            else atomicOr(err, ERR_B_COL);
        }
    }
}

template <int RG>
__global__ void __launch_bounds__(256, 5) k_symbolic_light(SymParams p) {
    extern __shared__ __align__(16) unsigned smem_u[];
    __shared__ long long s_nheavy, s_nrows;
    constexpr int R = 32 / RG;
    const int nw = blockDim.x >> 5, warp = warp_id(), lane = lane_id(), tid = threadIdx.x;
    const int g = lane / RG, gl = lane % RG;
    const int slotw = 8 * p.dw;  // words of one row's dpad bytes
    for (int i = tid; i < nw * R * slotw; i += blockDim.x) smem_u[i] = 0u;
    if (tid < 32) {  // one warp; its lanes store the same values
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
        s_nrows = nr;
    }
    __syncthreads();
    unsigned* fw = smem_u + (size_t)(warp * R + g) * slotw;
    unsigned char* fl = reinterpret_cast<unsigned char*>(fw);
    unsigned long long* err = &p.hdr->err;
    const long long* mark = p.s.flops;
    const long long end = s_nrows, step = (long long)gridDim.x * nw * R;
    const long long nnzB = p.segB.nnzB;
    for (long long idx = s_nheavy + ((long long)blockIdx.x * nw + warp) * R; idx < end; idx += step) {
        const long long my = idx + g;
        long long a0 = 0, a1 = 0;
        int row = -1;
        if (my < end) {
            row = __ldg(p.perm + my);
            a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
            a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
            if (is_split_row(mark, row, a1 - a0)) {
                a1 = a0;  // counted from its split parts
                row = -1;
            }
        }
        const int len = (int)(a1 - a0);
        const int lmax = (int)__reduce_max_sync(FULL, (unsigned)len);
        // chunks of RG entries, pipelined: while chunk e is marked, the
        // segment of chunk e + RG (B's row pointers) and the column of
        // chunk e + 2RG (A) are loaded
        auto col_at = [&](int e) { return e + gl < len ? __ldg(p.Ai + a0 + e + gl) : -1; };
        auto seg_of = [&](int k, long long& sg, int& L) {
            sg = 0;
            L = 0;
            if (k == -1) return;
            if ((unsigned)k < (unsigned)p.nB) p.segB(k, sg, L);
            else atomicOr(err, ERR_A_COL);
        };
        int k1 = col_at(RG);
        long long sg;
        int L;
        seg_of(col_at(0), sg, L);
        for (int e = 0; e < lmax; e += RG) {
            const int k2 = col_at(e + 2 * RG);
            long long nsg;
            int nL;
            seg_of(k1, nsg, nL);
            const int nu = lmax - e < RG ? lmax - e : RG;
            for (int u = 0; u < nu; u += 2) {
                const long long s0 = shfl64(sg, g * RG + u);
                const int L0 = __shfl_sync(FULL, L, g * RG + u);
                const int u1 = u + 1 < nu ? u + 1 : u;
                const long long s1 = shfl64(sg, g * RG + u1);
                const int L1 = u + 1 < nu ? __shfl_sync(FULL, L, g * RG + u1) : 0;
                const long long b0 = s0 & ~3LL, e0 = s0 + L0, b1 = s1 & ~3LL, e1 = s1 + L1;
                const int n0 = L0 > 0 ? (int)((e0 - b0 + 3) >> 2) : 0;
                const int n1 = L1 > 0 ? (int)((e1 - b1 + 3) >> 2) : 0;
                const int nm = n0 > n1 ? n0 : n1;
                for (int q = gl; q < nm; q += RG) {
                    int c0[4] = {-1, -1, -1, -1}, c1[4] = {-1, -1, -1, -1};
                    if (q < n0) symrg_quad(p.Bi, nnzB, b0 + 4LL * q, s0, e0, c0);
                    if (q < n1) symrg_quad(p.Bi, nnzB, b1 + 4LL * q, s1, e1, c1);
                    symrg_mark(fl, c0, p.d, err);
                    symrg_mark(fl, c1, p.d, err);
                }
            }
            sg = nsg;
            L = nL;
            k1 = k2;
        }
        __syncwarp();
        int c = 0;
        for (int w = 4 * gl; w < slotw; w += 4 * RG) {
            uint4* q = reinterpret_cast<uint4*>(fw + w);
            const uint4 v = *q;
            c += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
            if (v.x | v.y | v.z | v.w) *q = make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int o = RG / 2; o >= 1; o >>= 1) c += __shfl_xor_sync(FULL, c, o, RG);
        if (row >= 0 && gl == 0) p.Cp_next[row] = c;
        __syncwarp();
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

int persistent_grid(const void* kernel, int threads, size_t smem, int sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return per_sm * sms;
}

static cudaError_t set_smem(const void* kernel, size_t smem) {
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

cudaError_t launch_symbolic(const DevCsr& A, const DevCsr& B, long long d, const Sched& s,
                            const LaunchCfg& cfg, long long* Cp, cudaStream_t st) {
    cudaError_t e;
    const long long n = A.nrows;
    if ((e = cudaMemsetAsync(Cp, 0, sizeof(long long), st))) return e;
    if (n == 0) return cudaSuccess;
    if ((e = cudaMemsetAsync(&s.hdr->heavy_ctr, 0, 2 * sizeof(unsigned long long), st))) return e;
    const long long item_cap = split_item_capacity(A.nnz);
    count_launch();
    k_split_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, A.rowptr, A.nnz, s.flops, s, item_cap);
    SymParams p;
    p.Ap = A.rowptr;
    p.Ai = A.col;
    p.nnzA = A.nnz;
    p.segB = SegWhole{B.rowptr, B.nnz, (int)d};
    p.Bi = B.col;
    p.nB = (int)B.nrows;
    p.d = (int)d;
    p.dw = (int)((d + 31) / 32);
    const bool fl = d <= SYM_FLAG_MAX_D;
    p.slot = fl ? 8 * p.dw : p.dw;
    p.perm = s.perm;
    p.hdr = s.hdr;
    p.cta_class = cfg.cta_class;
    p.Cp_next = Cp + 1;
    p.s = s;
    p.item_cap = item_cap;
    p.skip_light = 0;
    p.tiny = 0;
    const int threads = 32 * cfg.warps_per_cta;
    const size_t smem = sizeof(unsigned) * (size_t)p.slot * cfg.warps_per_cta;
    const void* k;
    int group = cfg.group;
    if (group == 2 && (reinterpret_cast<uintptr_t>(B.col) & 15)) group = 16;  // quads need aligned columns
    switch (group) {
        case 1: k = fl ? (const void*)k_symbolic<1, true> : (const void*)k_symbolic<1, false>; break;
        case 2: k = fl ? (const void*)k_symbolic<2, true> : (const void*)k_symbolic<2, false>; break;
        case 4: k = fl ? (const void*)k_symbolic<4, true> : (const void*)k_symbolic<4, false>; break;
        case 8: k = fl ? (const void*)k_symbolic<8, true> : (const void*)k_symbolic<8, false>; break;
        case 16: k = fl ? (const void*)k_symbolic<16, true> : (const void*)k_symbolic<16, false>; break;
        case 32: k = fl ? (const void*)k_symbolic<32, true> : (const void*)k_symbolic<32, false>; break;
        default: return cudaErrorInvalidValue;
    }
    if (threads > 256) return cudaErrorInvalidValue;
    if ((e = set_smem(k, smem))) return e;
    // light rows in row groups of four lanes (quads; byte marks; aligned B.col;
    // d up to 512: wider rows make the per-row byte count cost more than the
    // groups save, measured at d = 1024)
    constexpr int SRG = 4;
    const bool rg = cfg.row_lanes != 32 && fl && d <= 512 && !(reinterpret_cast<uintptr_t>(B.col) & 15);
    const size_t lsmem = sizeof(unsigned) * (size_t)8 * p.dw * (32 / SRG) * cfg.warps_per_cta;
    const bool rg_ok = rg && lsmem <= 200 * 1024;
    if (rg_ok) p.skip_light = 1;
    // without the row-group kernel, tiny light rows are counted in registers
    // (one warp per light row forced: the classic walk for every row)
    if (!rg_ok && cfg.row_lanes != 32 && d > 256) {
        p.tiny = 1;
        const int tgrid = persistent_grid((const void*)k_symbolic_tiny, 256, 0, cfg.sms);
        count_launch();
        k_symbolic_tiny<<<tgrid, 256, 0, st>>>(p);
        if ((e = cudaGetLastError())) return e;
    }
    const int grid = persistent_grid(k, threads, smem, cfg.sms);
    void* args[] = {&p};
    count_launch();
    if ((e = cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, st))) return e;
    if ((e = cudaGetLastError())) return e;
    if (rg_ok) {
        const void* kl = (const void*)k_symbolic_light<SRG>;
        if ((e = set_smem(kl, lsmem))) return e;
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(persistent_grid(kl, threads, lsmem, cfg.sms));
        lc.blockDim = dim3(threads);
        lc.dynamicSmemBytes = lsmem;
        lc.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        count_launch();
        if ((e = cudaLaunchKernelEx(&lc, k_symbolic_light<SRG>, p))) return e;
    }
    return launch_scan_inplace(Cp + 1, n, s.partial, st);
}

// ---------------------------------------------------------------------------
// Inclusive scan of int64 (reduce, scan of block sums, apply).
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 512, SCAN_PER_THREAD = 8, SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;

size_t scan_partial_count(long long n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE) + 1; }

template <int THREADS>
__device__ __forceinline__ long long block_excl_scan(long long v, long long& total) {
    __shared__ long long s_w[THREADS / 32];
    __shared__ long long s_tot;
    const int lane = lane_id(), warp = warp_id();
    const long long inc = warp_incl_scan(v);
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const long long w = lane < THREADS / 32 ? s_w[lane] : 0;
        const long long wi = warp_incl_scan(w);
        if (lane < THREADS / 32) s_w[lane] = wi - w;
        if (lane == 31) s_tot = wi;
    }
    __syncthreads();
    const long long res = s_w[warp] + inc - v;
    total = s_tot;
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const long long* __restrict__ x,
                                                              long long n, long long* partial) {
    __shared__ long long s_w[SCAN_THREADS / 32];
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    long long s = 0;
#pragma unroll
    for (int u = 0; u < SCAN_PER_THREAD; ++u) {
        const long long i = base + (long long)u * SCAN_THREADS + threadIdx.x;
        if (i < n) s += x[i];
    }
    s = warp_sum(s);
    if (lane_id() == 0) s_w[warp_id()] = s;
    __syncthreads();
    if (warp_id() == 0) {
        long long v = lane_id() < SCAN_THREADS / 32 ? s_w[lane_id()] : 0;
        v = warp_sum(v);
        if (lane_id() == 0) partial[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(1024) k_scan_partials(long long* partial, long long nb) {
    long long carry = 0;
    for (long long b = 0; b < nb; b += 1024) {
        const long long i = b + threadIdx.x;
        const long long v = i < nb ? partial[i] : 0;
        long long tot;
        const long long ex = block_excl_scan<1024>(v, tot);
        if (i < nb) partial[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) partial[nb] = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(long long* x, long long n,
                                                             const long long* __restrict__ partial) {
    const long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_PER_THREAD;
    long long v[SCAN_PER_THREAD];
    long long run = 0;
#pragma unroll
    for (int u = 0; u < SCAN_PER_THREAD; ++u) {
        const long long i = base + u;
        run += (i < n) ? x[i] : 0;
        v[u] = run;
    }
    long long tot;
    const long long ex = block_excl_scan<SCAN_THREADS>(run, tot) + partial[blockIdx.x];
#pragma unroll
    for (int u = 0; u < SCAN_PER_THREAD; ++u) {
        const long long i = base + u;
        if (i < n) x[i] = ex + v[u];
    }
}

cudaError_t launch_scan_inplace(long long* x, long long n, long long* partial, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const long long nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    count_launch();
    k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(x, n, partial);
    count_launch();
    k_scan_partials<<<1, 1024, 0, st>>>(partial, nb);
    count_launch();
    k_scan_apply<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(x, n, partial);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Column tiles of B: first position of each tile boundary inside each row.
// ---------------------------------------------------------------------------
__global__ void k_tile_split(long long nB, const long long* __restrict__ Bp, const int* __restrict__ Bi,
                             long long nnzB, int W, int T, long long* __restrict__ tp) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nB * (T + 1)) return;
    const long long k = idx / (T + 1);
    const int t = (int)(idx - k * (T + 1));
    const long long s = clampll(Bp[k], 0, nnzB), e = clampll(Bp[k + 1], s, nnzB);
    long long r;
    if (t == 0) r = s;
    else if (t == T) r = e;
    else {
        const int key = t * W;
        long long lo = s, hi = e;  // first position with col >= key
        while (lo < hi) {
            const long long mid = lo + ((hi - lo) >> 1);
            if (Bi[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        r = lo;
    }
    tp[idx] = r;
}

cudaError_t launch_tile_split(const DevCsr& B, int W, int T, long long* tp, cudaStream_t st) {
    const long long tot = B.nrows * (T + 1);
    if (tot == 0) return cudaSuccess;
    count_launch();
    k_tile_split<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(B.nrows, B.rowptr, B.col, B.nnz, W, T, tp);
    return cudaGetLastError();
}

}  // namespace ts
