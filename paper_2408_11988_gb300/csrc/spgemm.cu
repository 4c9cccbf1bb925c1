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
// flops = number of multiplications).  Entry parallel: every warp takes a
// fixed slice of A's entries, so rows with very many entries are spread over
// many warps.  Partial row sums are added with atomics into a zeroed array.
// ---------------------------------------------------------------------------
constexpr int FLOPS_CHUNK = 256;  // entries of A per warp

__global__ void __launch_bounds__(256) k_flops_entries(long long n, const long long* __restrict__ Ap,
                                                       const int* __restrict__ Ai, long long nnzA,
                                                       SegWhole segB, int nB,
                                                       long long* __restrict__ flops,
                                                       WsHeader* hdr) {
    __shared__ unsigned long long s_sum[8][32];
    const int warp = warp_id(), lane = lane_id();
    const long long E0 = ((long long)blockIdx.x * 8 + warp) * FLOPS_CHUNK;
    if (E0 >= nnzA || n <= 0) return;
    const long long E1 = E0 + FLOPS_CHUNK < nnzA ? E0 + FLOPS_CHUNK : nnzA;

    // r = the row holding entry E0: the largest r in [0, n) with Ap[r] <= E0,
    // found by a 32-way search (the answer stays in [lo, hi)).
    auto find_row = [&](long long lo, long long hi, long long e) {
        while (hi - lo > 1) {
            const long long step = (hi - lo + 31) / 32;
            const long long cand = lo + (long long)lane * step;
            const bool le = cand < hi && __ldg(Ap + cand) <= e;
            const unsigned m = __ballot_sync(FULL, le) | 1u;
            const int q = 31 - __clz(m);
            lo = lo + (long long)q * step;
            const long long nh = lo + step;
            hi = nh < hi ? nh : hi;
        }
        return lo;
    };
    long long r = find_row(0, n, E0);
    long long e = E0;
    unsigned long long* err = &hdr->err;
    // every pass either consumes an entry or re-locates r once, so a well
    // formed A needs at most 2*FLOPS_CHUNK passes; the guard only ends the
    // loop on a row pointer array that is not monotone
    for (int guard = 0; e < E1; ++guard) {
        if (guard > 4 * FLOPS_CHUNK) {
            if (lane == 0) atomicOr(err, ERR_A_COL);
            break;
        }
        // skip a window of rows that ends before e (only with long empty runs)
        const long long nxt = (r + 32 <= n) ? __ldg(Ap + r + 32) : LLONG_MAX;
        if (nxt <= e) {
            r = find_row(r, n, e);
            continue;
        }
        const long long rr = r + lane;
        const long long st = rr < n ? __ldg(Ap + rr) : LLONG_MAX;
        s_sum[warp][lane] = 0;
        __syncwarp();
        const long long stop = nxt < E1 ? nxt : E1;
        for (long long base = e; base < stop; base += 32) {
            const long long ee = base + lane;
            const int q = owner_lane64(st, ee);
            if (ee < stop) {
                const int k = __ldg(Ai + ee);
                if ((unsigned)k < (unsigned)nB) {
                    long long s0;
                    int len;
                    segB(k, s0, len);
                    if (len) atomicAdd(&s_sum[warp][q], (unsigned long long)len);
                } else {
                    atomicOr(err, ERR_A_COL);
                }
            }
        }
        __syncwarp();
        const unsigned long long v = s_sum[warp][lane];
        if (v && rr < n) atomicAdd((unsigned long long*)(flops + rr), v);
        __syncwarp();
        e = stop;
        r += 32;
    }
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
    if (tid == 0) {
        long long run = 0;
        for (int c = NUM_CLASSES - 1; c >= 1; --c) {
            s_start[c] = run;
            run += hdr->hist[c];
        }
        s_start[0] = run;
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
    if ((e = cudaMemsetAsync(s.flops, 0, sizeof(long long) * n, st))) return e;
    if (A.nnz > 0) {
        const SegWhole segB{B.rowptr, B.nnz, (int)B.ncols};
        const long long warps = (A.nnz + FLOPS_CHUNK - 1) / FLOPS_CHUNK;
        const long long blocks = (warps + 7) / 8;
        count_launch();
        k_flops_entries<<<(unsigned)blocks, 256, 0, st>>>(n, A.rowptr, A.col, A.nnz, segB,
                                                          (int)B.nrows, s.flops, s.hdr);
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
// Symbolic pass: nnz(C_i) = number of distinct columns over the rows B_k,
// k in A_i (Eq. 1 on patterns).  A bitmap of d bits per warp (shared by the
// whole block for heavy rows) collects the columns; popcounts give the count.
// ---------------------------------------------------------------------------
struct SymVisit {
    const int* __restrict__ Bi;
    unsigned* bm;
    int d;
    unsigned long long* err;
    __device__ __forceinline__ void mark(int c) {
        if ((unsigned)c < (unsigned)d) atomicOr(bm + (c >> 5), 1u << (c & 31));
        else atomicOr(err, ERR_B_COL);
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
};

struct SymParams {
    const long long* Ap;
    const int* Ai;
    long long nnzA;
    SegWhole segB;
    const int* Bi;
    int nB;
    int d;
    int dw;  // bitmap words per row
    const int* perm;
    WsHeader* hdr;
    int cta_class;
    long long* Cp_next;
};

// Rows with products: all classes >= 1; heavy: classes >= cta_class.
__device__ __forceinline__ void sched_counts(const WsHeader* hdr, int cta_class, long long& nheavy,
                                             long long& nrows) {
    long long nh = 0, nr = 0;
    for (int c = 1; c < NUM_CLASSES; ++c) {
        const long long h = hdr->hist[c];
        nr += h;
        if (c >= cta_class) nh += h;
    }
    nheavy = nh;
    nrows = nr;
}

__global__ void __launch_bounds__(1024) k_symbolic(SymParams p) {
    extern __shared__ __align__(16) unsigned smem_u[];
    __shared__ long long s_item, s_nheavy, s_nrows;
    __shared__ int s_red[32];
    const int nw = blockDim.x >> 5, warp = warp_id(), lane = lane_id(), tid = threadIdx.x;
    for (int i = tid; i < nw * p.dw; i += blockDim.x) smem_u[i] = 0;
    if (tid == 0) {
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
        s_nrows = nr;
    }
    __syncthreads();
    const long long nheavy = s_nheavy, nrows = s_nrows;
    unsigned long long* err = &p.hdr->err;

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
        SymVisit vis{p.Bi, smem_u, p.d, err};
        for (long long e0 = a0 + 32LL * warp; e0 < a1; e0 += 32LL * nw)
            expand_chunk(e0, (int)(a1 - e0 < 32 ? a1 - e0 : 32), p.Ai, (const float*)nullptr, p.nB,
                         p.segB, vis, err);
        __syncthreads();
        int c = 0;
        for (int w = tid; w < p.dw; w += blockDim.x) {
            c += __popc(smem_u[w]);
            smem_u[w] = 0;
        }
        c = warp_sum(c);
        if (lane == 0) s_red[warp] = c;
        __syncthreads();
        if (warp == 0) {
            int v = lane < nw ? s_red[lane] : 0;
            v = warp_sum(v);
            if (lane == 0) p.Cp_next[row] = v;
        }
    }

    // light rows: one warp per row, static round robin over the class order
    unsigned* bm = smem_u + warp * p.dw;
    for (long long idx = nheavy + (long long)blockIdx.x * nw + warp; idx < nrows;
         idx += (long long)gridDim.x * nw) {
        const int row = p.perm[idx];
        const long long a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
        const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
        SymVisit vis{p.Bi, bm, p.d, err};
        for (long long e0 = a0; e0 < a1; e0 += 32)
            expand_chunk(e0, (int)(a1 - e0 < 32 ? a1 - e0 : 32), p.Ai, (const float*)nullptr, p.nB,
                         p.segB, vis, err);
        __syncwarp();
        int c = 0;
        for (int w = lane; w < p.dw; w += 32) {
            c += __popc(bm[w]);
            bm[w] = 0;
        }
        c = warp_sum(c);
        if (lane == 0) p.Cp_next[row] = c;
        __syncwarp();
    }
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
    if ((e = cudaMemsetAsync(&s.hdr->heavy_ctr, 0, sizeof(unsigned long long), st))) return e;
    SymParams p;
    p.Ap = A.rowptr;
    p.Ai = A.col;
    p.nnzA = A.nnz;
    p.segB = SegWhole{B.rowptr, B.nnz, (int)d};
    p.Bi = B.col;
    p.nB = (int)B.nrows;
    p.d = (int)d;
    p.dw = (int)((d + 31) / 32);
    p.perm = s.perm;
    p.hdr = s.hdr;
    p.cta_class = cfg.cta_class;
    p.Cp_next = Cp + 1;
    const int threads = 32 * cfg.warps_per_cta;
    const size_t smem = sizeof(unsigned) * (size_t)p.dw * cfg.warps_per_cta;
    if ((e = set_smem((const void*)k_symbolic, smem))) return e;
    const int grid = persistent_grid((const void*)k_symbolic, threads, smem, cfg.sms);
    count_launch();
    k_symbolic<<<grid, threads, smem, st>>>(p);
    if ((e = cudaGetLastError())) return e;
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

// ---------------------------------------------------------------------------
// Numeric pass, dense accumulator (the paper's SPA, Sec. III-C) of width W in
// shared memory plus one occupancy byte per column.  Row i of C is produced
// tile by tile (W columns each); inside a tile the occupied columns are read
// out in ascending order by ballot/popc over the flags, which also restores
// the accumulator to zero for the next row.
// ---------------------------------------------------------------------------
constexpr int MAX_DENSE_W = 4096;

template <bool VALUES>
struct NumVisit {
    const int* __restrict__ Bi;
    const float* __restrict__ Bx;
    float* acc;
    unsigned char* flg;
    int d;
    int c0;
    int W;
    unsigned long long* err;
    __device__ __forceinline__ void apply(int c, float v) {
        const int lc = c - c0;
        if ((unsigned)c < (unsigned)d && (unsigned)lc < (unsigned)W) {
            flg[lc] = 1;
            if (VALUES) atomicAdd(acc + lc, v);
        } else {
            atomicOr(err, ERR_B_COL);
        }
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
        for (int u = 0; u < 4; ++u) apply(c[u], a[u] * b[u]);
    }
    __device__ __forceinline__ void step1(long long j, float a, int, bool ok) {
        if (ok) {
            const int c = __ldg(Bi + j);
            const float b = VALUES ? __ldg(Bx + j) : 0.0f;
            apply(c, a * b);
        }
    }
};

struct NumParams {
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
};

template <bool VALUES>
__device__ __forceinline__ void warp_emit(float* acc, unsigned char* flg, int W, int c0, long long& out,
                                          long long out_end, int* Ci, float* Cx,
                                          unsigned long long* err) {
    const int lane = lane_id();
    const unsigned lt = lanemask_lt();
    for (int w0 = 0; w0 < W; w0 += 32) {
        const int c = w0 + lane;
        const bool f = flg[c] != 0;
        const unsigned bal = __ballot_sync(FULL, f);
        if (f) {
            const long long pos = out + __popc(bal & lt);
            if (pos < out_end) {
                Ci[pos] = c0 + c;
                if (VALUES) Cx[pos] = acc[c];
            } else {
                atomicOr(err, ERR_C_ROW);
            }
            flg[c] = 0;
            if (VALUES) acc[c] = 0.0f;
        }
        out += __popc(bal);
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

template <bool VALUES, bool CTA>
__device__ __forceinline__ void numeric_row(const NumParams& p, int row, float* acc, unsigned char* flg,
                                            int* wcnt) {
    unsigned long long* err = &p.hdr->err;
    const long long a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
    const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
    long long out = clampll(__ldg(p.Cp + row), 0, p.nnzC);
    const long long out_end = clampll(__ldg(p.Cp + row + 1), out, p.nnzC);
    const int nw = blockDim.x >> 5;
    const long long first = CTA ? a0 + 32LL * warp_id() : a0;
    const long long stride = CTA ? 32LL * nw : 32LL;
    const float* Ax = VALUES ? p.Ax : nullptr;
    for (int t = 0; t < p.T; ++t) {
        NumVisit<VALUES> vis{p.Bi, p.Bx, acc, flg, p.d, t * p.W, p.W, err};
        if (p.T == 1) {
            const SegWhole seg{p.Bp, p.nnzB, p.d};
            for (long long e0 = first; e0 < a1; e0 += stride)
                expand_chunk(e0, (int)(a1 - e0 < 32 ? a1 - e0 : 32), p.Ai, Ax, p.nB, seg, vis, err);
        } else {
            const SegTile seg{p.tp, p.T + 1, t, p.W};
            for (long long e0 = first; e0 < a1; e0 += stride)
                expand_chunk(e0, (int)(a1 - e0 < 32 ? a1 - e0 : 32), p.Ai, Ax, p.nB, seg, vis, err);
        }
        if (CTA) {
            __syncthreads();
            cta_emit<VALUES>(acc, flg, p.W, t * p.W, out, out_end, p.Ci, p.Cx, wcnt, err);
        } else {
            __syncwarp();
            warp_emit<VALUES>(acc, flg, p.W, t * p.W, out, out_end, p.Ci, p.Cx, err);
            __syncwarp();
        }
    }
    if (out != out_end && (CTA ? threadIdx.x == 0 : lane_id() == 0)) atomicOr(err, ERR_C_ROW);
}

template <bool VALUES>
__global__ void __launch_bounds__(1024) k_numeric_dense(NumParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_wcnt[MAX_DENSE_W / 32 + 1];
    __shared__ long long s_item, s_nheavy, s_nrows;
    const int nw = blockDim.x >> 5, warp = warp_id(), tid = threadIdx.x;
    const int slot = VALUES ? 5 * p.W : p.W;  // bytes per warp: W floats + W flags
    for (int i = tid; i < nw * slot / 4; i += blockDim.x) ((unsigned*)smem)[i] = 0;
    if (tid == 0) {
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
        s_nrows = nr;
    }
    __syncthreads();
    const long long nheavy = s_nheavy, nrows = s_nrows;
    {
        float* acc = (float*)smem;
        unsigned char* flg = smem + (VALUES ? 4 * p.W : 0);
        for (;;) {
            if (tid == 0) s_item = (long long)atomicAdd(&p.hdr->heavy_ctr, 1ull);
            __syncthreads();
            const long long h = s_item;
            __syncthreads();
            if (h >= nheavy) break;
            numeric_row<VALUES, true>(p, p.perm[h], acc, flg, s_wcnt);
        }
    }
    float* acc = (float*)(smem + (size_t)warp * slot);
    unsigned char* flg = smem + (size_t)warp * slot + (VALUES ? 4 * p.W : 0);
    for (long long idx = nheavy + (long long)blockIdx.x * nw + warp; idx < nrows;
         idx += (long long)gridDim.x * nw)
        numeric_row<VALUES, false>(p, p.perm[idx], acc, flg, nullptr);
}

size_t numeric_dense_smem(int W, int warps, bool values) {
    return (size_t)warps * (values ? 5 * (size_t)W : (size_t)W);
}

cudaError_t launch_numeric_dense(const DevCsr& A, const DevCsr& B, long long d, int W, int T,
                                 const long long* tp, bool values, const Sched& s,
                                 const LaunchCfg& cfg, const long long* Cp, int* Ci, float* Cx,
                                 long long nnzC, cudaStream_t st) {
    cudaError_t e;
    if (A.nrows == 0) return cudaSuccess;
    if (W <= 0 || W % 32 || W > MAX_DENSE_W || (long long)W * T < d) return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(&s.hdr->heavy_ctr, 0, sizeof(unsigned long long), st))) return e;
    NumParams p;
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
    const int threads = 32 * cfg.warps_per_cta;
    const size_t smem = numeric_dense_smem(W, cfg.warps_per_cta, values);
    const void* k = values ? (const void*)k_numeric_dense<true> : (const void*)k_numeric_dense<false>;
    if ((e = set_smem(k, smem))) return e;
    const int grid = persistent_grid(k, threads, smem, cfg.sms);
    if (values) {
        count_launch();
        k_numeric_dense<true><<<grid, threads, smem, st>>>(p);
    }
    else {
        count_launch();
        k_numeric_dense<false><<<grid, threads, smem, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace ts
