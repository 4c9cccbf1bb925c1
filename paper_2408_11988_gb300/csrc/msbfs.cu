// Multi-source BFS (paper Alg. 3), one level per call:
//   N = A * F over (or, select2nd);  F_next = N minus S;  S = S or N;
// fused into one gather pass per row (the boolean TS-SpGEMM with a d-bit
// accumulator), a scan for F_next's row pointers and a read-out of the new
// bits.  Rows whose visited set is already full cannot gain bits and are not
// scheduled at all; rows whose neighbours have empty frontier rows have no
// products and are skipped by the flops binning.
#include "common.cuh"
#include "kernels.h"

namespace ts {

// Rows whose visited bits are all set get flops 0 (nothing can be new).
__global__ void k_mask_full_rows(long long n, int d, int dw, const unsigned* __restrict__ S,
                                 long long* flops) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || flops[i] == 0) return;
    const unsigned* r = S + i * dw;
    for (int w = 0; w < dw; ++w) {
        const int bits = d - 32 * w;
        const unsigned want = bits >= 32 ? FULL : ((1u << bits) - 1u);
        if ((r[w] & want) != want) return;
    }
    flops[i] = 0;
}

struct OrVisit {
    const int* __restrict__ Fi;
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
        for (int u = 0; u < 4; ++u) c[u] = __ldg(Fi + j[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) mark(c[u]);
    }
    __device__ __forceinline__ void step1(long long j, float, int, bool ok) {
        if (ok) mark(__ldg(Fi + j));
    }
};

struct BfsParams {
    const long long* Ap;
    const int* Ai;
    long long nnzA;
    SegWhole segF;
    const int* Fi;
    int nF;
    int d;
    int dw;
    unsigned* S;
    int* levels;
    int level;
    unsigned* newbits;
    long long* cnt_next;  // F_next.rowptr + 1
    int* parents;         // int32[n][d] BFS-tree parents (pull form only), or nullptr
    const int* perm;
    WsHeader* hdr;
    int cta_class;
};

// Given the OR of the neighbours' frontier rows in bm (dw words), keep the
// bits not yet visited, mark them visited, record their level, store them for
// the read-out and return how many there are.  Threads t0, t0+nt, ... own words.
__device__ __forceinline__ int settle_row(const BfsParams& p, long long row, unsigned* bm, int t0, int nt) {
    int c = 0;
    for (int w = t0; w < p.dw; w += nt) {
        const int bits = p.d - 32 * w;
        const unsigned valid = bits >= 32 ? FULL : ((1u << bits) - 1u);
        const unsigned old = p.S[row * p.dw + w];
        unsigned nw = bm[w] & ~old & valid;
        bm[w] = 0u;
        p.newbits[row * p.dw + w] = nw;
        if (nw) {
            p.S[row * p.dw + w] = old | nw;
            c += __popc(nw);
            while (nw) {
                const int b = __ffs(nw) - 1;
                nw &= nw - 1;
                p.levels[row * p.d + 32 * w + b] = p.level;
            }
        }
    }
    return c;
}

__global__ void __launch_bounds__(1024) k_msbfs_expand(BfsParams p) {
    extern __shared__ __align__(16) unsigned smem_u[];
    __shared__ long long s_item, s_nheavy, s_nrows;
    __shared__ int s_red[32];
    const int nw = blockDim.x >> 5, warp = warp_id(), lane = lane_id(), tid = threadIdx.x;
    for (int i = tid; i < nw * p.dw; i += blockDim.x) smem_u[i] = 0u;
    if (tid < 32) {  // one warp; its lanes store the same values
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
        s_nrows = nr;
    }
    __syncthreads();
    const long long nheavy = s_nheavy, nrows = s_nrows;
    unsigned long long* err = &p.hdr->err;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&p.hdr->heavy_ctr, 1ull);
        __syncthreads();
        const long long h = s_item;
        __syncthreads();
        if (h >= nheavy) break;
        const int row = p.perm[h];
        const long long a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
        const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
        OrVisit vis{p.Fi, smem_u, p.d, err};
        for (long long e0 = a0 + 32LL * warp; e0 < a1; e0 += 32LL * nw)
            expand_chunk(e0, (int)(a1 - e0 < 32 ? a1 - e0 : 32), p.Ai, (const float*)nullptr, p.nF,
                         p.segF, vis, err);
        __syncthreads();
        int c = settle_row(p, row, smem_u, tid, blockDim.x);
        c = warp_sum(c);
        if (lane == 0) s_red[warp] = c;
        __syncthreads();
        if (warp == 0) {
            int v = lane < nw ? s_red[lane] : 0;
            v = warp_sum(v);
            if (lane == 0) p.cnt_next[row] = v;
        }
    }
    unsigned* bm = smem_u + warp * p.dw;
    for (long long idx = nheavy + (long long)blockIdx.x * nw + warp; idx < nrows;
         idx += (long long)gridDim.x * nw) {
        const int row = p.perm[idx];
        const long long a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
        const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
        OrVisit vis{p.Fi, bm, p.d, err};
        for (long long e0 = a0; e0 < a1; e0 += 32)
            expand_chunk(e0, (int)(a1 - e0 < 32 ? a1 - e0 : 32), p.Ai, (const float*)nullptr, p.nF,
                         p.segF, vis, err);
        __syncwarp();
        int c = settle_row(p, row, bm, lane, 32);
        c = warp_sum(c);
        if (lane == 0) p.cnt_next[row] = c;
        __syncwarp();
    }
}

// F_next columns from the stored new bits; one thread per row, rows without
// new bits (this level's count is 0) are skipped, so stale words of rows not
// scheduled this level are never read.
__global__ void k_msbfs_emit(long long n, int dw, const unsigned* __restrict__ newbits,
                             const long long* __restrict__ rp, int* __restrict__ col, long long cap,
                             unsigned long long* err) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long pos = rp[i];
    const long long end = rp[i + 1];
    if (end <= pos) return;
    for (int w = 0; w < dw; ++w) {
        unsigned word = newbits[i * dw + w];
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            if (pos < end && pos < cap) col[pos] = 32 * w + b;
            else atomicOr(err, ERR_CAPACITY);
            ++pos;
        }
    }
}

// Initial frontier and visited/level state from d sources (distinct vertices;
// a repeated vertex simply holds several columns).  Thread per vertex for the
// row pointers (counting the sources at or below it), thread per source for
// the columns.
__global__ void k_msbfs_init_rows(long long n, int d, const int* __restrict__ src, long long* rp) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v > n) return;
    if (v == 0) {
        rp[0] = 0;
        return;
    }
    long long c = 0;  // rp[v] = number of (valid) sources at vertices < v
    for (int s = 0; s < d; ++s) {
        const int u = __ldg(src + s);
        c += (u >= 0 && (long long)u < v) ? 1 : 0;
    }
    rp[v] = c;
}

__global__ void k_msbfs_init_cols(long long n, int d, int dw, const int* __restrict__ src, int* col,
                                  unsigned* S, int* levels) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d) return;
    const int v = src[s];
    if (v < 0 || (long long)v >= n) return;
    int pos = 0;
    for (int t = 0; t < d; ++t) {
        const int u = src[t];
        if (u < 0 || (long long)u >= n) continue;
        if (u < v || (u == v && t < s)) ++pos;
    }
    col[pos] = s;
    atomicOr(S + (long long)v * dw + (s >> 5), 1u << (s & 31));
    levels[(long long)v * d + s] = 0;
}


// ---------------------------------------------------------------------------
// Pull expansion with the frontier as a bitmap (the dense-frontier form of
// Alg. 3's N = A * F): F is first written as DWP words per row (d <= 256,
// DWP = dw rounded up to a power of two), then row v ORs the bitmap rows of
// its neighbours, one load of DWP words per entry of A, instead of gathering
// each neighbour's list of frontier columns.  The cost per entry no longer
// grows with the frontier's density.  The OR, the visited mask, the level
// write and the new-bit words are those of the list form.
// ---------------------------------------------------------------------------
template <int DWP>
__global__ void __launch_bounds__(256) k_frontier_bits(long long n, int d, const long long* __restrict__ Fp,
                                                       long long nnzF, const int* __restrict__ Fi,
                                                       unsigned* __restrict__ fb, unsigned long long* err) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        unsigned w[DWP];
#pragma unroll
        for (int m = 0; m < DWP; ++m) w[m] = 0u;
        const long long s = clampll(__ldg(Fp + v), 0, nnzF), e = clampll(__ldg(Fp + v + 1), s, nnzF);
        for (long long j = s; j < e; ++j) {
            const int c = __ldg(Fi + j);
            if ((unsigned)c < (unsigned)d) {
#pragma unroll
                for (int m = 0; m < DWP; ++m) w[m] |= (c >> 5) == m ? 1u << (c & 31) : 0u;
            } else {
                atomicOr(err, ERR_B_COL);
            }
        }
#pragma unroll
        for (int m = 0; m < DWP; ++m) fb[v * DWP + m] = w[m];
    }
}

// OR of the frontier bitmap rows of entries [e0, e1) of A, lane-strided.
template <int DWP>
__device__ __forceinline__ void pull_or(const BfsParams& p, const unsigned* __restrict__ fb, long long e0,
                                        long long e1, int t0, int nt, unsigned acc[DWP], unsigned long long* err) {
    // unrolled so that several neighbours' rows are in flight per thread; a
    // bad column reads row 0 and contributes nothing (keep = 0)
#pragma unroll 4
    for (long long e = e0 + t0; e < e1; e += nt) {
        int u = __ldg(p.Ai + e);
        unsigned keep = FULL;
        if ((unsigned)u >= (unsigned)p.nF) {
            atomicOr(err, ERR_A_COL);
            u = 0;
            keep = 0u;
        }
        const unsigned* r = fb + (long long)u * DWP;
        if constexpr (DWP >= 4) {
#pragma unroll
            for (int m = 0; m < DWP; m += 4) {
                const uint4 x = __ldg(reinterpret_cast<const uint4*>(r + m));
                acc[m] |= x.x & keep;
                acc[m + 1] |= x.y & keep;
                acc[m + 2] |= x.z & keep;
                acc[m + 3] |= x.w & keep;
            }
        } else {
#pragma unroll
            for (int m = 0; m < DWP; ++m) acc[m] |= __ldg(r + m) & keep;
        }
    }
}

// Settle row `row` from the OR of its neighbours (all lanes of the warp hold
// the full OR): new = N and not S; S |= new; new bits stored for the
// read-out; levels written, lane l taking bit l of every word.  Returns the
// number of new bits (all lanes).
template <int DWP>
__device__ __forceinline__ int pull_settle(const BfsParams& p, long long row, const unsigned acc[DWP],
                                           unsigned nws[DWP]) {
    const int lane = lane_id();
    int c = 0;
#pragma unroll
    for (int m = 0; m < DWP; ++m) {
        nws[m] = 0u;
        if (m >= p.dw) continue;
        const int bits = p.d - 32 * m;
        const unsigned valid = bits >= 32 ? FULL : ((1u << bits) - 1u);
        const unsigned old = __ldg(p.S + row * p.dw + m);
        const unsigned nw = acc[m] & ~old & valid;
        nws[m] = nw;
        if (lane == 0) {
            p.newbits[row * p.dw + m] = nw;
            if (nw) p.S[row * p.dw + m] = old | nw;
        }
        if ((nw >> lane) & 1u) p.levels[row * p.d + 32 * m + lane] = p.level;
        c += __popc(nw);
    }
    return c;
}

// Parents of the new bits of `row` (the (sel2nd, min) semiring of the
// BFS-tree variant: the smallest neighbour in the frontier of each source).
// A's row is ascending, so the neighbours are scanned 32 at a time in order
// and each still-open bit goes to the first lane whose frontier row holds it
// (an exclusive prefix OR over the lanes); the scan stops once every new bit
// has its parent.  One warp, all lanes converged; rem is warp-uniform.
template <int DWP>
__device__ __forceinline__ void pull_parents(const BfsParams& p, const unsigned* __restrict__ fb, long long row,
                                             long long a0, long long a1, unsigned rem[DWP]) {
    const int lane = lane_id();
    unsigned open = 0u;
#pragma unroll
    for (int m = 0; m < DWP; ++m) open |= rem[m];
    for (long long e0 = a0; e0 < a1 && open; e0 += 32) {
        const long long e = e0 + lane;
        int u = -1;
        unsigned hit[DWP];
#pragma unroll
        for (int m = 0; m < DWP; ++m) hit[m] = 0u;
        if (e < a1) {
            u = __ldg(p.Ai + e);
            if ((unsigned)u < (unsigned)p.nF) {
#pragma unroll
                for (int m = 0; m < DWP; ++m) hit[m] = __ldg(fb + (long long)u * DWP + m) & rem[m];
            }
        }
        open = 0u;
#pragma unroll
        for (int m = 0; m < DWP; ++m) {
            unsigned incl = hit[m];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl |= t;
            }
            unsigned excl = __shfl_up_sync(FULL, incl, 1);
            if (lane == 0) excl = 0u;
            unsigned mine = hit[m] & ~excl;
            while (mine) {
                const int b = __ffs(mine) - 1;
                mine &= mine - 1;
                p.parents[row * p.d + 32 * m + b] = u;
            }
            rem[m] &= ~__shfl_sync(FULL, incl, 31);
            open |= rem[m];
        }
    }
}

template <int DWP>
__global__ void __launch_bounds__(256, 6) k_msbfs_pull(BfsParams p, const unsigned* __restrict__ fb) {
    __shared__ long long s_item, s_nheavy, s_nrows;
    __shared__ unsigned s_or[DWP];
    const int nw = blockDim.x >> 5, warp = warp_id(), lane = lane_id(), tid = threadIdx.x;
    if (tid < 32) {  // one warp; its lanes store the same values
        long long nh, nr;
        sched_counts(p.hdr, p.cta_class, nh, nr);
        s_nheavy = nh;
        s_nrows = nr;
    }
    if (tid < DWP) s_or[tid] = 0u;
    __syncthreads();
    const long long nheavy = s_nheavy, nrows = s_nrows;
    unsigned long long* err = &p.hdr->err;
    // heavy rows: the block's threads split the row's entries
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&p.hdr->heavy_ctr, 1ull);
        __syncthreads();
        const long long h = s_item;
        __syncthreads();
        if (h >= nheavy) break;
        const int row = p.perm[h];
        const long long a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
        const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
        unsigned acc[DWP];
#pragma unroll
        for (int m = 0; m < DWP; ++m) acc[m] = 0u;
        pull_or<DWP>(p, fb, a0, a1, tid, blockDim.x, acc, err);
#pragma unroll
        for (int m = 0; m < DWP; ++m) {
            const unsigned x = __reduce_or_sync(FULL, acc[m]);
            if (lane == 0 && x) atomicOr(&s_or[m], x);
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int m = 0; m < DWP; ++m) acc[m] = s_or[m];
            unsigned nws[DWP];
            const int c = pull_settle<DWP>(p, row, acc, nws);
            if (lane == 0) p.cnt_next[row] = c;
            if (p.parents) pull_parents<DWP>(p, fb, row, a0, a1, nws);
        }
        __syncthreads();
        if (tid < DWP) s_or[tid] = 0u;
    }
    // light rows: one warp per row
    for (long long idx = nheavy + (long long)blockIdx.x * nw + warp; idx < nrows;
         idx += (long long)gridDim.x * nw) {
        const int row = p.perm[idx];
        const long long a0 = clampll(__ldg(p.Ap + row), 0, p.nnzA);
        const long long a1 = clampll(__ldg(p.Ap + row + 1), a0, p.nnzA);
        unsigned acc[DWP];
#pragma unroll
        for (int m = 0; m < DWP; ++m) acc[m] = 0u;
        pull_or<DWP>(p, fb, a0, a1, lane, 32, acc, err);
#pragma unroll
        for (int m = 0; m < DWP; ++m) acc[m] = __reduce_or_sync(FULL, acc[m]);
        unsigned nws[DWP];
        const int c = pull_settle<DWP>(p, row, acc, nws);
        if (lane == 0) p.cnt_next[row] = c;
        if (p.parents) pull_parents<DWP>(p, fb, row, a0, a1, nws);
    }
}

template <int DWP>
static cudaError_t launch_pull(const BfsParams& p, const DevCsr& F, unsigned* fb, const LaunchCfg& cfg,
                               cudaStream_t st) {
    const long long n = F.nrows;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    count_launch();
    k_frontier_bits<DWP><<<(unsigned)blocks, 256, 0, st>>>(n, p.d, F.rowptr, F.nnz, F.col, fb, &p.hdr->err);
    const int threads = 32 * cfg.warps_per_cta;
    const int grid = persistent_grid((const void*)k_msbfs_pull<DWP>, threads, 0, cfg.sms);
    count_launch();
    k_msbfs_pull<DWP><<<grid, threads, 0, st>>>(p, fb);
    return cudaGetLastError();
}

// Words per bitmap row of the pull form (0: list form only, d > 256).
int msbfs_pull_words(int d) {
    const int dw = (d + 31) / 32;
    if (dw > 8) return 0;
    return dw <= 1 ? 1 : (dw <= 2 ? 2 : (dw <= 4 ? 4 : 8));
}

// parents = -1, and each source its own parent in its column.
__global__ void k_msbfs_init_parents(long long n, int d, const int* __restrict__ src, int* parents) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d) return;
    const int v = src[s];
    if (v < 0 || (long long)v >= n) return;
    parents[(long long)v * d + s] = v;
}

cudaError_t launch_msbfs_init_parents(long long n, int d, const int* src, int* parents, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(parents, 0xFF, sizeof(int) * (size_t)n * d, st))) return e;
    count_launch();
    k_msbfs_init_parents<<<(d + 127) / 128, 128, 0, st>>>(n, d, src, parents);
    return cudaGetLastError();
}

cudaError_t launch_msbfs_init(long long n, int d, const int* src, unsigned* S, int* levels,
                              long long* rp, int* col, cudaStream_t st) {
    cudaError_t e;
    const int dw = (d + 31) / 32;
    if ((e = cudaMemsetAsync(S, 0, sizeof(unsigned) * (size_t)n * dw, st))) return e;
    if ((e = cudaMemsetAsync(levels, 0xFF, sizeof(int) * (size_t)n * d, st))) return e;
    count_launch();
    k_msbfs_init_rows<<<(unsigned)((n + 1 + 255) / 256), 256, 0, st>>>(n, d, src, rp);
    count_launch();
    k_msbfs_init_cols<<<(d + 127) / 128, 128, 0, st>>>(n, d, dw, src, col, S, levels);
    return cudaGetLastError();
}

cudaError_t launch_msbfs_step(const DevCsr& A, const DevCsr& F, int d, unsigned* S, int* levels, int level,
                              const Sched& s, unsigned* newbits, long long* rp_next, const LaunchCfg& cfg,
                              cudaStream_t st, unsigned* fbits, int* parents) {
    cudaError_t e;
    const long long n = A.nrows;
    if ((e = launch_row_flops(A, F, s, st))) return e;
    if (n == 0) return cudaMemsetAsync(rp_next, 0, sizeof(long long), st);
    const int dw = (d + 31) / 32;
    // prune rows that cannot gain bits, then histogram and order (rows left
    // without products get their count 0 here)
    count_launch();
    k_mask_full_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, d, dw, S, s.flops);
    if ((e = launch_reclassify(n, s, rp_next + 1, st))) return e;
    if ((e = cudaMemsetAsync(rp_next, 0, sizeof(long long), st))) return e;
    BfsParams p;
    p.Ap = A.rowptr;
    p.Ai = A.col;
    p.nnzA = A.nnz;
    p.segF = SegWhole{F.rowptr, F.nnz, d};
    p.Fi = F.col;
    p.nF = (int)F.nrows;
    p.d = d;
    p.dw = dw;
    p.S = S;
    p.levels = levels;
    p.level = level;
    p.newbits = newbits;
    p.cnt_next = rp_next + 1;
    p.parents = parents;
    p.perm = s.perm;
    p.hdr = s.hdr;
    p.cta_class = cfg.cta_class;
    const int dwp = msbfs_pull_words(d);
    if (parents && !(fbits && dwp)) return cudaErrorInvalidValue;  // parents: pull form only
    if (fbits && dwp) {
        switch (dwp) {
            case 1: e = launch_pull<1>(p, F, fbits, cfg, st); break;
            case 2: e = launch_pull<2>(p, F, fbits, cfg, st); break;
            case 4: e = launch_pull<4>(p, F, fbits, cfg, st); break;
            default: e = launch_pull<8>(p, F, fbits, cfg, st); break;
        }
        if (e) return e;
        return launch_scan_inplace(rp_next + 1, n, s.partial, st);
    }
    const int threads = 32 * cfg.warps_per_cta;
    const size_t smem = sizeof(unsigned) * (size_t)dw * cfg.warps_per_cta;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute((const void*)k_msbfs_expand, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
        return e;
    const int grid = persistent_grid((const void*)k_msbfs_expand, threads, smem, cfg.sms);
    count_launch();
    k_msbfs_expand<<<grid, threads, smem, st>>>(p);
    if ((e = cudaGetLastError())) return e;
    return launch_scan_inplace(rp_next + 1, n, s.partial, st);
}

cudaError_t launch_msbfs_emit(long long n, int d, const unsigned* newbits, const long long* rp, int* col,
                              long long cap, WsHeader* hdr, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    count_launch();
    k_msbfs_emit<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, (d + 31) / 32, newbits, rp, col, cap,
                                                                &hdr->err);
    return cudaGetLastError();
}

}  // namespace ts
