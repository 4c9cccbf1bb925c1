// Deterministic dB (option T): dB(k, j) = sum over the rows i with A(i, k)
// stored of A(i, k) * dC(i, j), for (k, j) on B's pattern, summed in
// ascending i (no float atomics, so dB is the same bit for bit on every
// run).  dA still comes from the backward kernels (they skip dB).
//
// 1. The transpose of A's pattern: the entry indices of A sorted by column,
//    stably (a least-significant-digit radix sort, eight bits per pass, of
//    the column indices with the entry index as payload, so that each
//    column's entries stay in ascending row order), and its column pointers
//    (a count per column and a scan).  row_of[e] is the row of entry e.
// 2. The pull: row k of dB is column k of A's entries against rows of dC.
//    Its entries of A are cut into chunks of at most TCH (a fixed cut, so
//    the order of the sums does not depend on scheduling); a warp takes a
//    chunk, a lane holds one entry of B's row k (column j) and, for the
//    chunk's entries (i, k), finds j in row i of C (rows of C are sorted and
//    hold every column of B's row k) by binary search and adds
//    A(i, k) * dC(i, j), in an order fixed by the chunk alone (see k_t_pull).
//    The chunk's sums go to a buffer.
// 3. The chunks of row k are added in order into dB(k, :).
#include <algorithm>
#include <utility>

#include "common.cuh"
#include "kernels.h"

namespace ts {

constexpr int RS_THREADS = 256, RS_ROUNDS = 8, RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int TCH = 512;  // entries of A per chunk of a column

// row_of[e] = row of entry e (a warp per row)
__global__ void __launch_bounds__(256) k_row_of(long long n, const long long* __restrict__ Ap, long long nnzA,
                                                int* __restrict__ row_of) {
    const int lane = lane_id();
    for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n;
         i += ((long long)gridDim.x * blockDim.x) >> 5) {
        const long long a0 = clampll(Ap[i], 0, nnzA), a1 = clampll(Ap[i + 1], a0, nnzA);
        for (long long e = a0 + lane; e < a1; e += 32) row_of[e] = (int)i;
    }
}

// Per tile of RS_TILE keys, the count of each digit: cnt[digit * nb + tile].
__global__ void __launch_bounds__(RS_THREADS) k_rs_count(const int* __restrict__ key, long long m, int shift,
                                                         long long* __restrict__ cnt, long long nb) {
    __shared__ int s_c[256];
    s_c[threadIdx.x] = 0;
    __syncthreads();
    const long long t0 = (long long)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const long long x = t0 + r * RS_THREADS + threadIdx.x;
        if (x < m) atomicAdd(&s_c[((unsigned)key[x] >> shift) & 255u], 1);
    }
    __syncthreads();
    cnt[(long long)threadIdx.x * nb + blockIdx.x] = s_c[threadIdx.x];
}

// Stable scatter of one tile: keys of a digit keep their order, after every
// key of a smaller digit and every key of that digit in earlier tiles
// (incl = inclusive scan of cnt in digit-major order).
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const int* __restrict__ kin, const int* __restrict__ vin,
                                                           int* __restrict__ kout, int* __restrict__ vout, long long m,
                                                           int shift, const long long* __restrict__ incl,
                                                           long long nb) {
    __shared__ int s_tile[256];
    __shared__ long long s_base[256];
    __shared__ int s_run[256];
    __shared__ int s_w[RS_THREADS / 32][256];
    const int tid = threadIdx.x, warp = warp_id(), lane = lane_id();
    const long long t0 = (long long)blockIdx.x * RS_TILE;
    s_tile[tid] = 0;
    s_run[tid] = 0;
    __syncthreads();
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const long long x = t0 + r * RS_THREADS + tid;
        if (x < m) atomicAdd(&s_tile[((unsigned)kin[x] >> shift) & 255u], 1);
    }
    __syncthreads();
    s_base[tid] = incl[(long long)tid * nb + blockIdx.x] - s_tile[tid];
    const unsigned lt = lanemask_lt();
    for (int r = 0; r < RS_ROUNDS; ++r) {
        for (int w = 0; w < RS_THREADS / 32; ++w) s_w[w][tid] = 0;
        __syncthreads();
        const long long x = t0 + r * RS_THREADS + tid;
        const bool ok = x < m;
        const int k = ok ? kin[x] : 0;
        const int dg = ok ? (int)(((unsigned)k >> shift) & 255u) : -1;
        const unsigned mm = __match_any_sync(FULL, dg);
        const int rank = __popc(mm & lt);
        if (ok && rank == 0) s_w[warp][dg] = __popc(mm);
        __syncthreads();
        if (ok) {
            int before = 0;
            for (int w = 0; w < warp; ++w) before += s_w[w][dg];
            const long long pos = s_base[dg] + s_run[dg] + before + rank;
            kout[pos] = k;
            vout[pos] = vin[x];
        }
        __syncthreads();
        int add = 0;
        for (int w = 0; w < RS_THREADS / 32; ++w) add += s_w[w][tid];
        s_run[tid] += add;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_iota(long long m, int* __restrict__ v) {
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < m; x += (long long)gridDim.x * blockDim.x)
        v[x] = (int)x;
}

// cnt[k + 1] = entries of A in column k; cnt[0] = 0 (then scanned: column
// pointers of the transpose).  Column indices outside [0, n) were reported
// by the forward; they are skipped here.
__global__ void __launch_bounds__(256) k_col_count(const int* __restrict__ Ai, long long m, long long n,
                                                   long long* __restrict__ cnt) {
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < m; x += (long long)gridDim.x * blockDim.x) {
        const int k = Ai[x];
        if ((unsigned)k < (unsigned)n) atomicAdd((unsigned long long*)&cnt[k + 1], 1ull);
    }
}

// Chunks of column k: ceil(|A(:, k)| / TCH) (at least one when B's row k has
// entries) and, for the partial sums, chunks * |B(k, :)| floats.
__global__ void __launch_bounds__(256) k_t_chunks(long long n, const long long* __restrict__ ATp,
                                                  const long long* __restrict__ Bp, long long nnzB,
                                                  long long* __restrict__ nch, long long* __restrict__ psz) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const long long c = ATp[k + 1] - ATp[k];
        const long long s = clampll(Bp[k], 0, nnzB), e = clampll(Bp[k + 1], s, nnzB);
        const long long q = e > s ? (c + TCH - 1) / TCH : 0;
        nch[k + 1] = q;
        psz[k + 1] = q * (e - s);
    }
}

// The sorted entries' rows and values, gathered once: ti[q], ta[q].
__global__ void __launch_bounds__(256) k_t_gather(long long m, const int* __restrict__ tperm,
                                                  const int* __restrict__ row_of, const float* __restrict__ Ax,
                                                  int* __restrict__ ti, float* __restrict__ ta) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (long long)gridDim.x * blockDim.x) {
        const int e = tperm[q];
        ti[q] = row_of[e];
        ta[q] = Ax[e];
    }
}

// The pull: warp per chunk; chunk c of the whole numbering belongs to
// column col_of[c].  With at
// most 16 entries in B's row k the warp's halves take alternate groups of
// four entries of A (lane l: entry l % 16 of B's row, half l / 16), else
// lane l takes entries l, l + 32, ... of B's row; each lane keeps four
// entries of A in flight and adds their terms in a fixed order, and the two
// halves are added last, so the sums are the same on every run.
__global__ void __launch_bounds__(256) k_t_pull(long long n, const long long* __restrict__ ATp,
                                                const int* __restrict__ ti, const float* __restrict__ ta,
                                                const long long* __restrict__ Bp,
                                                const int* __restrict__ Bi, long long nnzB,
                                                const long long* __restrict__ Cp, const int* __restrict__ Ci,
                                                const float* __restrict__ dC, long long nnzC,
                                                const long long* __restrict__ chbase, const int* __restrict__ col_of,
                                                const long long* __restrict__ pbase, float* __restrict__ part,
                                                WsHeader* hdr) {
    const int lane = lane_id();
    const long long nchunks = chbase[n];
    bool bad = false;
    for (long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks;
         c += ((long long)gridDim.x * blockDim.x) >> 5) {
        const long long k = __ldg(col_of + c), ci = c - __ldg(chbase + k);
        const long long bs = clampll(__ldg(Bp + k), 0, nnzB), be = clampll(__ldg(Bp + k + 1), bs, nnzB);
        const int L = (int)(be - bs);
        const long long q0 = __ldg(ATp + k) + ci * TCH;
        const long long q1 = min(q0 + TCH, __ldg(ATp + k + 1));
        float* out = part + __ldg(pbase + k) + ci * L;
        const bool halves = L <= 16;
        const int width = halves ? 16 : 32, half = halves ? lane >> 4 : 0;
        for (int jb = 0; jb < L; jb += width) {
            const int jl = jb + (halves ? (lane & 15) : lane);
            const bool on = jl < L;
            const int j = on ? __ldg(Bi + bs + jl) : -1;
            float acc = 0.0f;
            // groups of four entries of A: half h takes groups h, h + 2, ...
            const long long step = halves ? 8 : 4;
            for (long long q = q0 + 4 * half; q < q1; q += step) {
                int iv[4];
                float av[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    iv[u] = q + u < q1 ? __ldg(ti + q + u) : -1;
                    av[u] = q + u < q1 ? __ldg(ta + q + u) : 0.0f;
                }
                // four binary searches advanced together (one load of each per step)
                long long lo4[4], len4[4], end4[4];
                int steps = 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    lo4[u] = 0;
                    len4[u] = 0;
                    end4[u] = 0;
                    if (iv[u] >= 0) {
                        lo4[u] = clampll(__ldg(Cp + iv[u]), 0, nnzC);
                        end4[u] = clampll(__ldg(Cp + iv[u] + 1), lo4[u], nnzC);
                        len4[u] = end4[u] - lo4[u];
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    int b = 0;
                    while ((1LL << b) <= len4[u]) ++b;
                    steps = steps > b ? steps : b;
                }
                for (int t = 0; t < steps; ++t) {
                    int cv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) cv[u] = len4[u] > 0 ? __ldg(Ci + lo4[u] + (len4[u] >> 1)) : 0;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (len4[u] > 0) {
                            const long long h = len4[u] >> 1;
                            if (cv[u] < j) {
                                lo4[u] += h + 1;
                                len4[u] -= h + 1;
                            } else {
                                len4[u] = h;
                            }
                        }
                    }
                }
                long long pos[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    pos[u] = (on && iv[u] >= 0 && lo4[u] < end4[u] && __ldg(Ci + lo4[u]) == j) ? lo4[u] : -1;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (on && iv[u] >= 0) {
                        if (pos[u] >= 0) acc = fmaf(av[u], __ldg(dC + pos[u]), acc);
                        else bad = true;
                    }
                }
            }
            if (halves) acc += __shfl_down_sync(FULL, acc, 16);  // half 0 + half 1, always in this order
            if (on && half == 0) out[jl] = acc;
        }
    }
    if (bad) atomicOr(&hdr->err, ERR_C_ROW);
}

// col_of[c] = the column of chunk c (a thread per column).
__global__ void __launch_bounds__(256) k_t_colmap(long long n, const long long* __restrict__ chbase,
                                                  int* __restrict__ col_of) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        for (long long c = chbase[k]; c < chbase[k + 1]; ++c) col_of[c] = (int)k;
}

// dB(k, j) = the chunks of row k added in order.
__global__ void __launch_bounds__(256) k_t_sum(long long n, const long long* __restrict__ Bp, long long nnzB,
                                               const long long* __restrict__ chbase,
                                               const long long* __restrict__ pbase, const float* __restrict__ part,
                                               float* __restrict__ dB) {
    const int lane = lane_id();
    for (long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n;
         k += ((long long)gridDim.x * blockDim.x) >> 5) {
        const long long bs = clampll(Bp[k], 0, nnzB), be = clampll(Bp[k + 1], bs, nnzB);
        const int L = (int)(be - bs);
        const long long nc = chbase[k + 1] - chbase[k];
        const float* p = part + pbase[k];
        for (int j = lane; j < L; j += 32) {
            float s = 0.0f;
            for (long long c = 0; c < nc; ++c) s += p[c * L + j];
            dB[bs + j] = s;
        }
    }
}

size_t backward_t_bytes(long long n, long long nnzA, long long nnzB, long long d) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const long long nb = (nnzA + RS_TILE - 1) / RS_TILE;
    const long long hist = 256 * nb;
    size_t s = 0;
    s += al(sizeof(int) * (size_t)nnzA) * 5;                 // row_of, keys x2, vals x2
    s += al(sizeof(long long) * (size_t)(hist + 1));          // radix counts
    s += al(sizeof(long long) * (size_t)((hist + 4095) / 4096 + 2));  // scan partials
    s += al(sizeof(long long) * (size_t)(n + 1)) * 3;         // ATp, chbase, pbase
    s += al(sizeof(long long) * (size_t)((n + 1 + 4095) / 4096 + 2));
    // partial sums: every row of B once plus one more row per full chunk
    s += al(sizeof(float) * (size_t)(nnzB + (long long)d * (nnzA / TCH + 1)));
    return s;
}

cudaError_t launch_backward_t(const DevCsr& A, const DevCsr& B, long long d, const long long* Cp, const int* Ci,
                              long long nnzC, const float* dC, float* dB, void* ws, WsHeader* hdr, cudaStream_t st) {
    cudaError_t e;
    const long long n = A.nrows, m = A.nnz;
    if (!dB || B.nnz == 0) return cudaSuccess;
    if (m == 0) return cudaMemsetAsync(dB, 0, sizeof(float) * B.nnz, st);
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    char* w = (char*)ws;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = w + off;
        off += al(bytes);
        return p;
    };
    const long long nb = (m + RS_TILE - 1) / RS_TILE;
    const long long hist = 256 * nb;
    int* row_of = (int*)take(sizeof(int) * m);
    int* k0 = (int*)take(sizeof(int) * m);
    int* k1 = (int*)take(sizeof(int) * m);
    int* v0 = (int*)take(sizeof(int) * m);
    int* v1 = (int*)take(sizeof(int) * m);
    long long* cnt = (long long*)take(sizeof(long long) * (hist + 1));
    long long* spart = (long long*)take(sizeof(long long) * ((hist + 4095) / 4096 + 2));
    long long* ATp = (long long*)take(sizeof(long long) * (n + 1));
    long long* chbase = (long long*)take(sizeof(long long) * (n + 1));
    long long* pbase = (long long*)take(sizeof(long long) * (n + 1));
    long long* spart2 = (long long*)take(sizeof(long long) * ((n + 1 + 4095) / 4096 + 2));
    float* part = (float*)take(sizeof(float) * (B.nnz + d * (m / TCH + 1)));
    const unsigned g256 = (unsigned)std::min<long long>((m + 255) / 256, 152LL * 16);
    const unsigned gw = (unsigned)std::min<long long>((n * 32 + 255) / 256, 152LL * 16);
    // rows of the entries; keys = columns of A, values = entry indices
    count_launch();
    k_row_of<<<gw, 256, 0, st>>>(n, A.rowptr, m, row_of);
    if ((e = cudaMemcpyAsync(k0, A.col, sizeof(int) * m, cudaMemcpyDeviceToDevice, st))) return e;
    count_launch();
    k_iota<<<g256, 256, 0, st>>>(m, v0);
    int bits = 1;
    while ((1LL << bits) < n) ++bits;
    int *kin = k0, *vin = v0, *kout = k1, *vout = v1;
    for (int shift = 0; shift < bits; shift += 8) {
        count_launch();
        k_rs_count<<<(unsigned)nb, RS_THREADS, 0, st>>>(kin, m, shift, cnt, nb);
        if ((e = launch_scan_inplace(cnt, hist, spart, st))) return e;
        count_launch();
        k_rs_scatter<<<(unsigned)nb, RS_THREADS, 0, st>>>(kin, vin, kout, vout, m, shift, cnt, nb);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    // vin: entry indices sorted by column (stable); column pointers
    if ((e = cudaMemsetAsync(ATp, 0, sizeof(long long) * (n + 1), st))) return e;
    count_launch();
    k_col_count<<<g256, 256, 0, st>>>(A.col, m, n, ATp);
    if ((e = launch_scan_inplace(ATp + 1, n, spart2, st))) return e;
    // chunks per column and partial-sum offsets
    if ((e = cudaMemsetAsync(chbase, 0, sizeof(long long), st))) return e;
    if ((e = cudaMemsetAsync(pbase, 0, sizeof(long long), st))) return e;
    const unsigned gn = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16);
    count_launch();
    k_t_chunks<<<gn, 256, 0, st>>>(n, ATp, B.rowptr, B.nnz, chbase, pbase);
    if ((e = launch_scan_inplace(chbase + 1, n, spart2, st))) return e;
    if ((e = launch_scan_inplace(pbase + 1, n, spart2, st))) return e;
    // rows and values of the sorted entries (into the free sort buffers)
    int* ti = kout;
    float* ta = reinterpret_cast<float*>(vout);
    count_launch();
    k_t_gather<<<g256, 256, 0, st>>>(m, vin, row_of, A.val, ti, ta);
    // column of every chunk (into the row_of buffer, no longer needed)
    int* col_of = row_of;
    count_launch();
    k_t_colmap<<<gn, 256, 0, st>>>(n, chbase, col_of);
    count_launch();
    k_t_pull<<<152 * 16, 256, 0, st>>>(n, ATp, ti, ta, B.rowptr, B.col, B.nnz, Cp, Ci, dC, nnzC, chbase, col_of,
                                       pbase, part, hdr);
    count_launch();
    k_t_sum<<<gw, 256, 0, st>>>(n, B.rowptr, B.nnz, chbase, pbase, part, dB);
    return cudaGetLastError();
}

}  // namespace ts
