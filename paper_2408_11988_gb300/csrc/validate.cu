// CSR validation on the device: the preconditions every entry point assumes.
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace ts {

// Thread per row.  A row is bad if its range is not inside [0, nnz] or not
// non-decreasing, if it is row 0 and does not start at 0, if it is the last
// row and does not end at nnz, or if its columns are not strictly ascending
// inside [0, ncols).  The smallest bad row index is kept.
__global__ void k_validate(long long n, long long ncols, long long nnz, const long long* __restrict__ rp,
                           const int* __restrict__ ci, unsigned long long* bad) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long s = rp[i], e = rp[i + 1];
        bool ok = s >= 0 && e >= s && e <= nnz;
        if (i == 0 && s != 0) ok = false;
        if (i == n - 1 && e != nnz) ok = false;
        if (ok) {
            long long prev = -1;
            for (long long q = s; q < e; ++q) {
                const long long c = ci[q];
                if (c <= prev || c >= ncols) {
                    ok = false;
                    break;
                }
                prev = c;
            }
        }
        if (!ok) atomicMin(bad, (unsigned long long)i);
    }
}

cudaError_t launch_validate(const DevCsr& M, long long* bad, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(bad, 0xFF, sizeof(long long), st))) return e;
    if (M.nrows == 0) return cudaSuccess;
    long long blocks = (M.nrows + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    count_launch();
    k_validate<<<(unsigned)blocks, 256, 0, st>>>(M.nrows, M.ncols, M.nnz, M.rowptr, M.col,
                                                 (unsigned long long*)bad);
    return cudaGetLastError();
}

}  // namespace ts
