// Forward product without any device allocation: ts_spgemm_forward_noalloc.
//
// Some callers cannot allocate device memory at the moment they need a
// product: code running inside another framework's memory pool or under a
// fixed memory budget, serving loops that must never call cudaMalloc (it can
// synchronise the device and stall every stream), or code that runs from a
// callback where an allocation is not allowed.  For them this entry point
// takes its scratch space from a fixed array compiled into the library
// instead of a caller workspace.  The caller still allocates A, B and C.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/tsspgemm.h"
#include "kernels.h"

namespace ts {
ts_status set_last_error(ts_status s, const char* msg);
size_t forward_workspace_bytes(const ts_plan* plan);
}

namespace {

// Scratch of every call of ts_spgemm_forward_noalloc on a device.  Each GPU
// that loads the library holds this array until the process exits.
constexpr size_t kScratchBytes = 32u << 20;  // 32 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The host-side
// name of a __device__ array is only a stand-in; its device address has to be
// asked for, once per device, with that device current.
ts_status scratch_for_current_device(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ts::set_last_error(TS_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return ts::set_last_error(TS_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            snprintf(msg, sizeof msg, "ts_spgemm_forward_noalloc: cudaGetSymbolAddress failed: %s",
                     cudaGetErrorString(e));
            return ts::set_last_error(TS_ERR_CUDA, msg);
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return TS_OK;
}

}  // namespace

extern "C" size_t ts_noalloc_scratch_bytes(void) { return kScratchBytes; }

extern "C" ts_status ts_spgemm_forward_noalloc(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                               const ts_csr_desc* C, int64_t* nnzC_host, void* stream) {
    if (!plan || !A || !B || !C || !C->rowptr || !nnzC_host)
        return ts::set_last_error(TS_ERR_INVALID_ARG, "ts_spgemm_forward_noalloc: NULL argument");
    // the layout of the symbolic and numeric passes alone (without the
    // autotuner's trial regions that ts_workspace_size also covers)
    const size_t need = ts::forward_workspace_bytes(plan);
    ts_status s = TS_OK;
    if (need > kScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "ts_spgemm_forward_noalloc: this product needs %zu bytes of scratch, the built-in scratch "
                 "holds %zu; use ts_spgemm_symbolic/ts_spgemm_numeric with a workspace instead",
                 need, kScratchBytes);
        return ts::set_last_error(TS_ERR_UNSUPPORTED, msg);
    }
    void* ws = nullptr;
    if ((s = scratch_for_current_device(&ws)) != TS_OK) return s;
    int64_t nnz = 0;
    if ((s = ts_spgemm_symbolic(plan, A, B, C->rowptr, &nnz, ws, kScratchBytes, stream)) != TS_OK) return s;
    *nnzC_host = nnz;
    if (nnz > C->nnz) {
        char msg[256];
        snprintf(msg, sizeof msg, "ts_spgemm_forward_noalloc: C needs %lld entries, capacity %lld",
                 (long long)nnz, (long long)C->nnz);
        return ts::set_last_error(TS_ERR_CAPACITY, msg);
    }
    ts_csr_desc Cx = *C;
    Cx.nnz = nnz;
    return ts_spgemm_numeric(plan, A, B, &Cx, ws, kScratchBytes, stream);
}
