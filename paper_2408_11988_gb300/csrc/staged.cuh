// Asynchronous staging of gathered B entries (cp.async) for one warp.
//
// The products of a chunk of up to 32 entries of A are numbered 0..total-1
// (entry q owns positions [excl_q, excl_q + len_q), position p of q reads
// B at start_q + p - excl_q).  They are processed in windows of STAGE_P
// positions.  For a window the warp writes, per position, the owning entry
// (one byte) and issues one cp.async per position that copies B's entry
// (8 bytes: column and value bits, or 4 bytes: column) into shared memory;
// the copies of one window form one cp.async group.  Two buffers per warp
// let the warp process window k while window k+1 is in flight, so every
// warp keeps STAGE_P gathers outstanding without holding them in registers.
#pragma once

#include "common.cuh"

namespace ts {

constexpr int STAGE_P = 256;  // positions per window

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

template <int E>
__device__ __forceinline__ void cp_async(void* dst_smem, const void* src_gmem) {
    static_assert(E == 4 || E == 8, "cp.async size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(dst_smem)), "l"(src_gmem),
                 "n"(E)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Per-warp staging area: two buffers, each with STAGE_P payloads of E bytes,
// STAGE_P owner bytes and the 32 entries' value and B offset (start - excl).
template <int E>
struct StageArea {
    static constexpr int BYTES = 2 * (STAGE_P * E + STAGE_P + 32 * 4 + 32 * 8);
    unsigned char* base;
    __device__ __forceinline__ unsigned char* payload(int b) const { return base + b * (STAGE_P * E); }
    __device__ __forceinline__ unsigned char* owner(int b) const {
        return base + 2 * STAGE_P * E + b * STAGE_P;
    }
    __device__ __forceinline__ float* avals(int b) const {
        return reinterpret_cast<float*>(base + 2 * STAGE_P * E + 2 * STAGE_P) + b * 32;
    }
    __device__ __forceinline__ long long* shifts(int b) const {
        return reinterpret_cast<long long*>(base + 2 * STAGE_P * E + 2 * STAGE_P + 2 * 32 * 4) + b * 32;
    }
};

// Prefix data of a loaded chunk: this lane's first position and the total.
struct ChunkScan {
    int excl;
    int total;
};

__device__ __forceinline__ ChunkScan scan_chunk(const Chunk& ch) {
    const int incl = warp_incl_scan(ch.len);
    return ChunkScan{incl - ch.len, __shfl_sync(FULL, incl, 31)};
}

// Issue window [p0, p0 + m) of a chunk into buffer b (all lanes converged).
// src is B's packed (E = 8) or column (E = 4) array.  Returns m.
template <int E>
__device__ __forceinline__ int stage_issue(const StageArea<E>& sa, int b, const Chunk& ch, const ChunkScan& cs,
                                           int p0, const void* src) {
    const int lane = lane_id();
    __syncwarp();  // every lane is done with this buffer's previous window
    unsigned char* own = sa.owner(b);
    const int m = cs.total - p0 < STAGE_P ? cs.total - p0 : STAGE_P;
    const int lo = cs.excl > p0 ? cs.excl : p0;
    const int hi0 = cs.excl + ch.len, hi1 = p0 + STAGE_P;
    const int hi = hi0 < hi1 ? hi0 : hi1;
    for (int p = lo; p < hi; ++p) own[p - p0] = (unsigned char)lane;
    sa.avals(b)[lane] = ch.a;
    sa.shifts(b)[lane] = ch.start - cs.excl;
    __syncwarp();
    const long long* sh = sa.shifts(b);
    unsigned char* pay = sa.payload(b);
#pragma unroll
    for (int k = 0; k < STAGE_P / 32; ++k) {
        const int s = lane + 32 * k;
        if (s < m) {
            const long long j = sh[own[s]] + p0 + s;
            cp_async<E>(pay + s * E, static_cast<const unsigned char*>(src) + j * E);
        }
    }
    cp_async_commit();
    return m;
}

}  // namespace ts
