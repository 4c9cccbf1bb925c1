// Internal launchers of the TS-SpGEMM kernels (host side, C++).  The public C
// ABI in include/tsspgemm.h is implemented on top of these in api.cpp.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace ts {

struct WsHeader;

// CSR view with device pointers (int64 row pointers, int32 columns).
struct DevCsr {
    long long nrows = 0, ncols = 0, nnz = 0;
    const long long* rowptr = nullptr;
    const int* col = nullptr;
    const float* val = nullptr;
};

// Row schedule written by the binning kernels into the workspace.
struct Sched {
    WsHeader* hdr = nullptr;     // counters, class histogram
    long long* flops = nullptr;  // products per row of A, int64[n]
    int* perm = nullptr;         // non-empty rows, heaviest class first, int32[n]
    long long* partial = nullptr;// scan partial sums
    long long* items = nullptr;  // (row, chunk) work items of long rows for the flops pass
    int* blen = nullptr;         // row lengths of B (clamped), for the flops pass, or nullptr
    // split rows (more than SPLIT_ENTRIES entries of A): row ids, completion
    // counters, (slot, part) work items and per-slot staging of partial rows
    int* split_rows = nullptr;        // [MAX_SPLIT_ROWS]
    int* split_done = nullptr;        // [MAX_SPLIT_ROWS]
    long long* split_items = nullptr; // [split_item_capacity]
    unsigned* stg_bits = nullptr;     // [MAX_SPLIT_ROWS][dw]     symbolic
    float* stg_vals = nullptr;        // [MAX_SPLIT_ROWS][dpad]   numeric (dense)
    unsigned char* stg_flags = nullptr; // [MAX_SPLIT_ROWS][dpad] numeric (dense)
    int dw = 0, dpad = 0;
};

// Capacity (entries) of Sched::split_items for nnzA entries of A.
long long split_item_capacity(long long nnzA);

// Capacity (entries) of Sched::items for a matrix with n rows and nnzA entries.
long long flops_item_capacity(long long n, long long nnzA);

struct LaunchCfg {
    int warps_per_cta = 8;
    int cta_class = 14;      // rows of flops class >= this run CTA-per-row
    int sms = 152;
    int group = 1;           // lanes per A entry (1 = flattened products)
    int row_lanes = 32;      // numeric light rows: 32 = a warp per row, 4/8/16 = row groups,
                             // 1 = a warp per row on one shared accumulator (wide kernel)
};

// Bytes of the scan partials for n values.
size_t scan_partial_count(long long n);

// flops per row, class histogram and (when Cp != nullptr) Cp[i+1] = 0 for
// rows without products; then perm = non-empty rows ordered by class.
cudaError_t launch_row_schedule(const DevCsr& A, const DevCsr& B, const Sched& s, long long* Cp,
                                cudaStream_t st);
// The two halves: flops per row (clears the header), and histogram + perm
// from the flops array (Cp_next[i] = 0 for rows without products if given).
cudaError_t launch_row_flops(const DevCsr& A, const DevCsr& B, const Sched& s, cudaStream_t st);
cudaError_t launch_reclassify(long long n, const Sched& s, long long* Cp_next, cudaStream_t st);

// Symbolic pass: Cp[i+1] = nnz(C_i) for the scheduled rows, then Cp = running sum.
cudaError_t launch_symbolic(const DevCsr& A, const DevCsr& B, long long d, const Sched& s,
                            const LaunchCfg& cfg, long long* Cp, cudaStream_t st);

// In-place inclusive scan of x[0..n) (int64) using partial[] as scratch.
cudaError_t launch_scan_inplace(long long* x, long long n, long long* partial, cudaStream_t st);

// Column-tile offsets: tp[k*(T+1)+t] = first position of row k of B with
// column >= t*W (t = 0..T; t = T gives the row end).
cudaError_t launch_tile_split(const DevCsr& B, int W, int T, long long* tp, cudaStream_t st);

// Numeric pass with a dense accumulator of width W over T column tiles.
// Bpk: packed (column, value) copy of B or nullptr; G: lanes per A entry
// (1 = flattened products).
// Bq: row-aligned packed copy of B (launch_pack_b_rows, groups of 4 entries
// for row_lanes 4, else 2) for the row-group kernels with T = 1, or nullptr.
cudaError_t launch_numeric_dense(const DevCsr& A, const DevCsr& B, long long d, int W, int T,
                                 const long long* tp, bool values, const int2* Bpk, int G,
                                 const Sched& s, const LaunchCfg& cfg, const long long* Cp, int* Ci,
                                 float* Cx, long long nnzC, cudaStream_t st, const int4* Bq = nullptr);
// Numeric pass with the dense accumulator and cp.async staging of B.
cudaError_t launch_numeric_staged(const DevCsr& A, const DevCsr& B, long long d, int W, int T,
                                  const long long* tp, bool values, const int2* Bpk, const Sched& s,
                                  const LaunchCfg& cfg, const long long* Cp, int* Ci, float* Cx, long long nnzC,
                                  cudaStream_t st);
size_t numeric_staged_smem(int W, int warps, bool values);
// Plus-times numeric pass with per-group copies of the dense accumulator (no
// atomics); G = 8, 16 or 32 lanes per entry of A, 32/G copies per warp.
cudaError_t launch_numeric_copies(const DevCsr& A, const DevCsr& B, long long d, int W, int T,
                                  const long long* tp, const int2* Bpk, int G, const Sched& s,
                                  const LaunchCfg& cfg, const long long* Cp, int* Ci, float* Cx, long long nnzC,
                                  cudaStream_t st, bool skip_light = false);
// Dynamic shared memory of that pass (0 for an unsupported G).
size_t numeric_copies_smem(int W, int G, int warps);
// Packed (column, value bits) copy of B's entries.
cudaError_t launch_pack_b(const DevCsr& B, int2* P, cudaStream_t st);
// Row-aligned packed copy of B: row k starts at entry E*ceil((Bp[k] + (E-1)k)/E),
// its last group padded with column -1; columns outside [0, d) are stored as
// -1 and set ERR_B_COL in *err.  E = 2 or 4.
cudaError_t launch_pack_b_rows(const DevCsr& B, int E, long long d, int4* Q, unsigned long long* err,
                               cudaStream_t st);
size_t padded_b_bytes(long long nB, long long nnzB, long long d, int E);
// Whether the copy's groups can be numbered with 32 bits.
bool padded_b_fits(long long nB, long long nnzB, long long d, int E);

// Numeric pass with a per-warp hash accumulator of `slots` entries.
cudaError_t launch_numeric_hash(const DevCsr& A, const DevCsr& B, long long d, int slots,
                                bool values, const Sched& s, const LaunchCfg& cfg,
                                const long long* Cp, int* Ci, float* Cx, long long nnzC,
                                cudaStream_t st);
size_t numeric_dense_smem(int W, int warps, bool values);
// Light rows only, in row groups of cfg.row_lanes lanes (4, 8 or 16; packed
// B), launched with programmatic dependent launch behind a numeric kernel
// that skipped them.
cudaError_t launch_numeric_light_rows(const DevCsr& A, const DevCsr& B, long long d, int W, int T,
                                      const long long* tp, const int2* Bpk, const Sched& s, const LaunchCfg& cfg,
                                      const long long* Cp, int* Ci, float* Cx, long long nnzC, cudaStream_t st);
// Dynamic shared memory of the row-group light-row kernel (0: bad row_lanes).
size_t numeric_light_smem(int W, int warps, int row_lanes);
size_t numeric_rgcta_smem(int W, int warps, int row_lanes);
// Dynamic shared memory of the wide kernel (row_lanes = 1: one accumulator
// of W <= 1024 floats and its occupancy bitmap per warp).
size_t numeric_wide_smem(int W, int warps);
struct NumParams;
// Rows with 1 .. TINY_MAX products of the wide pass (numeric_tiny.cu).
cudaError_t launch_numeric_tiny(const NumParams& p, int sms, cudaStream_t st);
size_t numeric_hash_smem(int slots, int warps, bool values);

// Numeric pass with B expanded dense (plus-times, d <= 256): dense_ws holds
// dense_b_bytes(B.nrows, d) bytes for the copy and its pattern bitmap.
size_t dense_b_bytes(long long nB, long long d);
cudaError_t launch_numeric_denseb(const DevCsr& A, const DevCsr& B, long long d, const Sched& s,
                                  const LaunchCfg& cfg, const long long* Cp, int* Ci, float* Cx, long long nnzC,
                                  void* dense_ws, cudaStream_t st);

// Backward: dA (SDDMM on A's pattern) and dB (A^T dC on B's pattern).
cudaError_t launch_backward(const DevCsr& A, const DevCsr& B, long long d, const long long* Cp,
                            const int* Ci, long long nnzC, const float* dC, float* dA, float* dB,
                            const int2* Bpk, const Sched& s, const LaunchCfg& cfg, cudaStream_t st);
size_t backward_smem(long long d, int warps);

// Deterministic dB (option T): workspace bytes, and the pass (transpose of
// A's pattern by a stable radix sort, pull over B's rows, ordered sums).
size_t backward_t_bytes(long long n, long long nnzA, long long nnzB, long long d);
cudaError_t launch_backward_t(const DevCsr& A, const DevCsr& B, long long d, const long long* Cp, const int* Ci,
                              long long nnzC, const float* dC, float* dB, void* ws, WsHeader* hdr, cudaStream_t st);

// Multi-source BFS (Alg. 3) levels.
cudaError_t launch_msbfs_init(long long n, int d, const int* src, unsigned* S, int* levels,
                              long long* rp, int* col, cudaStream_t st);
// fbits: workspace for the frontier as a bitmap (n x msbfs_pull_words(d)
// words); with it and d <= 256 the pull form runs, else the list form.
cudaError_t launch_msbfs_step(const DevCsr& A, const DevCsr& F, int d, unsigned* S, int* levels,
                              int level, const Sched& s, unsigned* newbits, long long* rp_next,
                              const LaunchCfg& cfg, cudaStream_t st, unsigned* fbits = nullptr,
                              int* parents = nullptr);
int msbfs_pull_words(int d);
cudaError_t launch_msbfs_init_parents(long long n, int d, const int* src, int* parents, cudaStream_t st);
cudaError_t launch_msbfs_emit(long long n, int d, const unsigned* newbits, const long long* rp,
                              int* col, long long cap, WsHeader* hdr, cudaStream_t st);

// One instance of a batched product (device-side descriptor), with its own
// tuning: accumulator width W (d padded to 32, at most 1024), accumulator
// kind (BAT_SPARSE: shared accumulator with occupancy bits; BAT_DENSE_B:
// the dense-B form, d <= 256) and heavy-row threshold; Bq, Bd and Bbits
// point into the workspace (its packed and dense copies of B).
constexpr int BAT_SPARSE = 0;
constexpr int BAT_DENSE_B = 1;
struct InstDesc {
    long long n, d, annz, bnnz, cap;
    long long row_off;  // first row of this instance in the batch's numbering
    const long long* A_rowptr;
    const int* A_col;
    const float* A_val;
    const long long* B_rowptr;
    const int* B_col;
    const float* B_val;
    long long* C_rowptr;
    int* C_col;
    float* C_val;
    const float* dC;
    float* dA;
    float* dB;
    long long heavy_min;
    long long chunk_off;  // first 32-row chunk of this instance in the batch's chunk numbering
    int W, accum, Wd, pad;
    int4* Bq;
    float* Bd;
    unsigned* Bbits;
};
// Counters and error bits of a batched call (in the workspace).
// Counters of one batched forward (+ backward): heavy rows found, the
// heavy-row queues of the three passes (q_*) and their light-chunk queues
// (l_*), and the error flags.  The forward zeroes all of it, the backward
// q_bwd and l_bwd.
struct BatchCtl {
    unsigned long long nheavy, q_sym, q_num, q_bwd, l_bwd, l_sym, l_num, l_prep, err;
};
// 32-row chunks [c0, c1) of the batch's chunk numbering over the instances
// inst[0..count) (every chunk lies in one instance).
cudaError_t launch_bat_prepare(const InstDesc* inst, int count, long long c0, long long c1, long long* flops,
                               int* heavy, BatchCtl* ctl, int sms, cudaStream_t st);
// symbolic / numeric: 32-row chunks [c0, c1) of the batch's chunk numbering
// (every chunk lies in one instance); `values` = plus-times
cudaError_t launch_bat_symbolic(const InstDesc* inst, int count, long long c0, long long c1, long long unused,
                                const long long* flops, const int* heavy, BatchCtl* ctl, int Wmax, int sms,
                                cudaStream_t st);
cudaError_t launch_bat_scan(const InstDesc* inst, int count, BatchCtl* ctl, cudaStream_t st);
cudaError_t launch_bat_numeric(const InstDesc* inst, int count, long long c0, long long c1, long long values,
                               const long long* flops, const int* heavy, BatchCtl* ctl, int Wmax, int sms,
                               cudaStream_t st);
cudaError_t launch_bat_backward(const InstDesc* inst, int count, long long g0, long long g1, long long max_work,
                                const long long* flops, const int* heavy, BatchCtl* ctl, int Wmax, int sms,
                                cudaStream_t st);
cudaError_t launch_batch_bounds(const InstDesc* inst, int count, const long long* flops, long long* bound,
                                cudaStream_t st);

// Sparse Force2Vec step (force2vec.cu): W's pattern (count + scan, fill),
// the Z layout check, the weights on W's pattern, and update + top-k +
// commit into Z's batch rows.
cudaError_t launch_f2v_pattern(const DevCsr& A, long long r0, long long b, const int* neg, int s, long long* Wp,
                               unsigned* newmask, long long* partial, WsHeader* hdr, cudaStream_t st);
cudaError_t launch_f2v_fill(const DevCsr& A, long long r0, long long b, const int* neg, int s, const long long* Wp,
                            const unsigned* newmask, int* Wcol, int* Wmult, int* Wrow, cudaStream_t st);
cudaError_t launch_f2v_check(const DevCsr& Z, int k, WsHeader* hdr, cudaStream_t st);
cudaError_t launch_f2v_weights(const DevCsr& Z, int k, long long r0, long long b, const long long* Wp,
                               const int* Wcol, const int* Wmult, const int* Wrow, float* Wval, cudaStream_t st);
cudaError_t launch_f2v_update(const DevCsr& Z, int k, long long r0, long long b, const long long* Gp, const int* Gc,
                              const float* Gv, float lr, float* U_out, int* Sc, float* Sv, int sms, WsHeader* hdr,
                              cudaStream_t st);

// CSR validation; writes the first bad row (or -1) into *bad (device).
cudaError_t launch_validate(const DevCsr& M, long long* bad, cudaStream_t st);

// Process-wide count of kernel launches made by this library.
void count_launch();
long long launch_count();

// Occupancy-derived persistent grid size.
int persistent_grid(const void* kernel, int threads, size_t smem, int sms);

}  // namespace ts
