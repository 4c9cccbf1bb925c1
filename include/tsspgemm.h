/*
 * tsspgemm.h -- C ABI of the GB300 (sm_103a) TS-SpGEMM library.
 *
 * The product computed is the local TS-SpGEMM of the paper: C = A * B with A a
 * square n x n sparse matrix and B a sparse tall-and-skinny n x d matrix
 * (d << n), over a semiring (paper Sec. II-A), row by row after Gustavson
 * (paper Sec. III-A, Eq. 1): row r of C is the semiring sum, over the stored
 * entries (r,c) of A, of A(r,c) times row c of B.  With one GPU there is no
 * distribution: this is the paper's diagonal-tile product LocalSpGEMM over
 * the whole of A (Alg. 2, diagonal-tile step), with a dense accumulator of
 * width d (the SPA of Sec. III-C) or a hash accumulator.
 *
 * Conventions shared by every call
 *  - Matrices are CSR (ts_csr_desc): rowptr int64[nrows+1] with rowptr[0]=0
 *    and rowptr[nrows]=nnz, col int32[nnz] ascending and distinct within a
 *    row, val float32[nnz] (plus-times) or NULL (boolean semiring: a stored
 *    entry means true).  All pointers inside a descriptor are DEVICE pointers.
 *    ts_csr_validate checks these rules on the device.
 *  - The caller owns every device buffer (A, B, C, gradients, workspace).  The
 *    library never allocates device memory; scratch space is the caller's
 *    workspace, whose size the *_workspace_size calls report.  Plans are host
 *    objects owned by the caller and released with the matching destroy call.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    stream ordered; the only calls that synchronise the stream are those
 *    that return a count to the host (documented per call).
 *  - Every call returns a ts_status.  Argument errors are detected on the host
 *    before anything is enqueued.  Malformed CSR content that the host cannot
 *    see (a column index out of range, counts that do not match the symbolic
 *    pass) is caught on the device: the offending access is skipped, a flag
 *    is set in the workspace and the next call that synchronises returns
 *    TS_ERR_BAD_CSR.  No call traps, aborts or exits.  ts_last_error() gives a
 *    message for the calling thread's most recent failure.
 *  - Output rows list their columns in ascending order.  The output pattern is
 *    structural: (i,j) is stored iff some product A(i,k)*B(k,j) exists, even
 *    when plus-times values cancel to 0.
 */
#ifndef TSSPGEMM_H
#define TSSPGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define TS_API __attribute__((visibility("default")))
#else
#define TS_API
#endif

typedef int32_t ts_status;
#define TS_OK 0
#define TS_ERR_INVALID_ARG (-1)        /* bad pointer, size or enum value       */
#define TS_ERR_BAD_CSR (-2)            /* CSR content violates the rules above  */
#define TS_ERR_UNSUPPORTED (-3)        /* valid request this build cannot serve */
#define TS_ERR_WORKSPACE_TOO_SMALL (-4)
#define TS_ERR_CAPACITY (-5)           /* caller's output buffer too small      */
#define TS_ERR_OVERFLOW (-6)           /* a count does not fit its type         */
#define TS_ERR_CUDA (-7)               /* a CUDA runtime call failed            */
#define TS_ERR_STATE (-8)              /* calls made out of the required order  */

/* Semirings (paper Sec. II-A; (and, or) for BFS in Alg. 3). */
#define TS_SR_PLUS_TIMES_F32 0     /* (+, *) on float32 values                   */
#define TS_SR_OR_SELECT2ND_BOOL 1  /* add = OR, multiply = select2nd (= AND here) */

/* Accumulator kinds (paper Sec. III-C: SPA for d <= 1024, hash above). */
#define TS_ACC_AUTO 0
#define TS_ACC_DENSE 1   /* shared-memory dense accumulator + occupancy flags   */
#define TS_ACC_HASH 2    /* shared-memory open-addressing hash accumulator      */
#define TS_ACC_COPIES 3  /* dense accumulator, one private copy per lane group
                          * and no atomics (plus-times; the boolean semiring
                          * uses TS_ACC_DENSE)                                  */
#define TS_ACC_DENSE_B 4 /* B expanded dense in the workspace and each row of C
                          * summed in registers: the dense-B SpMM form of the
                          * product (plus-times, d <= 256; Sec. V's comparison
                          * with SpMM).  TS_ACC_AUTO picks it for plus-times
                          * when B holds at least 600/1000 (64 < d <= 128) or
                          * 450/1000 (128 < d <= 256) of its n*d entries: the
                          * crossovers measured on R-MAT scale-20 products; at
                          * d <= 64 the sparse path stays as fast up to a full
                          * B and is kept                                      */

typedef struct ts_csr_desc {
    int64_t nrows;
    int64_t ncols;
    int64_t nnz;
    int64_t* rowptr; /* device, nrows+1                      */
    int32_t* col;    /* device, nnz                          */
    void* val;       /* device float32[nnz], or NULL         */
} ts_csr_desc;

/*
 * Tuning of one product; 0 in any field means "choose automatically".
 *  accum          TS_ACC_*.
 *  col_tile       accumulator width in columns for the numeric pass (a
 *                 multiple of 32).  Below d, B's columns are processed in
 *                 tiles of this width and each output row is the
 *                 concatenation of its tiles (B column tiling).
 *  cta_min_flops  rows with at least this many products (rounded up to the
 *                 next boundary of the row classes, eighths of an octave of
 *                 products) run CTA-per-row; lighter rows warp-per-row.
 *  warps_per_cta  warps per thread block (1..8).
 *  hash_slots     slots of a warp's hash table (power of two, >= 64).
 *  group          how a warp spreads the products of 32 entries of A over its
 *                 lanes: 1 = one product per lane across entries (any mix of
 *                 B row lengths); 4, 8, 16 or 32 = that many lanes walk one
 *                 entry's row of B (best for rows of about that length);
 *                 2 = quads: four lanes walk one entry's row of B, four
 *                 consecutive entries per lane with 16-byte loads (numeric:
 *                 plus-times with pack_b = 1; symbolic: B.col 16-byte
 *                 aligned; backward: pack_b = 1 and dB 16-byte aligned, its
 *                 dB terms then go out as 16-byte float atomics).  Where a
 *                 pass cannot use quads it falls back to 16 lanes.
 *                 TS_ACC_COPIES needs 8, 16 or 32 (32/group copies per warp);
 *                 with 1 or 4 it picks from B's mean row length.
 *  pack_b         1 = gather B from a packed (column, value) copy built in the
 *                 workspace at each call (for the row-group numeric kernels
 *                 over one column tile: a copy whose rows start on 16-byte
 *                 groups), 2 = from B's own arrays.
 *  sym_group,     the same choice as `group` for the symbolic pass and for
 *  bwd_group      the backward pass (each pass may prefer its own).
 *  row_lanes      numeric pass (plus-times, pack_b = 1, dense accumulator):
 *                 lanes per light row.  32 = one warp per row; 4, 8 or 16 =
 *                 row groups, 32/row_lanes rows per warp in lockstep, each
 *                 with its own accumulator and no atomics (4: four entries
 *                 of B per lane, 8 and 16: two), in a kernel launched right
 *                 behind the one for the heavy rows; with one column tile the
 *                 heavy rows and split parts run in row groups too (slot
 *                 accumulators summed by the block).  Default: 8 for one
 *                 tile of at most 256 columns, else 32.  Any value but 32
 *                 also runs the symbolic pass's light rows in row groups of
 *                 four lanes (d <= 512, B.col 16-byte aligned).
 *  dB_mode        how the backward forms dB (dA is the same either way):
 *                 1 = option S, the dB terms of every product scattered
 *                 with float atomics in the forward's row order (fast; the
 *                 order of the additions, and so the last bits of dB, may
 *                 differ from run to run); 2 = option T, deterministic: the
 *                 transpose of A's pattern (a stable radix sort of A's
 *                 column indices in the workspace), then each row k of dB
 *                 summed over column k of A in ascending row order, dC(i, j)
 *                 found by binary search in the sorted row i of C; no
 *                 atomics, dB identical bit for bit on every run.  Default 1.
 *  stage          1 = gather B's entries into shared memory with asynchronous
 *                 copies, a window of 256 products per warp in flight (implies
 *                 pack_b = 1 for plus-times); 2 = load them into registers.
 */
typedef struct ts_tuning {
    int32_t accum;
    int32_t col_tile;
    int64_t cta_min_flops;
    int32_t warps_per_cta;
    int32_t hash_slots;
    int32_t group;
    int32_t pack_b;
    int32_t stage;
    int32_t sym_group;
    int32_t bwd_group;
    int32_t row_lanes;
    int32_t dB_mode;
} ts_tuning;

typedef struct ts_plan ts_plan;
typedef struct ts_batched_plan ts_batched_plan;

/* Message for the calling thread's most recent failed call ("" if none). */
TS_API const char* ts_last_error(void);
/* Static name of a status code. */
TS_API const char* ts_status_string(ts_status s);
/* Library version as major*10000 + minor*100 + patch. */
TS_API int32_t ts_version(void);
/* Number of CUDA kernels this library has launched in this process. */
TS_API int64_t ts_kernel_launches(void);

/*
 * Validate a CSR matrix on the device: rowptr[0] = 0, rowptr non-decreasing,
 * rowptr[nrows] = nnz, every column in [0, ncols) and strictly ascending in
 * its row.  Synchronises `stream`.  Returns TS_OK or TS_ERR_BAD_CSR, and
 * writes the first offending row (or -1) to *bad_row when bad_row != NULL.
 * ws: at least ts_validate_workspace_size() bytes of device memory.
 */
TS_API size_t ts_validate_workspace_size(void);
TS_API ts_status ts_csr_validate(const ts_csr_desc* M, int64_t* bad_row, void* ws, size_t ws_bytes,
                          void* stream);

/*
 * Plan for C = A * B over `semiring` (TS_SR_*).  Reads only the shapes of A
 * and B (host side, no device access).  `force` (may be NULL) fixes any
 * non-zero tuning field.  A plan may be reused for any A, B of the same
 * shapes.  Errors: INVALID_ARG (shapes: A must be n x n, B n x d, d >= 1),
 * UNSUPPORTED (d above the supported maximum).
 */
TS_API ts_status ts_plan_create(const ts_csr_desc* A, const ts_csr_desc* B, int32_t semiring,
                         const ts_tuning* force, ts_plan** out);
TS_API ts_status ts_plan_destroy(ts_plan* plan);
TS_API ts_status ts_plan_get_tuning(const ts_plan* plan, ts_tuning* out);
TS_API ts_status ts_plan_set_tuning(ts_plan* plan, const ts_tuning* tuning);

/* Device workspace needed by symbolic, numeric, backward and autotune (for
 * plus-times it covers every tuning the autotuner may choose). */
TS_API ts_status ts_workspace_size(const ts_plan* plan, size_t* bytes);

/*
 * Synchronise `stream` and report the device-side checks recorded in ws by
 * the calls since the last symbolic pass: TS_OK, or TS_ERR_BAD_CSR with the
 * failed checks in ts_last_error().
 */
TS_API ts_status ts_workspace_check(const ts_plan* plan, void* ws, size_t ws_bytes, void* stream);

/*
 * Symbolic pass (Eq. 1, pattern only): computes the products per row
 * (flops_i = sum of nnz(B_k) over the stored (i,k)), bins rows by flops,
 * counts nnz(C_i) = |union of the patterns of the rows B_k| and writes
 * C_rowptr (device int64[n+1], caller allocated) as their running sum.
 * When nnzC_host != NULL the total is copied to it and the stream is
 * synchronised; otherwise nothing synchronises and the total stays at
 * C_rowptr[n].  The row schedule it leaves in ws is reused by the numeric
 * and backward calls: keep ws and the patterns of A and B unchanged between
 * them.  Errors: INVALID_ARG, WORKSPACE_TOO_SMALL, BAD_CSR (only reported
 * when synchronising), CUDA.
 */
TS_API ts_status ts_spgemm_symbolic(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                             int64_t* C_rowptr, int64_t* nnzC_host, void* ws, size_t ws_bytes,
                             void* stream);

/*
 * Numeric pass (Eq. 1 with values): fills C->col (and C->val for plus-times)
 * for the C->rowptr of the preceding symbolic call on this plan and ws.
 * C->nnz is the room in C->col / C->val: the symbolic total, or any capacity
 * at least that large (a symbolic call without nnzC_host followed by this
 * call then runs with no host synchronisation at all, so both can be
 * captured in a CUDA graph; nnz(C) is C->rowptr[n]).  Entries past the
 * capacity are not written and are reported as a C row error.  Plus-times
 * sums in float32 in an unspecified order; columns are ascending per row.
 * Does not synchronise.
 * Errors: INVALID_ARG, STATE (no symbolic pass on this plan/ws before),
 * WORKSPACE_TOO_SMALL, CUDA; device-side checks as described at the top.
 */
TS_API ts_status ts_spgemm_numeric(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                            const ts_csr_desc* C, void* ws, size_t ws_bytes, void* stream);

/*
 * Backward of L = sum over C's pattern of dC(i,j) * C(i,j) for C = A*B in
 * plus-times, with the patterns of A, B and C fixed (the paper's sparse
 * embedding, Sec. IV-B, trains through this product):
 *   dA(i,k) = sum over j in B_k of dC(i,j) * B(k,j)          (sampled dense-
 *             dense product on A's pattern, SDDMM)
 *   dB(k,j) = sum over i with A(i,k) stored of A(i,k) * dC(i,j)  (A^T dC on
 *             B's pattern)
 * dC_val holds float32 values on C's pattern (C->val is not read); dA_val
 * (nnz_A floats) and dB_val (nnz_B floats) are outputs, either may be NULL.
 * dB is summed with float atomics, so its rounding is not deterministic.
 * Uses the row schedule of the preceding symbolic call on this plan and ws.
 * Does not synchronise.  Errors as for the numeric pass; UNSUPPORTED for the
 * boolean semiring.
 */
TS_API ts_status ts_spgemm_backward(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                             const ts_csr_desc* C, const float* dC_val, float* dA_val,
                             float* dB_val, void* ws, size_t ws_bytes, void* stream);
/* The two halves of ts_spgemm_backward on their own (same contract). */
TS_API ts_status ts_spgemm_backward_dA(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                const ts_csr_desc* C, const float* dC_val, float* dA_val,
                                void* ws, size_t ws_bytes, void* stream);
TS_API ts_status ts_spgemm_backward_dB(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                const ts_csr_desc* C, const float* dC_val, float* dB_val,
                                void* ws, size_t ws_bytes, void* stream);

/*
 * Autotuner: times the numeric pass (and, for plus-times, the backward when
 * dC_val != NULL) for a set of candidate tunings on these very inputs, keeps
 * the fastest in the plan and writes it to *chosen (may be NULL).  Fields
 * fixed by the plan's `force` are not varied.  C must come from a symbolic
 * call on this plan/ws (C's contents are overwritten; dA/dB scratch is
 * written into dA_scratch/dB_scratch when given).  `reps` timed repetitions
 * per candidate (>= 1).  Synchronises the stream.
 */
TS_API ts_status ts_plan_autotune(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                           const ts_csr_desc* C, const float* dC_val, float* dA_scratch,
                           float* dB_scratch, int32_t reps, ts_tuning* chosen, void* ws,
                           size_t ws_bytes, void* stream);

/*
 * Multi-source BFS (paper Alg. 3) one level at a time.
 *
 * msbfs_workspace_size: device workspace for a graph of n vertices and nnz_A
 * stored edges with d sources.
 *
 * msbfs_init: F0 gets the frontier of d sources (F0(src[s], s) = 1), the
 * visited bitmap S (uint32[n * ceil(d/32)], bit s of vertex v at word
 * v*ceil(d/32) + s/32) is set to F0, levels (int32[n*d], vertex-major) to
 * -1 except level 0 at the sources.  sources_dev: device int32[d], distinct
 * vertices in [0, n).  F0->rowptr is n+1 int64, F0->col must hold >= d
 * entries.  Does not synchronise.
 *
 * msbfs_step: one iteration of Alg. 3's loop body:
 *   N = A * F over (or, select2nd);  F_next = N minus S;  S = S or N;
 * and levels(v, s) = level for every bit of F_next.  A is the pattern of
 * the graph (val ignored); row v of N pulls from the rows of F at v's
 * neighbours, i.e. the traversal follows the edges of A transposed
 * (identical for a symmetric A).  F_next->rowptr (n+1) is always written;
 * F_next->col (capacity F_next_capacity) receives the frontier.
 * Synchronises the stream once and writes nnz(F_next) to *nnz_next_host.
 * If it exceeds the capacity, returns TS_ERR_CAPACITY with the needed size
 * in *nnz_next_host; S, levels and F_next->rowptr are then already updated
 * and the call must be repeated by msbfs_emit with a larger buffer.
 */
TS_API ts_status msbfs_workspace_size(int64_t n, int64_t nnz_A, int64_t d, size_t* bytes);
TS_API ts_status msbfs_init(int64_t n, int64_t d, const int32_t* sources_dev, uint32_t* visited,
                     int32_t* levels, const ts_csr_desc* F0, void* stream);
TS_API ts_status msbfs_step(const ts_csr_desc* A, const ts_csr_desc* F, uint32_t* visited,
                     int32_t* levels, int32_t level, const ts_csr_desc* F_next,
                     int64_t F_next_capacity, int64_t* nnz_next_host, void* ws, size_t ws_bytes,
                     void* stream);
/*
 * Sparse Force2Vec minibatch step (paper Sec. IV, "Distributed sparse
 * embedding": attractive and repulsive forces through TS-SpGEMM, SGD, then
 * sparsification keeping the largest entries).  For the rows [r0, r0 + b) of
 * the sparse embedding Z (n x d, exactly k entries per row, Z.rowptr[i] =
 * k*i, values float32), with A (n x n, pattern; values ignored):
 *   W(r, j) = npos - (npos + nneg) * sigmoid(z_i . z_j)   (i = r0 + r),
 *     npos = [A(i, j) stored], nneg = occurrences of j in the row's s
 *     negative samples neg[r*s .. r*s+s) (device int32, vertex ids);
 *   G = W * Z (this library's plus-times TS-SpGEMM);
 *   U_i = z_i + lr * G_r;  new row i = the k entries of U_i of largest
 *     magnitude (ties: smaller column), ascending columns.
 * Every row of the batch is computed from the old Z; the new rows then
 * overwrite Z's batch rows in place (Z.col and Z.val are written).  U_out:
 * optional device float32[b*d] receiving the dense U before sparsification
 * (NULL: not written).  ws: f2v_workspace_size bytes, 256-byte aligned.
 * Synchronises `stream`.  Errors: TS_ERR_INVALID_ARG (shapes, batch range,
 * NULL), TS_ERR_UNSUPPORTED (d > 4096, k > d, s > 32, n >= 2^31),
 * TS_ERR_WORKSPACE_TOO_SMALL, TS_ERR_BAD_CSR (device checks: columns out of
 * range, Z not k entries per row), TS_ERR_CUDA.
 */
TS_API ts_status f2v_workspace_size(int64_t n, int64_t d, int64_t nnz_A, int64_t b, int32_t s, int32_t k,
                                    size_t* bytes);
TS_API ts_status f2v_step(const ts_csr_desc* A, const ts_csr_desc* Z, int64_t r0, int64_t b, const int32_t* neg,
                          int32_t s, float lr, int32_t k, float* U_out, void* ws, size_t ws_bytes, void* stream);

/*
 * BFS-tree variant of the level step (paper Sec. IV: Alg. 3 with the
 * (sel2nd, min) semiring, used when the BFS tree is to be reconstructed): the
 * same step as msbfs_step, and in addition parents[v*d + s] = the smallest
 * neighbour u of v (a stored A(v,u)) that is in the frontier of source s, for
 * every (v, s) that enters the frontier at this level.  parents: device
 * int32[n*d], vertex-major like levels, caller-owned; entries of vertices not
 * reached at this level are left untouched.  Requires d <= 256 (the bitmap
 * pull form of the step); larger d returns TS_ERR_UNSUPPORTED.  Other
 * arguments, errors and synchronisation as msbfs_step.
 */
TS_API ts_status msbfs_step_parents(const ts_csr_desc* A, const ts_csr_desc* F, uint32_t* visited,
                                    int32_t* levels, int32_t* parents, int32_t level,
                                    const ts_csr_desc* F_next, int64_t F_next_capacity,
                                    int64_t* nnz_next_host, void* ws, size_t ws_bytes, void* stream);

/*
 * Parents before the first step: parents[v*d + s] = -1 everywhere, and
 * parents[src[s]*d + s] = src[s] (a source is its own parent).  sources_dev:
 * device int32[d]; parents: device int32[n*d].  d <= 256.  Stream-ordered,
 * no synchronisation.  Errors: TS_ERR_INVALID_ARG, TS_ERR_UNSUPPORTED,
 * TS_ERR_CUDA.
 */
TS_API ts_status msbfs_init_parents(int64_t n, int64_t d, const int32_t* sources_dev, int32_t* parents,
                                    void* stream);

/* Writes F_next->col from the state a TS_ERR_CAPACITY msbfs_step left in ws. */
TS_API ts_status msbfs_emit(const ts_csr_desc* F_next, int64_t F_next_capacity, void* ws,
                     size_t ws_bytes, void* stream);

/*
 * Batched products: `count` independent C_b = A_b * B_b of uneven shapes
 * (the serving pattern of many graphs at once; the paper has no batched
 * mode), each phase one launch over all instances, graph capturable.  The
 * kernels read and write every instance's own arrays through a device table
 * of instance descriptors; the rows of all instances are numbered one after
 * another and scheduled together (rows with products at or above their
 * instance's heavy threshold one block each from a list, the others one warp
 * each).  Forward: four launches (row flops with the packed and dense copies
 * of B, row counts, per-instance scan, numeric); backward: two (clear dA/dB,
 * gradients).  Every instance has its own tuning in its descriptor: the
 * accumulator (the shared accumulator with occupancy bits over one column
 * tile of d_b padded to 32, or the dense-B form for d_b <= 256) and the
 * heavy-row threshold.  d_b is at most 1024.
 *
 * Protocol (descriptor arrays are host arrays of `count` descriptors with
 * device pointers):
 *  1. ts_batched_plan_create reads shapes and nnz only (host).  `force`
 *     fixes, for every instance, accum (TS_ACC_DENSE_B: the dense-B form
 *     where d_b <= 256 and the product is plus-times; any other non-zero
 *     value: the shared accumulator) and cta_min_flops (the heavy
 *     threshold); 0 chooses per instance (dense-B above the density
 *     crossover of TS_ACC_DENSE_B, threshold 4096).  Other fields are unused.
 *  2. ts_batched_workspace_size, then ts_batched_bounds: computes, on the
 *     device, C_capacity[b] = sum over the rows of A_b of min(d_b, flops_i),
 *     an upper bound on nnz(C_b) (synchronises).
 *  3. ts_batched_bind: the caller allocates C_b (rowptr n_b+1, col/val with
 *     C_b.nnz >= C_capacity[b]) and binds A, B, C (uploads the descriptors,
 *     synchronises).  ts_batched_bind_grads binds per-instance dC (nnz(C_b)
 *     entries), dA (nnz(A_b)) and dB (nnz(B_b)) arrays; NULL entries skip an
 *     output.
 *  4. ts_spgemm_batched / ts_spgemm_batched_backward: no host
 *     synchronisation and no allocation, so they can be captured in a CUDA
 *     graph and replayed.  The descriptor / gradient arrays passed must equal
 *     those bound (checked on the host).  After the forward, C_b.rowptr holds
 *     the exact structure and nnz(C_b) = C_b.rowptr[n_b]; an instance whose C
 *     exceeds its capacity gets its entries up to the capacity only, and the
 *     error (TS_ERR_CAPACITY) is reported by ts_batched_check.  The backward
 *     uses the row flops and the C pattern of the preceding forward.
 *  ts_batched_check synchronises and reports device-side errors.
 *  ts_batched_autotune times, instance by instance, every accumulator kind
 *  it may use and heavy thresholds of 1024, 4096, 16384 products and none
 *  on that instance alone; then it times the whole batch under those
 *  choices, under the tuning it started from, and under the instances' own
 *  accumulators with one heavy threshold (1024, 4096 or 16384) for all, and
 *  keeps the fastest of these.  It leaves every C_b computed with the
 *  chosen tunings; `chosen` (may be NULL)
 *  receives instance 0's.  ts_batched_get_tuning reports instance b's
 *  tuning (accum TS_ACC_DENSE or TS_ACC_DENSE_B, col_tile = its accumulator
 *  width, cta_min_flops = its heavy threshold).
 */
TS_API ts_status ts_batched_plan_create(int32_t count, const ts_csr_desc* A, const ts_csr_desc* B,
                                        int32_t semiring, const ts_tuning* force, ts_batched_plan** out);
TS_API ts_status ts_batched_plan_destroy(ts_batched_plan* plan);
TS_API ts_status ts_batched_workspace_size(const ts_batched_plan* plan, size_t* bytes);
TS_API ts_status ts_batched_bounds(ts_batched_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                   int64_t* C_capacity, void* ws, size_t ws_bytes, void* stream);
TS_API ts_status ts_batched_bind(ts_batched_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                 const ts_csr_desc* C, void* ws, size_t ws_bytes, void* stream);
TS_API ts_status ts_batched_bind_grads(ts_batched_plan* plan, int32_t count, const float* const* dC_val,
                                       float* const* dA_val, float* const* dB_val, void* ws, size_t ws_bytes,
                                       void* stream);
TS_API ts_status ts_spgemm_batched(ts_batched_plan* plan, int32_t count, const ts_csr_desc* A,
                                   const ts_csr_desc* B, const ts_csr_desc* C, void* ws, size_t ws_bytes,
                                   void* stream);
TS_API ts_status ts_spgemm_batched_backward(ts_batched_plan* plan, int32_t count, const float* const* dC_val,
                                            float* const* dA_val, float* const* dB_val, void* ws,
                                            size_t ws_bytes, void* stream);
TS_API ts_status ts_batched_check(ts_batched_plan* plan, void* ws, size_t ws_bytes, void* stream);
TS_API ts_status ts_batched_autotune(ts_batched_plan* plan, int32_t reps, ts_tuning* chosen, void* ws,
                                     size_t ws_bytes, void* stream);
TS_API ts_status ts_batched_get_tuning(const ts_batched_plan* plan, int32_t b, ts_tuning* out);

/*
 * Forward product that allocates nothing (the paper has no counterpart; this
 * is a service for callers).  Some callers cannot allocate device memory when
 * they need a product: code running inside another framework's memory pool
 * or under a fixed memory budget, serving loops that must not call cudaMalloc
 * (it can synchronise the whole device), or code run from a callback where
 * allocation is not allowed.  This call runs the symbolic and numeric passes
 * with scratch space taken from a fixed array compiled into the library
 * (ts_noalloc_scratch_bytes(), 32 MiB, held by every GPU that loads the
 * library until the process exits) instead of a caller workspace.
 *
 * The caller passes A, B and C as for the other calls: C->rowptr (n+1 int64)
 * and C->col / C->val with room for C->nnz entries (the capacity).  On return
 * *nnzC_host holds nnz(C); if it exceeds the capacity the call returns
 * TS_ERR_CAPACITY after writing C->rowptr only.  Products whose forward
 * workspace (the symbolic and numeric passes of the plan's current tuning;
 * ts_workspace_size may be larger, since it also covers the autotuner's
 * trials) exceeds the scratch are rejected with TS_ERR_UNSUPPORTED before
 * anything is enqueued.  The call synchronises `stream` once (to read
 * nnz(C)) and calls no allocating function.  Because of that synchronisation
 * it cannot be called while `stream` is being captured into a CUDA graph.
 *
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress), which needs that device to be current.  All calls
 * on a device share the one scratch array and each call re-initialises what
 * it needs, so calls whose work overlaps on the GPU (different streams,
 * different threads) race: serialise them.
 */
TS_API size_t ts_noalloc_scratch_bytes(void);
TS_API ts_status ts_spgemm_forward_noalloc(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                           const ts_csr_desc* C, int64_t* nnzC_host, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TSSPGEMM_H */
