// Host side of the C ABI declared in include/tsspgemm.h: argument checks,
// plans and tuning, workspace layout, and dispatch to the kernel launchers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/tsspgemm.h"
#include "kernels.h"
#include "layout.h"

using namespace ts;

// NVTX range around an entry point or one of its phases, so that a profiler
// timeline (nsys, ncu --nvtx) shows the passes by name.  Without a tool
// attached the push and pop cost a few nanoseconds.
namespace {
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

static ts_status fail(ts_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

static ts_status cuda_fail(cudaError_t e, const char* where) {
    return fail(TS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define TS_CUDA(call, where)                         \
    do {                                             \
        cudaError_t _e = (call);                     \
        if (_e != cudaSuccess) return cuda_fail(_e, where); \
    } while (0)

static ts_status ok() {
    g_last_error.clear();
    return TS_OK;
}

extern "C" const char* ts_last_error(void) { return g_last_error.c_str(); }

// Lets other translation units of the library report an error message.
namespace ts {
ts_status set_last_error(ts_status s, const char* msg) {
    g_last_error = msg ? msg : "";
    return s;
}
}  // namespace ts

extern "C" const char* ts_status_string(ts_status s) {
    switch (s) {
        case TS_OK: return "TS_OK";
        case TS_ERR_INVALID_ARG: return "TS_ERR_INVALID_ARG";
        case TS_ERR_BAD_CSR: return "TS_ERR_BAD_CSR";
        case TS_ERR_UNSUPPORTED: return "TS_ERR_UNSUPPORTED";
        case TS_ERR_WORKSPACE_TOO_SMALL: return "TS_ERR_WORKSPACE_TOO_SMALL";
        case TS_ERR_CAPACITY: return "TS_ERR_CAPACITY";
        case TS_ERR_OVERFLOW: return "TS_ERR_OVERFLOW";
        case TS_ERR_CUDA: return "TS_ERR_CUDA";
        case TS_ERR_STATE: return "TS_ERR_STATE";
        default: return "TS_ERR_UNKNOWN";
    }
}

extern "C" int32_t ts_version(void) { return 100; }  // 0.1.0

extern "C" int64_t ts_kernel_launches(void) { return launch_count(); }

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
static long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

static int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return 152;
    return sms;
}

static ts_status check_desc(const ts_csr_desc* M, const char* name, bool need_val) {
    if (!M) return fail(TS_ERR_INVALID_ARG, "%s: descriptor is NULL", name);
    if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0)
        return fail(TS_ERR_INVALID_ARG, "%s: negative size", name);
    if (M->nrows > INT32_MAX || M->ncols > INT32_MAX)
        return fail(TS_ERR_UNSUPPORTED, "%s: more than 2^31-1 rows or columns", name);
    if (!M->rowptr) return fail(TS_ERR_INVALID_ARG, "%s: rowptr is NULL", name);
    if (M->nnz > 0 && !M->col) return fail(TS_ERR_INVALID_ARG, "%s: col is NULL", name);
    if (need_val && M->nnz > 0 && !M->val)
        return fail(TS_ERR_INVALID_ARG, "%s: val is NULL for the plus-times semiring", name);
    return TS_OK;
}

static DevCsr dev(const ts_csr_desc* M) {
    DevCsr c;
    c.nrows = M->nrows;
    c.ncols = M->ncols;
    c.nnz = M->nnz;
    c.rowptr = (const long long*)M->rowptr;
    c.col = M->col;
    c.val = (const float*)M->val;
    return c;
}

static int cta_class_of(long long min_flops) { return class_at_least(min_flops); }

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------
struct ts_plan {
    long long n = 0, d = 0;
    long long nnzA = 0, nnzB = 0;
    int semiring = 0;
    ts_tuning force{};
    ts_tuning cur{};
    // state of the last symbolic call (its row schedule lives in that ws)
    bool sym_valid = false;
    const void* sym_ws = nullptr;
    const void* sym_ptrs[4] = {nullptr, nullptr, nullptr, nullptr};
    long long sym_nnz[2] = {0, 0};
};

static const long long MAX_D = 1LL << 20;

// Lanes per A entry for pass 0 (numeric), 1 (symbolic), 2 (backward).
// Measured on the R-MAT embedding products (rows of B with 10-13 entries):
// the flag-based numeric pass is fastest flattened (its shared-memory float
// atomics collide more when eight rows of B are in flight, as with quads),
// the symbolic and backward passes with quads (16-byte loads, and 16-byte
// dB atomics in the backward); rows of B of fewer than 3 entries on average
// leave most quad lanes idle and use the flattened mode there.
static int auto_group(long long nB, long long nnzB, int pass) {
    const double avg = nB > 0 ? (double)nnzB / (double)nB : 0.0;
    if (pass == 2) return 2;  // backward: quads (16 lanes where quads do not apply)
    if (avg < 3.0) return 1;
    if (pass == 1) return 2;  // symbolic: quads (16 lanes where quads do not apply)
    if (avg >= 24.0) return 32;
    return 1;
}

static bool valid_group(int g) { return g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32; }

// Lanes per entry of A for TS_ACC_COPIES: the tuned group if it is 8, 16 or
// 32, else the smallest of those that covers B's mean row length.
static int copies_group(int group, long long nB, long long nnzB) {
    if (group == 8 || group == 16 || group == 32) return group;
    const double avg = nB > 0 ? (double)nnzB / (double)nB : 0.0;
    return avg <= 8.0 ? 8 : (avg <= 16.0 ? 16 : 32);
}

// Whether B is dense enough for the dense-B form (plus-times, 64 < d <= 256):
// the density above which it beat the sparse numeric pass on R-MAT scale-20
// products (edge factor 16) on GB300, per width of the accumulator.
static bool dense_b_auto(bool vals, long long d, long long nB, long long nnzB) {
    const long long dpad = round_up(d, 32);
    if (!vals || dpad <= 64 || dpad > 256 || nB <= 0) return false;
    const double permille = dpad <= 128 ? 600.0 : 450.0;
    return (double)nnzB * 1000.0 >= permille * (double)nB * (double)d;
}

static ts_status resolve_tuning(long long d, const ts_tuning& force, ts_tuning& t,
                                long long nB = 0, long long nnzB = 0, bool vals = false) {
    const long long dpad = round_up(d, 32);
    t = ts_tuning{};
    t.accum = force.accum ? force.accum
                          : (dense_b_auto(vals, d, nB, nnzB) ? TS_ACC_DENSE_B
                                                              : (dpad <= 4096 ? TS_ACC_DENSE : TS_ACC_HASH));
    t.col_tile = force.col_tile ? force.col_tile : (int)std::min<long long>(dpad, 1024);
    t.cta_min_flops = force.cta_min_flops ? force.cta_min_flops : 4096;
    t.warps_per_cta = force.warps_per_cta ? force.warps_per_cta : 8;
    t.hash_slots = force.hash_slots ? force.hash_slots : 1024;
    t.group = force.group ? force.group : auto_group(nB, nnzB, 0);
    t.sym_group = force.sym_group ? force.sym_group : auto_group(nB, nnzB, 1);
    t.bwd_group = force.bwd_group ? force.bwd_group : auto_group(nB, nnzB, 2);
    t.stage = force.stage ? force.stage : 2;
    t.pack_b = force.pack_b ? force.pack_b : 1;
    // row groups of 8 lanes (pairs) where four rows' accumulators fit well
    // (one tile, W <= 256); one warp per light row otherwise
    t.row_lanes = force.row_lanes ? force.row_lanes : 0;
    t.dB_mode = force.dB_mode ? force.dB_mode : 1;
    if (t.dB_mode != 1 && t.dB_mode != 2) return fail(TS_ERR_INVALID_ARG, "tuning: dB_mode must be 1 or 2");
    if (t.stage != 1 && t.stage != 2) return fail(TS_ERR_INVALID_ARG, "tuning: stage must be 1 or 2");
    if (t.stage == 1) t.pack_b = 1;
    if (!valid_group(t.group) || !valid_group(t.sym_group) || !valid_group(t.bwd_group))
        return fail(TS_ERR_INVALID_ARG, "tuning: group, sym_group and bwd_group must be 1, 2, 4, 8, 16 or 32");
    if (t.pack_b != 1 && t.pack_b != 2) return fail(TS_ERR_INVALID_ARG, "tuning: pack_b must be 1 or 2");
    if (t.row_lanes != 0 && t.row_lanes != 1 && t.row_lanes != 4 && t.row_lanes != 8 && t.row_lanes != 16 &&
        t.row_lanes != 32)
        return fail(TS_ERR_INVALID_ARG, "tuning: row_lanes must be 1, 4, 8, 16 or 32");
    if (t.accum != TS_ACC_DENSE && t.accum != TS_ACC_HASH && t.accum != TS_ACC_COPIES && t.accum != TS_ACC_DENSE_B)
        return fail(TS_ERR_INVALID_ARG,
                    "tuning: accum must be TS_ACC_DENSE, TS_ACC_HASH, TS_ACC_COPIES or TS_ACC_DENSE_B");
    if (t.accum == TS_ACC_DENSE_B && dpad > 256)
        return fail(TS_ERR_INVALID_ARG, "tuning: TS_ACC_DENSE_B needs d <= 256");
    if (t.accum == TS_ACC_COPIES && dpad > 4096)
        return fail(TS_ERR_INVALID_ARG, "tuning: TS_ACC_COPIES needs d <= 4096");
    if (t.col_tile < 32 || t.col_tile % 32 || t.col_tile > 4096)
        return fail(TS_ERR_INVALID_ARG, "tuning: col_tile must be a multiple of 32 in [32, 4096]");
    if (t.col_tile > dpad) t.col_tile = (int)dpad;
    // row groups only for a single tile of at most 256 columns: over several
    // tiles B's segments are short and one warp per light row is faster
    // wide rows (one tile of 256 < W <= 1024 columns): one shared accumulator
    // per warp with occupancy bits, so that A is walked once and only the
    // occupied columns are read out
    const bool one_tile = t.col_tile >= dpad;
    if (t.row_lanes == 0) {
        if (one_tile && t.col_tile <= 256) t.row_lanes = 8;
        else if (one_tile && t.col_tile <= 1024) t.row_lanes = 1;
        else t.row_lanes = 32;
    }
    if (t.row_lanes == 1 && !(one_tile && t.col_tile <= 1024))
        return fail(TS_ERR_INVALID_ARG, "tuning: row_lanes = 1 needs one column tile of at most 1024 columns");
    if (t.cta_min_flops < 1) return fail(TS_ERR_INVALID_ARG, "tuning: cta_min_flops must be >= 1");
    if (t.warps_per_cta < 1 || t.warps_per_cta > 8)
        return fail(TS_ERR_INVALID_ARG, "tuning: warps_per_cta must be in [1, 8]");
    if (t.hash_slots < 64 || (t.hash_slots & (t.hash_slots - 1)) || t.hash_slots > 8192)
        return fail(TS_ERR_INVALID_ARG, "tuning: hash_slots must be a power of two in [64, 8192]");
    return TS_OK;
}

struct Layout {
    size_t hdr = 0, flops = 0, perm = 0, partial = 0, items = 0, blen = 0, tp = 0, bpk = 0, bq = 0, denseb = 0,
           bt = 0, total = 0;
    size_t split_rows = 0, split_done = 0, split_items = 0, stg_bits = 0, stg_vals = 0, stg_flags = 0;
    int dw = 0, dpad = 0;
    int W = 0, T = 1;
};

// Workspace layout for tuning t.  With `cover_autotune`, the column-tile and
// packed-B regions are sized for every tuning the autotuner may try (tiles
// of at least max(64, d/8) columns, packing on), so that one workspace
// serves the whole search.
static Layout plan_layout(long long n, long long d, const ts_tuning& t, long long nnzA, long long nnzB,
                          bool cover_autotune = false) {
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    L.hdr = take(sizeof(WsHeader));
    L.flops = take(sizeof(long long) * (size_t)n);
    L.perm = take(sizeof(int) * (size_t)n);
    L.partial = take(sizeof(long long) * scan_partial_count(n));
    L.items = take(sizeof(long long) * (size_t)flops_item_capacity(n, nnzA));
    L.blen = take(sizeof(int) * (size_t)n);  // B has n rows
    L.dw = (int)((d + 31) / 32);
    L.dpad = 32 * L.dw;
    L.split_rows = take(sizeof(int) * MAX_SPLIT_ROWS);
    L.split_done = take(sizeof(int) * MAX_SPLIT_ROWS);
    L.split_items = take(sizeof(long long) * (size_t)split_item_capacity(nnzA));
    L.stg_bits = take(sizeof(unsigned) * (size_t)MAX_SPLIT_ROWS * L.dw);
    if (L.dpad <= 4096) {  // dense accumulators only
        L.stg_vals = take(sizeof(float) * (size_t)MAX_SPLIT_ROWS * L.dpad);
        L.stg_flags = take((size_t)MAX_SPLIT_ROWS * L.dpad);
    }
    L.W = t.col_tile;
    L.T = (int)((d + L.W - 1) / L.W);
    if (L.T < 1) L.T = 1;
    int Tmax = (t.accum != TS_ACC_HASH) ? L.T : 1;
    if (cover_autotune) {
        const long long dpad = round_up(d, 32);
        const long long wmin = std::max<long long>(64, round_up(dpad / 8, 32));
        Tmax = std::max<int>(Tmax, (int)((d + wmin - 1) / wmin));
    }
    if (Tmax > 1) L.tp = take(sizeof(long long) * (size_t)n * (Tmax + 1));
    // packed B, padded by four entries for the 16-byte loads of whole quads
    if (t.pack_b == 1 || cover_autotune) L.bpk = take(8 * ((size_t)nnzB + 4));
    // row-aligned packed B for the row-group numeric kernels (one column tile)
    if ((t.pack_b == 1 && L.T == 1 && t.row_lanes != 32) || cover_autotune) L.bq = take(padded_b_bytes(n, nnzB, d, 4));
    // dense copy of B and its pattern bitmap (dense-B form only)
    if (t.accum == TS_ACC_DENSE_B) L.denseb = take(dense_b_bytes(n, d));
    // the deterministic dB's transpose, chunk offsets and partial sums
    // (covered for the autotuner too, which may try it)
    if (t.dB_mode == 2 || cover_autotune) L.bt = take(backward_t_bytes(n, nnzA, nnzB, d));
    L.total = off;
    return L;
}

static Sched carve(void* ws, const Layout& L) {
    char* b = (char*)ws;
    Sched s;
    s.hdr = (WsHeader*)(b + L.hdr);
    s.flops = (long long*)(b + L.flops);
    s.perm = (int*)(b + L.perm);
    s.partial = (long long*)(b + L.partial);
    s.items = (long long*)(b + L.items);
    s.blen = (int*)(b + L.blen);
    s.split_rows = (int*)(b + L.split_rows);
    s.split_done = (int*)(b + L.split_done);
    s.split_items = (long long*)(b + L.split_items);
    s.stg_bits = (unsigned*)(b + L.stg_bits);
    s.stg_vals = L.stg_vals ? (float*)(b + L.stg_vals) : nullptr;
    s.stg_flags = L.stg_flags ? (unsigned char*)(b + L.stg_flags) : nullptr;
    s.dw = L.dw;
    s.dpad = L.dpad;
    return s;
}

static LaunchCfg cfg_of(const ts_tuning& t) {
    LaunchCfg c;
    c.warps_per_cta = t.warps_per_cta;
    c.cta_class = cta_class_of(t.cta_min_flops);
    c.sms = sm_count();
    c.group = t.group;
    c.row_lanes = t.row_lanes;
    return c;
}

extern "C" ts_status ts_plan_create(const ts_csr_desc* A, const ts_csr_desc* B, int32_t semiring,
                                    const ts_tuning* force, ts_plan** out) {
    if (!out) return fail(TS_ERR_INVALID_ARG, "ts_plan_create: out is NULL");
    *out = nullptr;
    if (semiring != TS_SR_PLUS_TIMES_F32 && semiring != TS_SR_OR_SELECT2ND_BOOL)
        return fail(TS_ERR_INVALID_ARG, "ts_plan_create: unknown semiring %d", semiring);
    if (!A || !B) return fail(TS_ERR_INVALID_ARG, "ts_plan_create: A or B is NULL");
    if (A->nrows < 0 || A->ncols != A->nrows)
        return fail(TS_ERR_INVALID_ARG, "ts_plan_create: A must be square (got %lld x %lld)",
                    (long long)A->nrows, (long long)A->ncols);
    if (B->nrows != A->ncols)
        return fail(TS_ERR_INVALID_ARG, "ts_plan_create: B has %lld rows, A has %lld columns",
                    (long long)B->nrows, (long long)A->ncols);
    if (B->ncols < 1) return fail(TS_ERR_INVALID_ARG, "ts_plan_create: B needs d >= 1 columns");
    if (B->ncols > MAX_D)
        return fail(TS_ERR_UNSUPPORTED, "ts_plan_create: d = %lld above the supported %lld",
                    (long long)B->ncols, MAX_D);
    if (A->nrows > INT32_MAX) return fail(TS_ERR_UNSUPPORTED, "ts_plan_create: n >= 2^31");
    ts_plan* p = new ts_plan;
    p->n = A->nrows;
    p->d = B->ncols;
    p->nnzA = A->nnz;
    p->nnzB = B->nnz;
    p->semiring = semiring;
    if (force) p->force = *force;
    ts_status s = resolve_tuning(p->d, p->force, p->cur, p->n, p->nnzB, semiring == TS_SR_PLUS_TIMES_F32);
    if (s != TS_OK) {
        delete p;
        return s;
    }
    *out = p;
    return ok();
}

extern "C" ts_status ts_plan_destroy(ts_plan* plan) {
    delete plan;
    return ok();
}

extern "C" ts_status ts_plan_get_tuning(const ts_plan* plan, ts_tuning* out) {
    if (!plan || !out) return fail(TS_ERR_INVALID_ARG, "ts_plan_get_tuning: NULL argument");
    *out = plan->cur;
    return ok();
}

extern "C" ts_status ts_plan_set_tuning(ts_plan* plan, const ts_tuning* tuning) {
    if (!plan || !tuning) return fail(TS_ERR_INVALID_ARG, "ts_plan_set_tuning: NULL argument");
    ts_tuning merged = *tuning, t;
    ts_status s = resolve_tuning(plan->d, merged, t, plan->n, plan->nnzB, plan->semiring == TS_SR_PLUS_TIMES_F32);
    if (s != TS_OK) return s;
    plan->cur = t;
    return ok();
}

extern "C" ts_status ts_workspace_size(const ts_plan* plan, size_t* bytes) {
    if (!plan || !bytes) return fail(TS_ERR_INVALID_ARG, "ts_workspace_size: NULL argument");
    *bytes = plan_layout(plan->n, plan->d, plan->cur, plan->nnzA, plan->nnzB,
                         plan->semiring == TS_SR_PLUS_TIMES_F32).total;
    return ok();
}

namespace ts {
// Workspace of the symbolic and numeric passes under the plan's current
// tuning (no autotuner regions); used by ts_spgemm_forward_noalloc.
size_t forward_workspace_bytes(const ts_plan* plan) {
    return plan_layout(plan->n, plan->d, plan->cur, plan->nnzA, plan->nnzB).total;
}
}  // namespace ts

static ts_status check_operands(const ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                void* ws, size_t ws_bytes, const Layout& L, const char* fn) {
    if (!plan) return fail(TS_ERR_INVALID_ARG, "%s: plan is NULL", fn);
    const bool vals = plan->semiring == TS_SR_PLUS_TIMES_F32;
    ts_status s;
    if ((s = check_desc(A, "A", vals)) != TS_OK) return s;
    if ((s = check_desc(B, "B", vals)) != TS_OK) return s;
    if (A->nrows != plan->n || A->ncols != plan->n || B->nrows != plan->n || B->ncols != plan->d)
        return fail(TS_ERR_INVALID_ARG, "%s: shapes differ from the plan's (n=%lld, d=%lld)", fn,
                    plan->n, plan->d);
    if (!ws && L.total) return fail(TS_ERR_INVALID_ARG, "%s: workspace is NULL", fn);
    if (ws_bytes < L.total)
        return fail(TS_ERR_WORKSPACE_TOO_SMALL, "%s: workspace of %zu bytes, %zu needed", fn,
                    ws_bytes, L.total);
    if (((uintptr_t)ws) & 255) return fail(TS_ERR_INVALID_ARG, "%s: workspace not 256-byte aligned", fn);
    return TS_OK;
}

static bool same_operands(const ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B, void* ws) {
    return plan->sym_valid && plan->sym_ws == ws && plan->sym_ptrs[0] == A->rowptr &&
           plan->sym_ptrs[1] == A->col && plan->sym_ptrs[2] == B->rowptr &&
           plan->sym_ptrs[3] == B->col && plan->sym_nnz[0] == A->nnz && plan->sym_nnz[1] == B->nnz;
}

static ts_status read_errors(void* ws, const Layout& L, cudaStream_t st, const char* fn) {
    unsigned long long err = 0;
    WsHeader* h = (WsHeader*)((char*)ws + L.hdr);
    TS_CUDA(cudaMemcpyAsync(&err, &h->err, sizeof err, cudaMemcpyDeviceToHost, st), fn);
    TS_CUDA(cudaStreamSynchronize(st), fn);
    if (err)
        return fail(TS_ERR_BAD_CSR, "%s: device checks failed (flags 0x%llx: %s%s%s%s)", fn, err,
                    (err & ERR_A_COL) ? "column of A out of range; " : "",
                    (err & ERR_B_COL) ? "column of B out of range; " : "",
                    (err & ERR_C_ROW) ? "C row does not match its rowptr; " : "",
                    (err & ERR_HASH_FULL) ? "hash table overflow; " : "");
    return TS_OK;
}

extern "C" ts_status ts_spgemm_symbolic(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                        int64_t* C_rowptr, int64_t* nnzC_host, void* ws,
                                        size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("ts_spgemm_symbolic");
    const char* fn = "ts_spgemm_symbolic";
    if (!plan) return fail(TS_ERR_INVALID_ARG, "%s: plan is NULL", fn);
    const Layout L = plan_layout(plan->n, plan->d, plan->cur, A ? A->nnz : plan->nnzA, B ? B->nnz : plan->nnzB);
    ts_status s = check_operands(plan, A, B, ws, ws_bytes, L, fn);
    if (s != TS_OK) return s;
    if (!C_rowptr) return fail(TS_ERR_INVALID_ARG, "%s: C_rowptr is NULL", fn);
    cudaStream_t st = (cudaStream_t)stream;
    const Sched sc = carve(ws, L);
    const DevCsr dA = dev(A), dB = dev(B);
    plan->sym_valid = false;
    {
        NvtxRange r("row flops and classes");
        TS_CUDA(launch_row_schedule(dA, dB, sc, (long long*)C_rowptr, st), fn);
    }
    LaunchCfg scfg = cfg_of(plan->cur);
    scfg.group = plan->cur.sym_group;
    {
        NvtxRange r("row counts and scan");
        TS_CUDA(launch_symbolic(dA, dB, plan->d, sc, scfg, (long long*)C_rowptr, st), fn);
    }
    plan->sym_valid = true;
    plan->sym_ws = ws;
    plan->sym_ptrs[0] = A->rowptr;
    plan->sym_ptrs[1] = A->col;
    plan->sym_ptrs[2] = B->rowptr;
    plan->sym_ptrs[3] = B->col;
    plan->sym_nnz[0] = A->nnz;
    plan->sym_nnz[1] = B->nnz;
    if (nnzC_host) {
        long long tot = 0;
        TS_CUDA(cudaMemcpyAsync(&tot, (long long*)C_rowptr + plan->n, sizeof tot,
                                cudaMemcpyDeviceToHost, st), fn);
        s = read_errors(ws, L, st, fn);
        if (s != TS_OK) return s;
        if (tot > INT32_MAX * 64LL) return fail(TS_ERR_OVERFLOW, "%s: nnz(C) = %lld", fn, tot);
        *nnzC_host = tot;
    }
    return ok();
}

extern "C" ts_status ts_workspace_check(const ts_plan* plan, void* ws, size_t ws_bytes, void* stream) {
    if (!plan || !ws) return fail(TS_ERR_INVALID_ARG, "ts_workspace_check: NULL argument");
    const Layout L = plan_layout(plan->n, plan->d, plan->cur, plan->nnzA, plan->nnzB);
    if (ws_bytes < sizeof(WsHeader)) return fail(TS_ERR_WORKSPACE_TOO_SMALL, "ts_workspace_check");
    ts_status s = read_errors(ws, L, (cudaStream_t)stream, "ts_workspace_check");
    return s == TS_OK ? ok() : s;
}

static ts_status run_numeric(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                             const ts_csr_desc* C, void* ws, const Layout& L, cudaStream_t st,
                             const char* fn) {
    const bool vals = plan->semiring == TS_SR_PLUS_TIMES_F32;
    const Sched sc = carve(ws, L);
    const DevCsr dA = dev(A), dB = dev(B);
    const LaunchCfg cfg = cfg_of(plan->cur);
    if (plan->cur.accum == TS_ACC_DENSE_B && vals) {
        TS_CUDA(launch_numeric_denseb(dA, dB, plan->d, sc, cfg, (const long long*)C->rowptr, C->col, (float*)C->val,
                                      C->nnz, (char*)ws + L.denseb, st),
                fn);
    } else if (plan->cur.accum == TS_ACC_DENSE || plan->cur.accum == TS_ACC_COPIES ||
               plan->cur.accum == TS_ACC_DENSE_B) {
        long long* tp = nullptr;
        if (L.T > 1) {
            tp = (long long*)((char*)ws + L.tp);
            TS_CUDA(launch_tile_split(dB, L.W, L.T, tp, st), fn);
        }
        const int cg = copies_group(plan->cur.group, plan->n, plan->nnzB);
        const bool copies = vals && plan->cur.accum == TS_ACC_COPIES &&
                            numeric_copies_smem(L.W, cg, cfg.warps_per_cta) <= 227 * 1024;
        const bool staged = !copies && plan->cur.stage == 1 &&
                            numeric_staged_smem(L.W, cfg.warps_per_cta, vals) <= 227 * 1024;
        // the row-group kernels over one column tile read the row-aligned copy
        const int qE = cfg.row_lanes == 4 ? 4 : 2;
        const bool use_bq = !copies && !staged && vals && plan->cur.pack_b == 1 && L.T == 1 && L.bq &&
                            B->nnz > 0 && cfg.row_lanes != 32 &&
                            numeric_rgcta_smem(L.W, cfg.warps_per_cta, cfg.row_lanes) <= 220 * 1024 &&
                            padded_b_fits(B->nrows, B->nnz, plan->d, qE);
        int2* bpk = nullptr;
        int4* bq = nullptr;
        if (use_bq) {
            bq = (int4*)((char*)ws + L.bq);
            TS_CUDA(launch_pack_b_rows(dB, qE, plan->d, bq, &sc.hdr->err, st), fn);
        } else if (vals && plan->cur.pack_b == 1 && B->nnz > 0) {
            bpk = (int2*)((char*)ws + L.bpk);
            TS_CUDA(launch_pack_b(dB, bpk, st), fn);
        }
        if (copies) {
            // light rows in row groups behind the copies kernel when they fit
            const bool rg = cfg.row_lanes != 32 && cfg.row_lanes != 1 && bpk &&
                            numeric_light_smem(L.W, cfg.warps_per_cta, cfg.row_lanes) <= 220 * 1024;
            TS_CUDA(launch_numeric_copies(dA, dB, plan->d, L.W, L.T, tp, bpk, cg, sc, cfg,
                                          (const long long*)C->rowptr, C->col, (float*)C->val, C->nnz, st, rg),
                    fn);
            if (rg)
                TS_CUDA(launch_numeric_light_rows(dA, dB, plan->d, L.W, L.T, tp, bpk, sc, cfg,
                                                  (const long long*)C->rowptr, C->col, (float*)C->val, C->nnz, st),
                        fn);
        } else if (staged && (!vals || bpk || B->nnz == 0)) {
            TS_CUDA(launch_numeric_staged(dA, dB, plan->d, L.W, L.T, tp, vals, bpk, sc, cfg, (const long long*)C->rowptr, C->col, (float*)C->val, C->nnz, st),
                    fn);
        } else {
            LaunchCfg ncfg = cfg;
            if (ncfg.row_lanes != 32 &&
                (!vals || !(bpk || bq) || numeric_rgcta_smem(L.W, cfg.warps_per_cta, ncfg.row_lanes) > 220 * 1024))
                ncfg.row_lanes = 32;  // row groups need a packed copy and room for their accumulators
            TS_CUDA(launch_numeric_dense(dA, dB, plan->d, L.W, L.T, tp, vals, bpk, plan->cur.group, sc, ncfg,
                                         (const long long*)C->rowptr, C->col, (float*)C->val, C->nnz, st, bq),
                    fn);
        }
    } else {
        TS_CUDA(launch_numeric_hash(dA, dB, plan->d, plan->cur.hash_slots, vals, sc, cfg,
                                    (const long long*)C->rowptr, C->col, (float*)C->val, C->nnz, st),
                fn);
    }
    return TS_OK;
}

extern "C" ts_status ts_spgemm_numeric(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                       const ts_csr_desc* C, void* ws, size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("ts_spgemm_numeric");
    const char* fn = "ts_spgemm_numeric";
    if (!plan) return fail(TS_ERR_INVALID_ARG, "%s: plan is NULL", fn);
    const Layout L = plan_layout(plan->n, plan->d, plan->cur, A ? A->nnz : plan->nnzA, B ? B->nnz : plan->nnzB);
    ts_status s = check_operands(plan, A, B, ws, ws_bytes, L, fn);
    if (s != TS_OK) return s;
    const bool vals = plan->semiring == TS_SR_PLUS_TIMES_F32;
    if ((s = check_desc(C, "C", vals)) != TS_OK) return s;
    if (C->nrows != plan->n || C->ncols != plan->d)
        return fail(TS_ERR_INVALID_ARG, "%s: C must be %lld x %lld", fn, plan->n, plan->d);
    if (!same_operands(plan, A, B, ws))
        return fail(TS_ERR_STATE, "%s: no symbolic pass on this plan with these A, B and workspace", fn);
    s = run_numeric(plan, A, B, C, ws, L, (cudaStream_t)stream, fn);
    return s == TS_OK ? ok() : s;
}

static ts_status run_backward(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                              const ts_csr_desc* C, const float* dC, float* dA, float* dB, void* ws,
                              size_t ws_bytes, void* stream, const char* fn) {
    NvtxRange nvtx_range("ts_spgemm_backward");
    if (!plan) return fail(TS_ERR_INVALID_ARG, "%s: plan is NULL", fn);
    if (plan->semiring != TS_SR_PLUS_TIMES_F32)
        return fail(TS_ERR_UNSUPPORTED, "%s: the boolean semiring has no gradient", fn);
    const Layout L = plan_layout(plan->n, plan->d, plan->cur, A ? A->nnz : plan->nnzA, B ? B->nnz : plan->nnzB);
    ts_status s = check_operands(plan, A, B, ws, ws_bytes, L, fn);
    if (s != TS_OK) return s;
    if (!C || !C->rowptr || (C->nnz > 0 && (!C->col || !dC)))
        return fail(TS_ERR_INVALID_ARG, "%s: C pattern or dC is NULL", fn);
    if (C->nrows != plan->n || C->ncols != plan->d || C->nnz < 0)
        return fail(TS_ERR_INVALID_ARG, "%s: C must be %lld x %lld", fn, plan->n, plan->d);
    if (!same_operands(plan, A, B, ws))
        return fail(TS_ERR_STATE, "%s: no symbolic pass on this plan with these A, B and workspace", fn);
    if (plan->d > 8192) return fail(TS_ERR_UNSUPPORTED, "%s: backward supports d <= 8192", fn);
    const Sched sc = carve(ws, L);
    int2* bpk = nullptr;
    if (plan->cur.pack_b == 1 && B->nnz > 0) {
        bpk = (int2*)((char*)ws + L.bpk);
        TS_CUDA(launch_pack_b(dev(B), bpk, (cudaStream_t)stream), fn);
    }
    LaunchCfg bcfg = cfg_of(plan->cur);
    bcfg.group = plan->cur.bwd_group;
    if (bcfg.group == 2 && (!bpk || (reinterpret_cast<uintptr_t>(dB) & 15))) bcfg.group = 16;  // no quads
    // option T: dA from the kernels (dB skipped), dB by the ordered pull
    const bool det = plan->cur.dB_mode == 2 && dB && L.bt;
    TS_CUDA(launch_backward(dev(A), dev(B), plan->d, (const long long*)C->rowptr, C->col, C->nnz, dC,
                            dA, det ? nullptr : dB, bpk, sc, bcfg, (cudaStream_t)stream),
            fn);
    if (det)
        TS_CUDA(launch_backward_t(dev(A), dev(B), plan->d, (const long long*)C->rowptr, C->col, C->nnz, dC, dB,
                                  (char*)ws + L.bt, sc.hdr, (cudaStream_t)stream),
                fn);
    return ok();
}

extern "C" ts_status ts_spgemm_backward(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                        const ts_csr_desc* C, const float* dC_val, float* dA_val,
                                        float* dB_val, void* ws, size_t ws_bytes, void* stream) {
    return run_backward(plan, A, B, C, dC_val, dA_val, dB_val, ws, ws_bytes, stream,
                        "ts_spgemm_backward");
}

extern "C" ts_status ts_spgemm_backward_dA(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                           const ts_csr_desc* C, const float* dC_val, float* dA_val,
                                           void* ws, size_t ws_bytes, void* stream) {
    if (!dA_val) return fail(TS_ERR_INVALID_ARG, "ts_spgemm_backward_dA: dA_val is NULL");
    return run_backward(plan, A, B, C, dC_val, dA_val, nullptr, ws, ws_bytes, stream,
                        "ts_spgemm_backward_dA");
}

extern "C" ts_status ts_spgemm_backward_dB(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                           const ts_csr_desc* C, const float* dC_val, float* dB_val,
                                           void* ws, size_t ws_bytes, void* stream) {
    if (!dB_val) return fail(TS_ERR_INVALID_ARG, "ts_spgemm_backward_dB: dB_val is NULL");
    return run_backward(plan, A, B, C, dC_val, nullptr, dB_val, ws, ws_bytes, stream,
                        "ts_spgemm_backward_dB");
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
extern "C" ts_status ts_plan_autotune(ts_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                      const ts_csr_desc* C, const float* dC_val, float* dA_scratch,
                                      float* dB_scratch, int32_t reps, ts_tuning* chosen, void* ws,
                                      size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("ts_plan_autotune");
    const char* fn = "ts_plan_autotune";
    if (!plan) return fail(TS_ERR_INVALID_ARG, "%s: plan is NULL", fn);
    if (reps < 1) return fail(TS_ERR_INVALID_ARG, "%s: reps must be >= 1", fn);
    const Layout L0 = plan_layout(plan->n, plan->d, plan->cur, A ? A->nnz : plan->nnzA, B ? B->nnz : plan->nnzB);
    ts_status s = check_operands(plan, A, B, ws, ws_bytes, L0, fn);
    if (s != TS_OK) return s;
    if (!same_operands(plan, A, B, ws))
        return fail(TS_ERR_STATE, "%s: run ts_spgemm_symbolic on this plan and workspace first", fn);
    const bool vals = plan->semiring == TS_SR_PLUS_TIMES_F32;
    if ((s = check_desc(C, "C", vals)) != TS_OK) return s;
    const bool do_bwd = vals && dC_val && (dA_scratch || dB_scratch) && plan->d <= 8192;
    cudaStream_t st = (cudaStream_t)stream;
    const long long dpad = round_up(plan->d, 32);

    // coordinate descent from the heuristic default: each field in turn takes
    // the value that times fastest with the others fixed; fields fixed by the
    // plan's `force` are not varied
    // errors the symbolic pass found in the operands end the search at once;
    // after that the error word is cleared before every trial and read after
    // it, so that a candidate whose kernels flagged a failure (a hash table
    // too small for a row, which skips the row and so also times faster) is
    // dropped instead of chosen, and does not fail the final check
    s = read_errors(ws, L0, st, fn);
    if (s != TS_OK) return s;
    unsigned long long* err_word = &((WsHeader*)((char*)ws + L0.hdr))->err;
    cudaEvent_t e0, e1;
    TS_CUDA(cudaEventCreate(&e0), fn);
    TS_CUDA(cudaEventCreate(&e1), fn);
    const ts_tuning saved = plan->cur;
    ts_tuning best = saved;
    float best_ms = 1e30f;
    auto try_one = [&](const ts_tuning& cand_in) -> ts_status {
        ts_tuning cand;
        if (resolve_tuning(plan->d, cand_in, cand, plan->n, B->nnz, vals) != TS_OK) return TS_OK;  // skip
        const Layout L = plan_layout(plan->n, plan->d, cand, A->nnz, B->nnz);
        if (L.total > ws_bytes) return TS_OK;  // does not fit the caller's workspace
        plan->cur = cand;
        TS_CUDA(cudaMemsetAsync(err_word, 0, sizeof *err_word, st), fn);
        float tot = 0.0f;
        for (int r = 0; r <= reps; ++r) {  // the first run warms up
            TS_CUDA(cudaEventRecord(e0, st), fn);
            ts_status q = run_numeric(plan, A, B, C, ws, L, st, fn);
            if (q != TS_OK) return q;
            if (do_bwd) {
                q = run_backward(plan, A, B, C, dC_val, dA_scratch, dB_scratch, ws, ws_bytes, stream, fn);
                if (q != TS_OK) return q;
            }
            TS_CUDA(cudaEventRecord(e1, st), fn);
            TS_CUDA(cudaEventSynchronize(e1), fn);
            float ms = 0.0f;
            TS_CUDA(cudaEventElapsedTime(&ms, e0, e1), fn);
            if (r > 0) tot += ms;
        }
        unsigned long long err = 0;
        TS_CUDA(cudaMemcpyAsync(&err, err_word, sizeof err, cudaMemcpyDeviceToHost, st), fn);
        TS_CUDA(cudaStreamSynchronize(st), fn);
        if (err) return TS_OK;  // this candidate cannot run the product: skip it
        const float avg = tot / reps;
        if (avg < best_ms) {
            best_ms = avg;
            best = cand;
        }
        return TS_OK;
    };
    s = try_one(best);
    std::vector<int> tiles;
    for (int w : {64, 128, 256, 512, 1024, 2048, 4096})
        if (w <= dpad && w >= std::max<long long>(64, round_up(dpad / 8, 32))) tiles.push_back(w);
    if (tiles.empty() || tiles.back() < std::min<long long>(dpad, 4096))
        tiles.push_back((int)std::min<long long>(dpad, 4096));
    for (int field = 0; field < 10 && s == TS_OK; ++field) {
        std::vector<ts_tuning> cands;
        ts_tuning c = best;
        switch (field) {
            case 0:
                if (plan->force.group) break;
                for (int g : {1, 4, 8, 16, 32}) { c.group = g; cands.push_back(c); }
                break;
            case 1:
                if (plan->force.pack_b || !vals) break;
                for (int pk : {1, 2}) { c.pack_b = pk; cands.push_back(c); }
                break;
            case 2:
                if (plan->force.accum) break;
                for (int acc : {TS_ACC_DENSE, TS_ACC_COPIES, TS_ACC_HASH, TS_ACC_DENSE_B}) {
                    if (acc == TS_ACC_HASH && plan->d <= 256) continue;
                    if (acc == TS_ACC_COPIES && (!vals || dpad > 4096)) continue;
                    if (acc == TS_ACC_DENSE_B && (!vals || dpad > 256)) continue;
                    c.accum = acc;
                    cands.push_back(c);
                }
                break;
            case 3:
                if (plan->force.col_tile || best.accum == TS_ACC_HASH) break;
                for (int w : tiles) { c.col_tile = w; cands.push_back(c); }
                break;
            case 4:
                if (plan->force.cta_min_flops) break;
                for (long long th : {1024LL, 4096LL, 16384LL, 65536LL}) { c.cta_min_flops = th; cands.push_back(c); }
                break;
            case 5:
                if (plan->force.warps_per_cta) break;
                for (int w : {2, 4, 8}) { c.warps_per_cta = w; cands.push_back(c); }
                break;
            case 7:
                if (plan->force.bwd_group || !do_bwd) break;
                for (int g : {1, 2, 8, 16, 32}) { c.bwd_group = g; cands.push_back(c); }
                break;
            case 9:
                if (plan->force.dB_mode || !do_bwd) break;
                for (int m : {1, 2}) { c.dB_mode = m; cands.push_back(c); }
                break;
            case 8:
                if (plan->force.row_lanes || !vals) break;
                for (int rl : {32, 4, 8, 16, 1}) {
                    if (rl == 1 && !(best.col_tile >= dpad && best.col_tile <= 1024)) continue;
                    c.row_lanes = rl;
                    cands.push_back(c);
                }
                break;
            case 6:
                if (plan->force.stage) break;
                for (int sg : {1, 2}) { c.stage = sg; c.pack_b = sg == 1 ? 1 : best.pack_b; cands.push_back(c); }
                break;
        }
        for (const ts_tuning& cand : cands) {
            s = try_one(cand);
            if (s != TS_OK) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != TS_OK) {
        plan->cur = saved;
        return s;
    }
    plan->cur = best;
    if (chosen) *chosen = best;
    // leave C holding the product of the chosen tuning
    const Layout Lb = plan_layout(plan->n, plan->d, best, A->nnz, B->nnz);
    TS_CUDA(cudaMemsetAsync(err_word, 0, sizeof *err_word, st), fn);
    s = run_numeric(plan, A, B, C, ws, Lb, st, fn);
    if (s != TS_OK) return s;
    s = read_errors(ws, Lb, st, fn);
    return s == TS_OK ? ok() : s;
}


// ---------------------------------------------------------------------------
// sparse Force2Vec minibatch step (paper Sec. IV, sparse embedding)
// ---------------------------------------------------------------------------
struct F2vLayout {
    Layout inner;  // schedule and SpGEMM regions for the b x n by n x d product
    size_t inner_off = 0, Wp = 0, Wcol = 0, Wmult = 0, Wrow = 0, Wval = 0, newmask = 0, Gp = 0, Gc = 0, Gv = 0;
    size_t Sc = 0, Sv = 0, total = 0;
    long long wcap = 0, gcap = 0;
};

static ts_tuning f2v_tuning(long long d, long long n, long long nnzZ) {
    ts_tuning t{};
    ts_tuning force{};
    force.col_tile = (int32_t)round_up(d, 32);  // one tile: G's rows are at most d wide
    resolve_tuning(d, force, t, n, nnzZ);
    return t;
}

static F2vLayout f2v_layout(long long n, long long d, long long nnzA, long long b, long long s, long long k) {
    F2vLayout F;
    F.wcap = nnzA + b * s;
    F.gcap = b * round_up(d, 32);
    const ts_tuning t = f2v_tuning(d, n, n * k);
    F.inner = plan_layout(n, d, t, F.wcap, n * k);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    F.inner_off = take(F.inner.total);
    F.Wp = take(sizeof(long long) * (size_t)(b + 1));
    F.Wcol = take(sizeof(int) * (size_t)F.wcap);
    F.Wmult = take(sizeof(int) * (size_t)F.wcap);
    F.Wrow = take(sizeof(int) * (size_t)F.wcap);
    F.Wval = take(sizeof(float) * (size_t)F.wcap);
    F.newmask = take(sizeof(unsigned) * (size_t)(b > 0 ? b : 1));
    F.Gp = take(sizeof(long long) * (size_t)(b + 1));
    F.Gc = take(sizeof(int) * (size_t)F.gcap);
    F.Gv = take(sizeof(float) * (size_t)F.gcap);
    F.Sc = take(sizeof(int) * (size_t)(b * k));
    F.Sv = take(sizeof(float) * (size_t)(b * k));
    F.total = off;
    return F;
}

extern "C" ts_status f2v_workspace_size(int64_t n, int64_t d, int64_t nnz_A, int64_t b, int32_t s, int32_t k,
                                        size_t* bytes) {
    if (!bytes || n < 0 || d < 1 || nnz_A < 0 || b < 0 || s < 0 || k < 1)
        return fail(TS_ERR_INVALID_ARG, "f2v_workspace_size: bad argument");
    if (d > 4096 || k > d || s > 32) return fail(TS_ERR_UNSUPPORTED, "f2v_workspace_size: need k <= d <= 4096, s <= 32");
    *bytes = f2v_layout(n, d, nnz_A, b, s, k).total;
    return ok();
}

extern "C" ts_status f2v_step(const ts_csr_desc* A, const ts_csr_desc* Z, int64_t r0, int64_t b,
                              const int32_t* neg, int32_t s, float lr, int32_t k, float* U_out, void* ws,
                              size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("f2v_step");
    const char* fn = "f2v_step";
    ts_status st_;
    if ((st_ = check_desc(A, "A", false)) != TS_OK) return st_;
    if ((st_ = check_desc(Z, "Z", true)) != TS_OK) return st_;
    const long long n = A->nrows, d = Z->ncols;
    if (A->ncols != n || Z->nrows != n) return fail(TS_ERR_INVALID_ARG, "%s: A must be n x n and Z n x d", fn);
    if (n > INT32_MAX) return fail(TS_ERR_UNSUPPORTED, "%s: n >= 2^31", fn);
    if (d > 4096 || k < 1 || k > d || s < 0 || s > 32)
        return fail(TS_ERR_UNSUPPORTED, "%s: need 1 <= k <= d <= 4096 and 0 <= s <= 32", fn);
    if (Z->nnz != n * (long long)k) return fail(TS_ERR_INVALID_ARG, "%s: Z must hold exactly k entries per row", fn);
    if (r0 < 0 || b < 0 || r0 + b > n) return fail(TS_ERR_INVALID_ARG, "%s: batch rows outside Z", fn);
    if (s > 0 && b > 0 && !neg) return fail(TS_ERR_INVALID_ARG, "%s: negatives are NULL", fn);
    const F2vLayout F = f2v_layout(n, d, A->nnz, b, s, k);
    if (!ws || ws_bytes < F.total)
        return fail(TS_ERR_WORKSPACE_TOO_SMALL, "%s: workspace of %zu bytes, %zu needed", fn, ws_bytes, F.total);
    if (((uintptr_t)ws) & 255) return fail(TS_ERR_INVALID_ARG, "%s: workspace not 256-byte aligned", fn);
    if (b == 0) return ok();
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)ws;
    const Sched sc = carve(w + F.inner_off, F.inner);
    long long* Wp = (long long*)(w + F.Wp);
    int* Wcol = (int*)(w + F.Wcol);
    int* Wmult = (int*)(w + F.Wmult);
    int* Wrow = (int*)(w + F.Wrow);
    float* Wval = (float*)(w + F.Wval);
    unsigned* newmask = (unsigned*)(w + F.newmask);
    long long* Gp = (long long*)(w + F.Gp);
    int* Gc = (int*)(w + F.Gc);
    float* Gv = (float*)(w + F.Gv);
    const ts_tuning t = f2v_tuning(d, n, n * k);
    const LaunchCfg cfg = cfg_of(t);
    const DevCsr dA = dev(A), dZ = dev(Z);
    // 1. W's pattern (neighbours and negatives merged) and the Z layout check
    TS_CUDA(cudaMemsetAsync(sc.hdr, 0, sizeof(WsHeader), st), fn);
    TS_CUDA(launch_f2v_check(dZ, k, sc.hdr, st), fn);
    TS_CUDA(launch_f2v_pattern(dA, r0, b, neg, s, Wp, newmask, sc.partial, sc.hdr, st), fn);
    TS_CUDA(launch_f2v_fill(dA, r0, b, neg, s, Wp, newmask, Wcol, Wmult, Wrow, st), fn);
    // 2. weights on W's pattern
    TS_CUDA(launch_f2v_weights(dZ, k, r0, b, Wp, Wcol, Wmult, Wrow, Wval, st), fn);
    // errors so far live in the header the schedule is about to reset
    unsigned long long err0 = 0;
    TS_CUDA(cudaMemcpyAsync(&err0, &sc.hdr->err, sizeof err0, cudaMemcpyDeviceToHost, st), fn);
    // 3. G = W * Z (b x n by n x d), the library's TS-SpGEMM passes
    DevCsr dW;
    dW.nrows = b;
    dW.ncols = n;
    dW.nnz = F.wcap;
    dW.rowptr = Wp;
    dW.col = Wcol;
    dW.val = Wval;
    TS_CUDA(launch_row_schedule(dW, dZ, sc, Gp, st), fn);
    LaunchCfg scfg = cfg;
    scfg.group = t.sym_group;
    TS_CUDA(launch_symbolic(dW, dZ, d, sc, scfg, Gp, st), fn);
    int2* bpk = (int2*)((char*)(w + F.inner_off) + F.inner.bpk);
    TS_CUDA(launch_pack_b(dZ, bpk, st), fn);
    TS_CUDA(launch_numeric_dense(dW, dZ, d, F.inner.W, F.inner.T, nullptr, true, bpk, t.group, sc, cfg, Gp, Gc, Gv,
                                 F.gcap, st),
            fn);
    // 4-5. update, top-k, commit into Z's batch rows
    TS_CUDA(launch_f2v_update(dZ, k, r0, b, Gp, Gc, Gv, lr, U_out, (int*)(w + F.Sc), (float*)(w + F.Sv), cfg.sms,
                              sc.hdr, st),
            fn);
    unsigned long long err1 = 0;
    TS_CUDA(cudaMemcpyAsync(&err1, &sc.hdr->err, sizeof err1, cudaMemcpyDeviceToHost, st), fn);
    TS_CUDA(cudaStreamSynchronize(st), fn);
    if (err0 | err1)
        return fail(TS_ERR_BAD_CSR, "%s: device checks failed (flags 0x%llx)", fn, (unsigned long long)(err0 | err1));
    return ok();
}

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------
extern "C" size_t ts_validate_workspace_size(void) { return 256; }

extern "C" ts_status ts_csr_validate(const ts_csr_desc* M, int64_t* bad_row, void* ws, size_t ws_bytes,
                                     void* stream) {
    NvtxRange nvtx_range("ts_csr_validate");
    const char* fn = "ts_csr_validate";
    ts_status s = check_desc(M, "M", false);
    if (s != TS_OK) return s;
    if (!ws || ws_bytes < ts_validate_workspace_size())
        return fail(TS_ERR_WORKSPACE_TOO_SMALL, "%s: needs %zu bytes of workspace", fn,
                    ts_validate_workspace_size());
    cudaStream_t st = (cudaStream_t)stream;
    long long bad = -1;
    TS_CUDA(launch_validate(dev(M), (long long*)ws, st), fn);
    TS_CUDA(cudaMemcpyAsync(&bad, ws, sizeof bad, cudaMemcpyDeviceToHost, st), fn);
    TS_CUDA(cudaStreamSynchronize(st), fn);
    if (bad_row) *bad_row = bad;
    if (bad != -1) return fail(TS_ERR_BAD_CSR, "%s: row %lld violates the CSR rules", fn, bad);
    return ok();
}

// ---------------------------------------------------------------------------
// multi-source BFS (paper Alg. 3)
// ---------------------------------------------------------------------------
static const long long MSBFS_MAX_D = 65536;

struct BfsLayout {
    size_t hdr = 0, flops = 0, perm = 0, partial = 0, items = 0, newbits = 0, blen = 0, fbits = 0, total = 0;
};

static BfsLayout bfs_layout(long long n, long long d, long long nnzA) {
    BfsLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    L.hdr = take(sizeof(WsHeader));
    L.flops = take(sizeof(long long) * (size_t)n);
    L.perm = take(sizeof(int) * (size_t)n);
    L.partial = take(sizeof(long long) * scan_partial_count(n));
    // newbits before items: msbfs_emit finds it without knowing nnz(A)
    L.newbits = take(sizeof(unsigned) * (size_t)n * (size_t)((d + 31) / 32));
    L.items = take(sizeof(long long) * (size_t)flops_item_capacity(n, nnzA));
    L.blen = take(sizeof(int) * (size_t)n);
    const int dwp = msbfs_pull_words((int)std::min<long long>(d, 1 << 20));
    if (dwp) L.fbits = take(sizeof(unsigned) * (size_t)n * (size_t)dwp);  // frontier bitmap, pull form
    L.total = off;
    return L;
}

extern "C" ts_status msbfs_workspace_size(int64_t n, int64_t nnz_A, int64_t d, size_t* bytes) {
    if (!bytes || n < 0 || nnz_A < 0 || d < 1)
        return fail(TS_ERR_INVALID_ARG, "msbfs_workspace_size: bad argument");
    if (d > MSBFS_MAX_D) return fail(TS_ERR_UNSUPPORTED, "msbfs: d above %lld", MSBFS_MAX_D);
    *bytes = bfs_layout(n, d, nnz_A).total;
    return ok();
}

extern "C" ts_status msbfs_init(int64_t n, int64_t d, const int32_t* sources_dev, uint32_t* visited,
                                int32_t* levels, const ts_csr_desc* F0, void* stream) {
    const char* fn = "msbfs_init";
    if (n < 0 || d < 1 || !sources_dev || !visited || !levels || !F0 || !F0->rowptr || !F0->col)
        return fail(TS_ERR_INVALID_ARG, "%s: NULL or negative argument", fn);
    if (n > INT32_MAX) return fail(TS_ERR_UNSUPPORTED, "%s: n >= 2^31", fn);
    if (d > MSBFS_MAX_D) return fail(TS_ERR_UNSUPPORTED, "%s: d above %lld", fn, MSBFS_MAX_D);
    if (F0->nrows != n || F0->ncols != d)
        return fail(TS_ERR_INVALID_ARG, "%s: F0 must be %lld x %lld", fn, (long long)n, (long long)d);
    if (F0->nnz < d) return fail(TS_ERR_CAPACITY, "%s: F0 needs room for %lld entries", fn, (long long)d);
    TS_CUDA(launch_msbfs_init(n, (int)d, sources_dev, visited, levels, (long long*)F0->rowptr, F0->col,
                              (cudaStream_t)stream),
            fn);
    return ok();
}

static ts_status bfs_step(const ts_csr_desc* A, const ts_csr_desc* F, uint32_t* visited, int32_t* levels,
                          int32_t* parents, int32_t level, const ts_csr_desc* F_next, int64_t F_next_capacity,
                          int64_t* nnz_next_host, void* ws, size_t ws_bytes, void* stream, const char* fn) {
    ts_status s;
    if ((s = check_desc(A, "A", false)) != TS_OK) return s;
    if ((s = check_desc(F, "F", false)) != TS_OK) return s;
    if (!F_next || !F_next->rowptr || !visited || !levels || !nnz_next_host)
        return fail(TS_ERR_INVALID_ARG, "%s: NULL argument", fn);
    const long long n = A->nrows, d = F->ncols;
    if (A->ncols != n || F->nrows != n || F_next->nrows != n || F_next->ncols != d)
        return fail(TS_ERR_INVALID_ARG, "%s: A must be n x n, F and F_next n x d", fn);
    if (d < 1 || d > MSBFS_MAX_D) return fail(TS_ERR_UNSUPPORTED, "%s: d must be in [1, %lld]", fn, MSBFS_MAX_D);
    if (F_next_capacity < 0 || (F_next_capacity > 0 && !F_next->col))
        return fail(TS_ERR_INVALID_ARG, "%s: bad F_next capacity", fn);
    const BfsLayout L = bfs_layout(n, d, A->nnz);
    if (!ws || ws_bytes < L.total)
        return fail(TS_ERR_WORKSPACE_TOO_SMALL, "%s: workspace of %zu bytes, %zu needed", fn, ws_bytes, L.total);
    if (((uintptr_t)ws) & 255) return fail(TS_ERR_INVALID_ARG, "%s: workspace not 256-byte aligned", fn);
    cudaStream_t st = (cudaStream_t)stream;
    char* b = (char*)ws;
    Sched sc;
    sc.hdr = (WsHeader*)(b + L.hdr);
    sc.flops = (long long*)(b + L.flops);
    sc.perm = (int*)(b + L.perm);
    sc.partial = (long long*)(b + L.partial);
    sc.items = (long long*)(b + L.items);
    sc.blen = (int*)(b + L.blen);
    unsigned* newbits = (unsigned*)(b + L.newbits);
    ts_tuning t{};
    resolve_tuning(d, ts_tuning{}, t);
    LaunchCfg cfg = cfg_of(t);
    unsigned* fbits = L.fbits ? (unsigned*)(b + L.fbits) : nullptr;
    if (parents && !fbits) return fail(TS_ERR_UNSUPPORTED, "%s: parents need d <= 256", fn);
    TS_CUDA(launch_msbfs_step(dev(A), dev(F), (int)d, visited, levels, level, sc, newbits,
                              (long long*)F_next->rowptr, cfg, st, fbits, parents),
            fn);
    long long tot = 0;
    TS_CUDA(cudaMemcpyAsync(&tot, (long long*)F_next->rowptr + n, sizeof tot, cudaMemcpyDeviceToHost, st), fn);
    unsigned long long err = 0;
    TS_CUDA(cudaMemcpyAsync(&err, &sc.hdr->err, sizeof err, cudaMemcpyDeviceToHost, st), fn);
    TS_CUDA(cudaStreamSynchronize(st), fn);
    if (err) return fail(TS_ERR_BAD_CSR, "%s: device checks failed (flags 0x%llx)", fn, err);
    *nnz_next_host = tot;
    if (tot > F_next_capacity)
        return fail(TS_ERR_CAPACITY, "%s: next frontier has %lld entries, capacity %lld", fn, tot,
                    (long long)F_next_capacity);
    TS_CUDA(launch_msbfs_emit(n, (int)d, newbits, (const long long*)F_next->rowptr, F_next->col,
                              F_next_capacity, sc.hdr, st),
            fn);
    return ok();
}

extern "C" ts_status msbfs_step(const ts_csr_desc* A, const ts_csr_desc* F, uint32_t* visited,
                                int32_t* levels, int32_t level, const ts_csr_desc* F_next,
                                int64_t F_next_capacity, int64_t* nnz_next_host, void* ws,
                                size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("msbfs_step");
    return bfs_step(A, F, visited, levels, nullptr, level, F_next, F_next_capacity, nnz_next_host, ws, ws_bytes,
                    stream, "msbfs_step");
}

extern "C" ts_status msbfs_step_parents(const ts_csr_desc* A, const ts_csr_desc* F, uint32_t* visited,
                                        int32_t* levels, int32_t* parents, int32_t level,
                                        const ts_csr_desc* F_next, int64_t F_next_capacity,
                                        int64_t* nnz_next_host, void* ws, size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("msbfs_step_parents");
    if (!parents) return fail(TS_ERR_INVALID_ARG, "msbfs_step_parents: parents is NULL");
    return bfs_step(A, F, visited, levels, parents, level, F_next, F_next_capacity, nnz_next_host, ws, ws_bytes,
                    stream, "msbfs_step_parents");
}

extern "C" ts_status msbfs_init_parents(int64_t n, int64_t d, const int32_t* sources_dev, int32_t* parents,
                                        void* stream) {
    const char* fn = "msbfs_init_parents";
    if (n < 0 || d < 1 || !sources_dev || !parents) return fail(TS_ERR_INVALID_ARG, "%s: bad argument", fn);
    if (n > INT32_MAX) return fail(TS_ERR_UNSUPPORTED, "%s: n >= 2^31", fn);
    if (d > 256) return fail(TS_ERR_UNSUPPORTED, "%s: parents need d <= 256", fn);
    TS_CUDA(launch_msbfs_init_parents(n, (int)d, sources_dev, parents, (cudaStream_t)stream), fn);
    return ok();
}

extern "C" ts_status msbfs_emit(const ts_csr_desc* F_next, int64_t F_next_capacity, void* ws,
                                size_t ws_bytes, void* stream) {
    const char* fn = "msbfs_emit";
    if (!F_next || !F_next->rowptr || !F_next->col || F_next_capacity < 0)
        return fail(TS_ERR_INVALID_ARG, "%s: bad F_next", fn);
    const long long n = F_next->nrows, d = F_next->ncols;
    if (n < 0 || d < 1 || d > MSBFS_MAX_D) return fail(TS_ERR_INVALID_ARG, "%s: bad shape", fn);
    const BfsLayout L = bfs_layout(n, d, 0);
    if (!ws || ws_bytes < L.newbits + sizeof(unsigned) * (size_t)n * (size_t)((d + 31) / 32))
        return fail(TS_ERR_WORKSPACE_TOO_SMALL, "%s", fn);
    cudaStream_t st = (cudaStream_t)stream;
    long long tot = 0;
    TS_CUDA(cudaMemcpyAsync(&tot, (long long*)F_next->rowptr + n, sizeof tot, cudaMemcpyDeviceToHost, st), fn);
    TS_CUDA(cudaStreamSynchronize(st), fn);
    if (tot > F_next_capacity)
        return fail(TS_ERR_CAPACITY, "%s: %lld entries, capacity %lld", fn, tot, (long long)F_next_capacity);
    char* b = (char*)ws;
    TS_CUDA(launch_msbfs_emit(n, (int)d, (const unsigned*)(b + L.newbits), (const long long*)F_next->rowptr,
                              F_next->col, F_next_capacity, (WsHeader*)(b + L.hdr), st),
            fn);
    return ok();
}

// ---------------------------------------------------------------------------
// batched products: one launch per phase over all instances, each instance
// read and written in place through a device table of descriptors
// ---------------------------------------------------------------------------
static const long long BAT_MAX_D = 1024;

struct ts_batched_plan {
    int count = 0;
    int semiring = 0;
    std::vector<long long> n, d, annz, bnnz, row_off, chunk_off, cap;
    // per-instance tuning: accumulator width, kind, dense copy width, heavy threshold
    std::vector<int> W, accum, Wd;
    std::vector<long long> heavy_min;
    long long N = 0, NC = 0, max_work = 0;  // rows, 32-row chunks (a chunk lies in one instance)
    int Wmax = 32;
    bool have_bounds = false;
    bool bound = false;
    std::vector<ts_csr_desc> bA, bB, bC;
    std::vector<const float*> gdC;
    std::vector<float*> gdA, gdB;
    bool grads = false;
    std::vector<InstDesc> host;  // the table last uploaded
};

struct BLayout {
    size_t inst = 0, bound = 0, ctl = 0, flops = 0, heavy = 0, total = 0;
    std::vector<size_t> q, dense;  // per instance: packed copy, dense copy (0: none)
};

static bool bat_vals(const ts_batched_plan* p) { return p->semiring == TS_SR_PLUS_TIMES_F32; }

static BLayout batched_layout(const ts_batched_plan* p) {
    BLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    L.inst = take(sizeof(InstDesc) * (size_t)p->count);
    L.bound = take(sizeof(long long) * (size_t)p->count);
    L.ctl = take(sizeof(BatchCtl));
    L.flops = take(sizeof(long long) * (size_t)std::max<long long>(p->N, 1));
    L.heavy = take(sizeof(int) * (size_t)std::max<long long>(p->N, 1));
    L.q.assign((size_t)p->count, 0);
    L.dense.assign((size_t)p->count, 0);
    for (int b = 0; b < p->count; ++b) {
        L.q[b] = take(padded_b_bytes(p->n[b], p->bnnz[b], p->d[b], 2));
        // every plus-times instance narrow enough for the dense-B form keeps
        // room for its dense copy, so that the autotuner may choose it
        if (bat_vals(p) && p->Wd[b] <= 256) L.dense[b] = take(dense_b_bytes(p->n[b], p->d[b]));
    }
    L.total = off;
    return L;
}

static ts_status batched_ws_check(const ts_batched_plan* p, void* ws, size_t ws_bytes, const BLayout& L,
                                  const char* fn) {
    if (!ws) return fail(TS_ERR_INVALID_ARG, "%s: workspace is NULL", fn);
    if (((uintptr_t)ws) & 255) return fail(TS_ERR_INVALID_ARG, "%s: workspace not 256-byte aligned", fn);
    if (ws_bytes < L.total)
        return fail(TS_ERR_WORKSPACE_TOO_SMALL, "%s: workspace of %zu bytes, %zu needed", fn, ws_bytes, L.total);
    (void)p;
    return TS_OK;
}

static void fill_insts(ts_batched_plan* p, const ts_csr_desc* A, const ts_csr_desc* B, const ts_csr_desc* C,
                       char* ws, const BLayout& L) {
    p->host.assign((size_t)p->count, InstDesc{});
    for (int b = 0; b < p->count; ++b) {
        InstDesc& I = p->host[b];
        I.n = p->n[b];
        I.d = p->d[b];
        I.annz = p->annz[b];
        I.bnnz = p->bnnz[b];
        I.cap = C ? C[b].nnz : 0;
        I.row_off = p->row_off[b];
        I.chunk_off = p->chunk_off[b];
        I.A_rowptr = (const long long*)A[b].rowptr;
        I.A_col = A[b].col;
        I.A_val = (const float*)A[b].val;
        I.B_rowptr = (const long long*)B[b].rowptr;
        I.B_col = B[b].col;
        I.B_val = (const float*)B[b].val;
        I.C_rowptr = C ? (long long*)C[b].rowptr : nullptr;
        I.C_col = C ? C[b].col : nullptr;
        I.C_val = C ? (float*)C[b].val : nullptr;
        I.dC = p->grads ? p->gdC[b] : nullptr;
        I.dA = p->grads ? p->gdA[b] : nullptr;
        I.dB = p->grads ? p->gdB[b] : nullptr;
        I.heavy_min = p->heavy_min[b];
        I.W = p->W[b];
        I.accum = p->accum[b];
        I.Wd = p->Wd[b];
        I.Bq = (int4*)(ws + L.q[b]);
        I.Bd = L.dense[b] ? (float*)(ws + L.dense[b]) : nullptr;
        I.Bbits = L.dense[b] ? (unsigned*)(ws + L.dense[b] + (size_t)p->n[b] * p->Wd[b] * 4) : nullptr;
        if (!I.Bd) I.accum = BAT_SPARSE;
    }
}

static ts_status upload_insts(ts_batched_plan* p, const ts_csr_desc* A, const ts_csr_desc* B,
                              const ts_csr_desc* C, char* ws, const BLayout& L, cudaStream_t st, const char* fn) {
    fill_insts(p, A, B, C, ws, L);
    TS_CUDA(cudaMemcpyAsync(ws + L.inst, p->host.data(), sizeof(InstDesc) * p->host.size(), cudaMemcpyHostToDevice,
                            st),
            fn);
    TS_CUDA(cudaStreamSynchronize(st), fn);
    return TS_OK;
}

static ts_status batched_errors(char* ws, const BLayout& L, cudaStream_t st, const char* fn) {
    unsigned long long err = 0;
    TS_CUDA(cudaMemcpyAsync(&err, &((BatchCtl*)(ws + L.ctl))->err, sizeof err, cudaMemcpyDeviceToHost, st), fn);
    TS_CUDA(cudaStreamSynchronize(st), fn);
    if (err & ERR_CAPACITY) return fail(TS_ERR_CAPACITY, "%s: an instance's C exceeds its capacity", fn);
    if (err)
        return fail(TS_ERR_BAD_CSR, "%s: device checks failed (flags 0x%llx: %s%s%s)", fn, err,
                    (err & ERR_A_COL) ? "column of A out of range; " : "",
                    (err & ERR_B_COL) ? "column of B out of range; " : "",
                    (err & ERR_C_ROW) ? "C row does not match its rowptr; " : "");
    return TS_OK;
}

extern "C" ts_status ts_batched_plan_create(int32_t count, const ts_csr_desc* A, const ts_csr_desc* B,
                                            int32_t semiring, const ts_tuning* force,
                                            ts_batched_plan** out) {
    const char* fn = "ts_batched_plan_create";
    if (!out) return fail(TS_ERR_INVALID_ARG, "%s: out is NULL", fn);
    *out = nullptr;
    if (count < 1 || !A || !B) return fail(TS_ERR_INVALID_ARG, "%s: need count >= 1 and descriptor arrays", fn);
    if (semiring != TS_SR_PLUS_TIMES_F32 && semiring != TS_SR_OR_SELECT2ND_BOOL)
        return fail(TS_ERR_INVALID_ARG, "%s: unknown semiring %d", fn, semiring);
    const ts_tuning f = force ? *force : ts_tuning{};
    if (f.cta_min_flops < 0) return fail(TS_ERR_INVALID_ARG, "%s: cta_min_flops must be >= 0", fn);
    if (f.accum < 0 || f.accum > TS_ACC_DENSE_B) return fail(TS_ERR_INVALID_ARG, "%s: unknown accum", fn);
    ts_batched_plan* p = new ts_batched_plan;
    p->count = count;
    p->semiring = semiring;
    const bool vals = semiring == TS_SR_PLUS_TIMES_F32;
    for (int b = 0; b < count; ++b) {
        if (A[b].nrows < 0 || A[b].ncols != A[b].nrows || B[b].nrows != A[b].nrows || B[b].ncols < 1 ||
            A[b].nnz < 0 || B[b].nnz < 0) {
            delete p;
            return fail(TS_ERR_INVALID_ARG, "%s: instance %d: A must be n x n and B n x d (d >= 1)", fn, b);
        }
        if (B[b].ncols > BAT_MAX_D) {
            delete p;
            return fail(TS_ERR_UNSUPPORTED, "%s: instance %d: d = %lld above the batched limit %lld", fn, b,
                        (long long)B[b].ncols, BAT_MAX_D);
        }
        p->n.push_back(A[b].nrows);
        p->d.push_back(B[b].ncols);
        p->annz.push_back(A[b].nnz);
        p->bnnz.push_back(B[b].nnz);
        p->row_off.push_back(p->N);
        p->chunk_off.push_back(p->NC);
        p->N += A[b].nrows;
        p->NC += (A[b].nrows + 31) / 32;
        const int w = (int)round_up(B[b].ncols, 32);
        int wd = 32;
        while (wd < w) wd *= 2;
        p->W.push_back(w);
        p->Wd.push_back(wd);
        p->Wmax = std::max(p->Wmax, w);
        // default tuning of the instance; `force` fixes a field for all
        const bool dense = f.accum == TS_ACC_DENSE_B ? (vals && wd <= 256)
                         : f.accum == 0 ? (dense_b_auto(vals, B[b].ncols, A[b].nrows, B[b].nnz) && wd <= 256)
                                         : false;
        p->accum.push_back(dense ? BAT_DENSE_B : BAT_SPARSE);
        p->heavy_min.push_back(f.cta_min_flops ? f.cta_min_flops : 4096);
        p->max_work = std::max<long long>(p->max_work, std::max<long long>(A[b].nnz, B[b].nnz));
    }
    if (p->N > INT32_MAX) {
        delete p;
        return fail(TS_ERR_UNSUPPORTED, "%s: more than 2^31-1 rows in total", fn);
    }
    p->cap.assign((size_t)count, 0);
    *out = p;
    return ok();
}

extern "C" ts_status ts_batched_plan_destroy(ts_batched_plan* plan) {
    delete plan;
    return ok();
}

extern "C" ts_status ts_batched_workspace_size(const ts_batched_plan* plan, size_t* bytes) {
    if (!plan || !bytes) return fail(TS_ERR_INVALID_ARG, "ts_batched_workspace_size: NULL argument");
    *bytes = batched_layout(plan).total;
    return ok();
}

extern "C" ts_status ts_batched_get_tuning(const ts_batched_plan* plan, int32_t b, ts_tuning* out) {
    if (!plan || !out || b < 0 || b >= plan->count)
        return fail(TS_ERR_INVALID_ARG, "ts_batched_get_tuning: bad arguments");
    ts_tuning t{};
    t.accum = plan->accum[b] == BAT_DENSE_B ? TS_ACC_DENSE_B : TS_ACC_DENSE;
    t.col_tile = plan->W[b];
    t.cta_min_flops = plan->heavy_min[b];
    t.warps_per_cta = 8;
    t.row_lanes = 1;
    t.pack_b = 1;
    *out = t;
    return ok();
}

// The forward passes over instances [b0, b0 + nb) (32-row chunks c0 .. c1 - 1).
static ts_status bat_forward(ts_batched_plan* plan, char* w, const BLayout& L, int b0, int nb, cudaStream_t st,
                             const char* fn, bool numeric = true) {
    const InstDesc* inst = (const InstDesc*)(w + L.inst) + b0;
    BatchCtl* ctl = (BatchCtl*)(w + L.ctl);
    long long* flops = (long long*)(w + L.flops);
    int* heavy = (int*)(w + L.heavy);
    const long long c0 = plan->chunk_off[b0];
    const long long c1 = plan->chunk_off[b0 + nb - 1] + (plan->n[b0 + nb - 1] + 31) / 32;
    const int sms = sm_count();
    TS_CUDA(cudaMemsetAsync(ctl, 0, sizeof(BatchCtl), st), fn);
    TS_CUDA(launch_bat_prepare(inst, nb, c0, c1, flops, heavy, ctl, sms, st), fn);
    if (!numeric) return TS_OK;
    TS_CUDA(launch_bat_symbolic(inst, nb, c0, c1, 0, flops, heavy, ctl, plan->Wmax, sms, st), fn);
    TS_CUDA(launch_bat_scan(inst, nb, ctl, st), fn);
    TS_CUDA(launch_bat_numeric(inst, nb, c0, c1, bat_vals(plan) ? 1 : 0, flops, heavy, ctl, plan->Wmax, sms, st),
            fn);
    return TS_OK;
}

extern "C" ts_status ts_batched_bounds(ts_batched_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                       int64_t* C_capacity, void* ws, size_t ws_bytes, void* stream) {
    const char* fn = "ts_batched_bounds";
    if (!plan || !A || !B || !C_capacity) return fail(TS_ERR_INVALID_ARG, "%s: NULL argument", fn);
    const BLayout L = batched_layout(plan);
    ts_status s = batched_ws_check(plan, ws, ws_bytes, L, fn);
    if (s != TS_OK) return s;
    const bool vals = bat_vals(plan);
    for (int b = 0; b < plan->count; ++b) {
        if (A[b].nrows != plan->n[b] || A[b].nnz != plan->annz[b] || B[b].ncols != plan->d[b] ||
            B[b].nnz != plan->bnnz[b])
            return fail(TS_ERR_INVALID_ARG, "%s: instance %d differs from the plan", fn, b);
        if ((s = check_desc(&A[b], "A", vals)) != TS_OK || (s = check_desc(&B[b], "B", vals)) != TS_OK) return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)ws;
    if ((s = upload_insts(plan, A, B, nullptr, w, L, st, fn)) != TS_OK) return s;
    if ((s = bat_forward(plan, w, L, 0, plan->count, st, fn, false)) != TS_OK) return s;
    const InstDesc* inst = (const InstDesc*)(w + L.inst);
    TS_CUDA(launch_batch_bounds(inst, plan->count, (const long long*)(w + L.flops), (long long*)(w + L.bound), st),
            fn);
    std::vector<long long> bnd((size_t)plan->count);
    TS_CUDA(cudaMemcpyAsync(bnd.data(), w + L.bound, sizeof(long long) * bnd.size(), cudaMemcpyDeviceToHost, st), fn);
    if ((s = batched_errors(w, L, st, fn)) != TS_OK) return s;
    for (int b = 0; b < plan->count; ++b) {
        plan->cap[b] = bnd[b];
        C_capacity[b] = bnd[b];
    }
    plan->have_bounds = true;
    plan->bound = false;
    return ok();
}

extern "C" ts_status ts_batched_bind(ts_batched_plan* plan, const ts_csr_desc* A, const ts_csr_desc* B,
                                     const ts_csr_desc* C, void* ws, size_t ws_bytes, void* stream) {
    const char* fn = "ts_batched_bind";
    if (!plan || !A || !B || !C) return fail(TS_ERR_INVALID_ARG, "%s: NULL argument", fn);
    if (!plan->have_bounds) return fail(TS_ERR_STATE, "%s: call ts_batched_bounds first", fn);
    const BLayout L = batched_layout(plan);
    ts_status s = batched_ws_check(plan, ws, ws_bytes, L, fn);
    if (s != TS_OK) return s;
    const bool vals = bat_vals(plan);
    for (int b = 0; b < plan->count; ++b) {
        if (A[b].nrows != plan->n[b] || A[b].nnz != plan->annz[b] || B[b].ncols != plan->d[b] ||
            B[b].nnz != plan->bnnz[b])
            return fail(TS_ERR_INVALID_ARG, "%s: instance %d differs from the plan", fn, b);
        if ((s = check_desc(&A[b], "A", vals)) != TS_OK || (s = check_desc(&B[b], "B", vals)) != TS_OK) return s;
        if (!C[b].rowptr || C[b].nrows != plan->n[b] || C[b].ncols != plan->d[b] ||
            (C[b].nnz > 0 && (!C[b].col || (vals && !C[b].val))))
            return fail(TS_ERR_INVALID_ARG, "%s: instance %d: bad C descriptor", fn, b);
    }
    plan->bA.assign(A, A + plan->count);
    plan->bB.assign(B, B + plan->count);
    plan->bC.assign(C, C + plan->count);
    if ((s = upload_insts(plan, A, B, C, (char*)ws, L, (cudaStream_t)stream, fn)) != TS_OK) return s;
    plan->bound = true;
    return ok();
}

extern "C" ts_status ts_batched_bind_grads(ts_batched_plan* plan, int32_t count, const float* const* dC_val,
                                           float* const* dA_val, float* const* dB_val, void* ws, size_t ws_bytes,
                                           void* stream) {
    const char* fn = "ts_batched_bind_grads";
    if (!plan || !dC_val || count != plan->count) return fail(TS_ERR_INVALID_ARG, "%s: bad arguments", fn);
    if (plan->semiring != TS_SR_PLUS_TIMES_F32)
        return fail(TS_ERR_UNSUPPORTED, "%s: the boolean semiring has no gradient", fn);
    if (!plan->bound) return fail(TS_ERR_STATE, "%s: call ts_batched_bind first", fn);
    const BLayout L = batched_layout(plan);
    ts_status s = batched_ws_check(plan, ws, ws_bytes, L, fn);
    if (s != TS_OK) return s;
    plan->gdC.assign(dC_val, dC_val + count);
    plan->gdA.assign((size_t)count, nullptr);
    plan->gdB.assign((size_t)count, nullptr);
    for (int b = 0; b < count; ++b) {
        if (dA_val) plan->gdA[b] = dA_val[b];
        if (dB_val) plan->gdB[b] = dB_val[b];
    }
    plan->grads = true;
    return upload_insts(plan, plan->bA.data(), plan->bB.data(), plan->bC.data(), (char*)ws, L,
                        (cudaStream_t)stream, fn) == TS_OK ? ok() : TS_ERR_CUDA;
}

static bool same_descs(const std::vector<ts_csr_desc>& v, const ts_csr_desc* x, int count) {
    if ((int)v.size() != count || !x) return false;
    for (int b = 0; b < count; ++b)
        if (v[b].nrows != x[b].nrows || v[b].ncols != x[b].ncols || v[b].nnz != x[b].nnz ||
            v[b].rowptr != x[b].rowptr || v[b].col != x[b].col || v[b].val != x[b].val)
            return false;
    return true;
}

extern "C" ts_status ts_spgemm_batched(ts_batched_plan* plan, int32_t count, const ts_csr_desc* A,
                                       const ts_csr_desc* B, const ts_csr_desc* C, void* ws, size_t ws_bytes,
                                       void* stream) {
    NvtxRange nvtx_range("ts_spgemm_batched");
    const char* fn = "ts_spgemm_batched";
    if (!plan) return fail(TS_ERR_INVALID_ARG, "%s: plan is NULL", fn);
    if (!plan->bound) return fail(TS_ERR_STATE, "%s: call ts_batched_bind first", fn);
    if (count != plan->count || !same_descs(plan->bA, A, count) || !same_descs(plan->bB, B, count) ||
        !same_descs(plan->bC, C, count))
        return fail(TS_ERR_INVALID_ARG, "%s: descriptors differ from those bound", fn);
    const BLayout L = batched_layout(plan);
    ts_status s = batched_ws_check(plan, ws, ws_bytes, L, fn);
    if (s != TS_OK) return s;
    s = bat_forward(plan, (char*)ws, L, 0, plan->count, (cudaStream_t)stream, fn);
    return s == TS_OK ? ok() : s;
}

extern "C" ts_status ts_spgemm_batched_backward(ts_batched_plan* plan, int32_t count,
                                                const float* const* dC_val, float* const* dA_val,
                                                float* const* dB_val, void* ws, size_t ws_bytes,
                                                void* stream) {
    NvtxRange nvtx_range("ts_spgemm_batched_backward");
    const char* fn = "ts_spgemm_batched_backward";
    if (!plan) return fail(TS_ERR_INVALID_ARG, "%s: plan is NULL", fn);
    if (!plan->grads) return fail(TS_ERR_STATE, "%s: call ts_batched_bind_grads first", fn);
    if (count != plan->count || !dC_val) return fail(TS_ERR_INVALID_ARG, "%s: bad arguments", fn);
    for (int b = 0; b < count; ++b)
        if (dC_val[b] != plan->gdC[b] || (dA_val ? dA_val[b] : nullptr) != plan->gdA[b] ||
            (dB_val ? dB_val[b] : nullptr) != plan->gdB[b])
            return fail(TS_ERR_INVALID_ARG, "%s: gradient arrays differ from those bound", fn);
    const BLayout L = batched_layout(plan);
    ts_status s = batched_ws_check(plan, ws, ws_bytes, L, fn);
    if (s != TS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)ws;
    BatchCtl* ctl = (BatchCtl*)(w + L.ctl);
    // the backward reuses the forward's row flops, heavy list and C pattern
    TS_CUDA(cudaMemsetAsync(&ctl->q_bwd, 0, 2 * sizeof ctl->q_bwd, st), fn);  // q_bwd, l_bwd
    TS_CUDA(launch_bat_backward((const InstDesc*)(w + L.inst), plan->count, 0, plan->N, plan->max_work,
                                (const long long*)(w + L.flops), (const int*)(w + L.heavy), ctl, plan->Wmax,
                                sm_count(), st),
            fn);
    return ok();
}

extern "C" ts_status ts_batched_check(ts_batched_plan* plan, void* ws, size_t ws_bytes, void* stream) {
    const char* fn = "ts_batched_check";
    if (!plan) return fail(TS_ERR_INVALID_ARG, "%s: plan is NULL", fn);
    const BLayout L = batched_layout(plan);
    ts_status s = batched_ws_check(plan, ws, ws_bytes, L, fn);
    if (s != TS_OK) return s;
    s = batched_errors((char*)ws, L, (cudaStream_t)stream, fn);
    return s == TS_OK ? ok() : s;
}

// Per instance, every candidate (accumulator kind x heavy-row threshold) is
// timed on that instance alone (its four forward launches over its rows
// only) and the fastest kept in its descriptor; then a few whole-batch
// tunings built from those choices are timed and the fastest kept.
extern "C" ts_status ts_batched_autotune(ts_batched_plan* plan, int32_t reps, ts_tuning* chosen, void* ws,
                                         size_t ws_bytes, void* stream) {
    const char* fn = "ts_batched_autotune";
    if (!plan || !plan->bound) return fail(TS_ERR_STATE, "%s: bind the plan first", fn);
    if (reps < 1) return fail(TS_ERR_INVALID_ARG, "%s: reps must be >= 1", fn);
    const BLayout L = batched_layout(plan);
    ts_status s = batched_ws_check(plan, ws, ws_bytes, L, fn);
    if (s != TS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)ws;
    cudaEvent_t e0, e1;
    TS_CUDA(cudaEventCreate(&e0), fn);
    TS_CUDA(cudaEventCreate(&e1), fn);
    const long long mins[] = {1024, 4096, 16384, 1LL << 50};
    const std::vector<int> start_acc = plan->accum;
    const std::vector<long long> start_min = plan->heavy_min;
    for (int b = 0; b < plan->count && s == TS_OK; ++b) {
        if (plan->n[b] == 0) continue;
        int best_acc = plan->accum[b];
        long long best_min = plan->heavy_min[b];
        float best_ms = 1e30f;
        for (int acc = BAT_SPARSE; acc <= BAT_DENSE_B && s == TS_OK; ++acc) {
            if (acc == BAT_DENSE_B && !L.dense[b]) continue;
            for (long long hm : mins) {
                plan->accum[b] = acc;
                plan->heavy_min[b] = hm;
                fill_insts(plan, plan->bA.data(), plan->bB.data(), plan->bC.data(), w, L);
                if (cudaMemcpyAsync(w + L.inst + b * sizeof(InstDesc), &plan->host[b], sizeof(InstDesc),
                                    cudaMemcpyHostToDevice, st) != cudaSuccess) {
                    s = cuda_fail(cudaGetLastError(), fn);
                    break;
                }
                float tot = 0.0f;
                for (int r = 0; r <= reps && s == TS_OK; ++r) {
                    if (cudaEventRecord(e0, st) != cudaSuccess) s = cuda_fail(cudaGetLastError(), fn);
                    if (s == TS_OK) s = bat_forward(plan, w, L, b, 1, st, fn);
                    if (s == TS_OK && cudaEventRecord(e1, st) != cudaSuccess) s = cuda_fail(cudaGetLastError(), fn);
                    if (s == TS_OK && cudaEventSynchronize(e1) != cudaSuccess) s = cuda_fail(cudaGetLastError(), fn);
                    float ms = 0.0f;
                    if (s == TS_OK) cudaEventElapsedTime(&ms, e0, e1);
                    if (r > 0) tot += ms;
                }
                if (s == TS_OK && tot / reps < best_ms) {
                    best_ms = tot / reps;
                    best_acc = acc;
                    best_min = hm;
                }
            }
        }
        plan->accum[b] = best_acc;
        plan->heavy_min[b] = best_min;
    }
    // An instance timed alone favours a low heavy threshold (more blocks on
    // a GPU it cannot fill); in the batch the GPU is full and the tail is
    // short.  So the whole batch is timed under (a) every instance's own
    // choice, (b) the tuning the autotuner started from and (c) the
    // instances' own accumulators with one heavy threshold for all, and the
    // fastest is kept.
    struct Cand {
        std::vector<int> acc;
        std::vector<long long> hm;
    };
    std::vector<Cand> cands;
    cands.push_back({plan->accum, plan->heavy_min});
    cands.push_back({start_acc, start_min});
    for (long long hm : {1024LL, 4096LL, 16384LL})
        cands.push_back({plan->accum, std::vector<long long>((size_t)plan->count, hm)});
    size_t best = 0;
    float best_ms = 1e30f;
    for (size_t c = 0; c < cands.size() && s == TS_OK; ++c) {
        plan->accum = cands[c].acc;
        plan->heavy_min = cands[c].hm;
        if ((s = upload_insts(plan, plan->bA.data(), plan->bB.data(), plan->bC.data(), w, L, st, fn)) != TS_OK) break;
        float tot = 0.0f;
        for (int r = 0; r <= reps && s == TS_OK; ++r) {
            if (cudaEventRecord(e0, st) != cudaSuccess) s = cuda_fail(cudaGetLastError(), fn);
            if (s == TS_OK) s = bat_forward(plan, w, L, 0, plan->count, st, fn);
            if (s == TS_OK && cudaEventRecord(e1, st) != cudaSuccess) s = cuda_fail(cudaGetLastError(), fn);
            if (s == TS_OK && cudaEventSynchronize(e1) != cudaSuccess) s = cuda_fail(cudaGetLastError(), fn);
            float ms = 0.0f;
            if (s == TS_OK) cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) tot += ms;
        }
        if (s == TS_OK && tot / reps < best_ms) {
            best_ms = tot / reps;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != TS_OK) return s;
    plan->accum = cands[best].acc;
    plan->heavy_min = cands[best].hm;
    if ((s = upload_insts(plan, plan->bA.data(), plan->bB.data(), plan->bC.data(), w, L, st, fn)) != TS_OK) return s;
    // leave every C_b holding the product of the chosen tunings
    if ((s = bat_forward(plan, w, L, 0, plan->count, st, fn)) != TS_OK) return s;
    if ((s = batched_errors(w, L, st, fn)) != TS_OK) return s;
    if (chosen) ts_batched_get_tuning(plan, 0, chosen);
    return ok();
}
