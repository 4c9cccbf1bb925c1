// Workspace header and device-check flags shared by the kernels and the host
// side of the C ABI (plain C++, no device code).
#pragma once

namespace ts {

// Row classes by products (flops): class 0 = no products; class
// 1 + 8*lg + sub (lg = floor(log2 f), sub = the three bits of f below its
// leading one) holds an eighth of an octave, so the rows of one class differ
// in flops by less than 12.5 % and rows taken side by side in lockstep have
// nearly equal lengths.
constexpr int CLASS_SUB_BITS = 3;
constexpr int NUM_CLASSES = 1 + 48 * (1 << CLASS_SUB_BITS);

// Host copy of the device-side class function (common.cuh).
inline int flops_class_host(long long f) {
    if (f <= 0) return 0;
    const int lg = 63 - __builtin_clzll((unsigned long long)f);
    const int sub = lg >= CLASS_SUB_BITS ? (int)((f >> (lg - CLASS_SUB_BITS)) & ((1 << CLASS_SUB_BITS) - 1))
                                         : (int)((f << (CLASS_SUB_BITS - lg)) & ((1 << CLASS_SUB_BITS) - 1));
    const int c = 1 + (lg << CLASS_SUB_BITS) + sub;
    return c < NUM_CLASSES ? c : NUM_CLASSES - 1;
}

// First class whose rows all have at least min_flops products (rounded up
// to a class boundary).
inline int class_at_least(long long min_flops) {
    return min_flops <= 1 ? 1 : flops_class_host(min_flops - 1) + 1;
}

// error bits recorded in the workspace header by device-side checks
constexpr unsigned long long ERR_A_COL = 1ull;     // column of A outside [0, n)
constexpr unsigned long long ERR_B_COL = 2ull;     // column of B outside [0, d)
constexpr unsigned long long ERR_C_ROW = 4ull;     // row of C longer/shorter than its rowptr
constexpr unsigned long long ERR_HASH_FULL = 8ull; // hash table overflow (row too wide)
constexpr unsigned long long ERR_CAPACITY = 16ull; // output capacity exceeded

// Rows of A with more than SPLIT_ENTRIES entries are cut into work items of
// SPLIT_ENTRIES entries that any thread block can take; at most
// MAX_SPLIT_ROWS rows per product are cut (the rest run whole).
constexpr int SPLIT_ENTRIES = 1024;
constexpr int MAX_SPLIT_ROWS = 8192;

// Workspace header (offset 0 of every workspace).
struct WsHeader {
    unsigned long long heavy_ctr;     // next heavy row (dynamic CTA scheduling)
    unsigned long long item_ctr;      // next split-row work item
    unsigned long long err;           // ERR_* bits
    long long hist[NUM_CLASSES];      // rows per flops class
    long long cursor[NUM_CLASSES];    // scatter cursors per class
    long long scratch[8];             // [0] flops items, [1] split rows, [2] split items
};

}  // namespace ts
