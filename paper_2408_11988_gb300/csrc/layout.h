// Workspace header and device-check flags shared by the kernels and the host
// side of the C ABI (plain C++, no device code).
#pragma once

namespace ts {

constexpr int NUM_CLASSES = 48;  // class 0: no products; class c >= 1: flops in [2^(c-1), 2^c)

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
