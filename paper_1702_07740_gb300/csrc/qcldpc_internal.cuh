// Internal definitions shared by the qcldpc CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "qcldpc.h"

namespace qc {

constexpr int kMaxRows = QCLDPC_MAX_BASE_ROWS;
constexpr int kMaxCols = QCLDPC_MAX_BASE_COLS;
constexpr int kMaxCirc = QCLDPC_MAX_CIRCULANTS;
constexpr int kMaxHeavyCols = QCLDPC_MAX_HEAVY_COLS;
constexpr int kMaxRowDeg = QCLDPC_MAX_ROW_DEGREE;

// One circulant as seen from its base row. Heavy entries come first in each
// row; `slot` is the heavy-column slot (heavy) or -1 (degree-1); `id` is the
// heavy-circulant index (message array) or the degree-1 circulant index.
struct RowEnt {
    int32_t shift;
    int32_t slot;
    int32_t id;
    int32_t col;  // base column
};

// One heavy circulant as seen from its heavy column.
struct ColEnt {
    int32_t shift;
    int32_t id;  // heavy-circulant index
};

// Everything the check-node pass needs about one base row, in one aligned
// 64-byte record (read with four vector loads at block start): the row, its
// first entry, its heavy and degree-1 counts and, for rows of up to
// kDescEnts entries, every entry's off_a / off_b (see Table).
constexpr int kDescEnts = 6;
// Heavy-column lists up to these sizes also travel inline in the Table.
constexpr int kInlineCols = 512;
constexpr int kInlineHcols = 32;
struct alignas(16) RowDesc {
    int32_t r, rp, nh, nd;
    int32_t off_a[kDescEnts];
    int32_t off_b[kDescEnts];
};
static_assert(sizeof(RowDesc) == 64, "RowDesc is four 16-byte loads");

// Row shapes (heavy, degree-1 circulants) with an exactly unrolled, staged
// check-node body; other shapes take the generic path.
__host__ __device__ constexpr bool exact_shape(int nh, int nd) {
    return (nd == 1 && nh >= 1 && nh <= 4) || (nd == 0 && nh >= 2 && nh <= 4);
}

// Code tables as the kernels see them: scalars, and pointers into the code's
// block of the library's static device table arena (uploaded on the first
// call that launches work). Passed to kernels by value as a
// __grid_constant__ parameter; the kernels read the arrays with warp-uniform
// indices through the L1 cache.
struct Table {
    int32_t Z, mb, nb;
    int32_t n_circ;   // all circulants
    int32_t n_h;      // heavy circulants (own message arrays)
    int32_t n_d1;     // degree-1 circulants (one per degree-1 column)
    int32_t n_hcols;  // heavy columns (posterior arrays)
    int32_t k;        // key bits = n - m
    int32_t max_row_deg;
    int32_t stage_rows_max;   // max over exact-shape rows of 2 nh + nd (staged float rows)
    int32_t stage_words_max;  // max over exact-shape rows of nd (staged decision-word rows)
    int32_t pad_;
    const int32_t *row_ptr;    // [mb + 1] into rows[]
    const int32_t *row_nh;     // [mb] heavy entries of the row
    const int32_t *row_order;  // [mb] rows sorted by shape (check-node grid order)
    const RowDesc *row_desc;      // [mb] per base row
    const RowDesc *row_desc_ord;  // [mb] in row_order (flooding check-pass grid order)
    const int32_t *col_ptr;    // [n_hcols + 1] into cols[]
    const int32_t *hcol_base;  // [n_hcols] base column of each heavy slot
    const int32_t *col_kind;   // [nb] >= 0 heavy slot; <= -2: d1 id = -kind-2
    const RowEnt *rows;        // [n_circ]
    // Per row entry, in elements of one frame's arrays: heavy entries
    // off_a = slot * 2Z + shift (posterior read), off_b = id * Z (messages);
    // degree-1 entries off_a = id * Z (Phi values), off_b = id * ceil(Z/32)
    // (decision words).
    const int32_t *row_off_a;  // [n_circ]
    const int32_t *row_off_b;  // [n_circ]
    const ColEnt *cols;        // [n_h] heavy circulants by heavy column
    const int32_t *col_row;    // [n_h] base row of each cols[] entry
    const int32_t *d1_shift;   // [n_d1]
    const int32_t *d1_row;     // [n_d1]
    const int32_t *d1_col;     // [n_d1]
};

// Inline copy of the heavy-column lists for codes that fit, a kernel
// parameter of the variable pass alone (read through the constant bank).
struct ColsInline {
    int32_t ok;  // 0: the code does not fit; use Table::col_ptr / cols
    int32_t col_ptr[kInlineHcols + 1];
    ColEnt cols[kInlineCols];
};

// Host copy of the same arrays (built by qcldpc_create_code).
struct HostTable {
    std::vector<int32_t> row_ptr, row_nh, row_order, col_ptr, hcol_base, col_kind;
    std::vector<RowDesc> row_desc, row_desc_ord;
    std::vector<RowEnt> rows;
    std::vector<int32_t> row_off_a, row_off_b;
    std::vector<ColEnt> cols;
    std::vector<int32_t> col_row, d1_shift, d1_row, d1_col;
};

// Uploads the code's tables to the device table arena if they are not there
// yet (first call on a device); fills the pointers of code->tab.
int upload_tables(qcldpc_code *code);
// Returns the code's arena block (qcldpc_destroy_code).
void release_tables(qcldpc_code *code);

}  // namespace qc

struct qcldpc_code {
    qc::Table tab;       // device pointers are null until upload_tables
    qc::ColsInline cols_in;
    qc::HostTable host;
    std::mutex table_mu;  // guards the upload
    size_t arena_off, arena_bytes;  // the code's block of the table arena (bytes == 0: none)
    int device;
    int64_t n, m, k, n_edges;
    std::mutex mu;      // serialises decode calls on this handle
    void *graph_cache;  // decoder graph state (decode.cu), may be NULL
    void *last_ws;      // workspace, frame count and soft flag of the last decode
    int last_frames;
    int last_soft;
    unsigned char last_work[320];  // the last decode's kernel arguments (decode.cu)
};

namespace qc {

// Status helpers (api.cu).
int fail(int status, const std::string &msg);
int cuda_fail(cudaError_t err, const char *what);
void clear_error();

// Release decoder graph state of a code (decode.cu).
void destroy_graph_cache(qcldpc_code *code);
// Drop cached batched-decode graphs that decode this code (decode.cu).
void purge_multi_graphs(const qcldpc_code *code);

inline bool aligned(const void *p, size_t a) {
    return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0;
}

}  // namespace qc
