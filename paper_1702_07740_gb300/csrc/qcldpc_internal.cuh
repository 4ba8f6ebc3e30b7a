// Internal definitions shared by the qcldpc CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

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
    int16_t slot;
    int16_t id;
    int16_t col;  // base column
    int16_t pad;
};

// One heavy circulant as seen from its heavy column.
struct ColEnt {
    int32_t shift;
    int32_t id;  // heavy-circulant index
};

// Code tables, passed to kernels by value as a __grid_constant__ parameter
// (read through the constant cache with warp-uniform indices).
struct Table {
    int32_t Z, mb, nb;
    int32_t n_circ;   // all circulants
    int32_t n_h;      // heavy circulants (own message arrays)
    int32_t n_d1;     // degree-1 circulants (one per degree-1 column)
    int32_t n_hcols;  // heavy columns (posterior arrays)
    int32_t k;        // key bits = n - m
    int32_t max_row_deg;
    int32_t pad_;
    uint16_t row_ptr[kMaxRows + 1];     // into rows[]
    uint8_t row_nh[kMaxRows];           // heavy entries of the row
    uint8_t row_order[kMaxRows];        // rows sorted by shape (check-node grid order)
    uint16_t col_ptr[kMaxHeavyCols + 1];  // into cols[]
    int16_t hcol_base[kMaxHeavyCols];   // base column of each heavy slot
    int16_t col_kind[kMaxCols];         // >= 0 heavy slot; <= -2: d1 id = -kind-2
    RowEnt rows[kMaxCirc];
    // Per row entry, in elements of one frame's arrays: heavy entries
    // off_a = slot * 2Z + shift (posterior read), off_b = id * Z (messages);
    // degree-1 entries off_a = id * Z (Phi values), off_b = id * ceil(Z/32)
    // (decision words).
    int32_t row_off_a[kMaxCirc];
    int32_t row_off_b[kMaxCirc];
    ColEnt cols[kMaxCirc];
    int16_t col_row[kMaxCirc];          // base row of each cols[] entry
    int32_t d1_shift[kMaxCirc];
    int16_t d1_row[kMaxCirc];
    int16_t d1_col[kMaxCirc];
};

}  // namespace qc

struct qcldpc_code {
    qc::Table tab;
    int device;
    int64_t n, m, k, n_edges;
    std::mutex mu;      // serialises decode calls on this handle
    void *graph_cache;  // decoder graph state (decode.cu), may be NULL
    void *last_ws;      // workspace, frame count and soft flag of the last decode
    int last_frames;
    int last_soft;
    unsigned char last_work[256];  // the last decode's kernel arguments (decode.cu)
};

namespace qc {

// Status helpers (api.cu).
int fail(int status, const std::string &msg);
int cuda_fail(cudaError_t err, const char *what);
void clear_error();

// Release decoder graph state of a code (decode.cu).
void destroy_graph_cache(qcldpc_code *code);

inline bool aligned(const void *p, size_t a) {
    return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0;
}

}  // namespace qc
