// Code construction, status reporting and option defaults of the qcldpc C ABI.
//
// QC expansion (arXiv 1702.07740, Sec. III-D): a base entry holding shift s
// stands for the Z x Z identity shifted right by s, so row i of the block has
// its one at column (i + s) mod Z. The expansion is never materialised: the
// kernels address messages as (circulant, offset) and compute (i + s) mod Z
// on the fly. This file classifies the base columns (degree-1 diagonal
// columns vs heavy columns) and lays out the per-row and per-column circulant
// tables the kernels read.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "qcldpc_internal.cuh"

namespace {
thread_local std::string g_last_error;
}

namespace qc {

int fail(int status, const std::string &msg) {
    g_last_error = msg;
    return status;
}

int cuda_fail(cudaError_t err, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(err);
    return QCLDPC_E_CUDA;
}

void clear_error() { g_last_error.clear(); }

}  // namespace qc

extern "C" const char *qcldpc_last_error(void) { return g_last_error.c_str(); }

extern "C" void qcldpc_params_init(qcldpc_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->clip = 15.0f;
    p->phi_floor = 1e-6f;
    p->et_start = 1;
    p->schedule = 0;
    p->msg_format = 0;
    p->soft_output = 0;
    p->launch_mode = 0;
    p->msg_step = 0.0f;
    p->layers = 0;
}

extern "C" int qcldpc_create_code(int mb, int nb, int Z, int n_circ,
                                  const int32_t *circ_row,
                                  const int32_t *circ_col,
                                  const int32_t *circ_shift,
                                  qcldpc_code **out) {
    using namespace qc;
    if (!out) return fail(QCLDPC_E_INVAL, "create_code: out is NULL");
    *out = nullptr;
    if (!circ_row || !circ_col || !circ_shift)
        return fail(QCLDPC_E_INVAL, "create_code: NULL circulant array");
    if (mb < 1 || nb < 1 || Z < 1 || n_circ < 1)
        return fail(QCLDPC_E_INVAL, "create_code: mb, nb, Z, n_circ must be >= 1");
    if (mb > kMaxRows || nb > kMaxCols || n_circ > kMaxCirc || Z > QCLDPC_MAX_Z)
        return fail(QCLDPC_E_UNSUPPORTED,
                    "create_code: base matrix, circulant count or Z above the table limits");
    const int64_t n = (int64_t)nb * Z, m = (int64_t)mb * Z;
    // Offsets inside one frame's arrays are 32-bit: every array (n_circ Z
    // messages, 2Z per heavy posterior row) and n, m stay below 2^30.
    if (n > (1 << 30) || m > (1 << 30) || (int64_t)n_circ * Z > (1 << 29))
        return fail(QCLDPC_E_UNSUPPORTED, "create_code: n, m or n_circ * Z too large");

    std::vector<int> col_count(nb, 0), row_count(mb, 0);
    for (int h = 0; h < n_circ; h++) {
        if (circ_row[h] < 0 || circ_row[h] >= mb || circ_col[h] < 0 || circ_col[h] >= nb)
            return fail(QCLDPC_E_INVAL, "create_code: circulant row/column out of range");
        if (circ_shift[h] < 0 || circ_shift[h] >= Z)
            return fail(QCLDPC_E_SHIFT_RANGE, "create_code: circulant shift outside [0, Z)");
        col_count[circ_col[h]]++;
        row_count[circ_row[h]]++;
    }
    // Equal shifts in one base entry would cancel over GF(2).
    {
        std::vector<int64_t> keys(n_circ);
        for (int h = 0; h < n_circ; h++)
            keys[h] = ((int64_t)circ_row[h] * nb + circ_col[h]) * (int64_t)Z + circ_shift[h];
        std::sort(keys.begin(), keys.end());
        for (int h = 1; h < n_circ; h++)
            if (keys[h] == keys[h - 1])
                return fail(QCLDPC_E_DUP_SHIFT, "create_code: duplicate shift in one base entry");
    }
    for (int r = 0; r < mb; r++)
        if (row_count[r] > kMaxRowDeg)
            return fail(QCLDPC_E_UNSUPPORTED, "create_code: base row holds more circulants than QCLDPC_MAX_ROW_DEGREE");

    qcldpc_code *code = new (std::nothrow) qcldpc_code();
    if (!code) return fail(QCLDPC_E_NOMEM, "create_code: out of host memory");
    Table &T = code->tab;
    std::memset(&T, 0, sizeof(T));
    T.Z = Z;
    T.mb = mb;
    T.nb = nb;
    T.n_circ = n_circ;

    // Column classification: exactly one circulant -> degree-1 column.
    int n_hcols = 0;
    for (int c = 0; c < nb; c++) {
        if (col_count[c] == 1) continue;
        if (n_hcols >= kMaxHeavyCols) {
            delete code;
            return fail(QCLDPC_E_UNSUPPORTED, "create_code: more heavy columns than QCLDPC_MAX_HEAVY_COLS");
        }
        T.hcol_base[n_hcols] = (int16_t)c;
        T.col_kind[c] = (int16_t)n_hcols;
        n_hcols++;
    }
    T.n_hcols = n_hcols;

    // Circulant ids: heavy ones in input order, degree-1 ones in input order.
    std::vector<int> hid(n_circ, -1), did(n_circ, -1);
    int n_h = 0, n_d1 = 0;
    for (int h = 0; h < n_circ; h++) {
        if (col_count[circ_col[h]] == 1) {
            did[h] = n_d1;
            T.d1_shift[n_d1] = circ_shift[h];
            T.d1_row[n_d1] = (int16_t)circ_row[h];
            T.d1_col[n_d1] = (int16_t)circ_col[h];
            T.col_kind[circ_col[h]] = (int16_t)(-n_d1 - 2);
            n_d1++;
        } else {
            hid[h] = n_h++;
        }
    }
    T.n_h = n_h;
    T.n_d1 = n_d1;

    // Per-row table: heavy entries first, then degree-1 entries.
    int pos = 0, max_deg = 0;
    for (int r = 0; r < mb; r++) {
        T.row_ptr[r] = (uint16_t)pos;
        int nh = 0;
        for (int pass = 0; pass < 2; pass++) {
            for (int h = 0; h < n_circ; h++) {
                if (circ_row[h] != r) continue;
                bool heavy = hid[h] >= 0;
                if ((pass == 0) != heavy) continue;
                RowEnt e;
                e.shift = circ_shift[h];
                e.slot = heavy ? T.col_kind[circ_col[h]] : (int16_t)-1;
                e.id = (int16_t)(heavy ? hid[h] : did[h]);
                e.col = (int16_t)circ_col[h];
                e.pad = 0;
                T.rows[pos++] = e;
                if (heavy) nh++;
            }
        }
        T.row_nh[r] = (uint8_t)nh;
        max_deg = std::max(max_deg, pos - (int)T.row_ptr[r]);
    }
    T.row_ptr[mb] = (uint16_t)pos;
    T.max_row_deg = max_deg;
    // Check-node blocks visit rows in this order: rows of one shape (heavy
    // and degree-1 counts) are adjacent, so blocks resident together tend to
    // run the same code.
    {
        std::vector<int> order(mb);
        for (int r = 0; r < mb; r++) order[r] = r;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            const int da = T.row_ptr[a + 1] - T.row_ptr[a], db = T.row_ptr[b + 1] - T.row_ptr[b];
            if (T.row_nh[a] != T.row_nh[b]) return T.row_nh[a] < T.row_nh[b];
            return da < db;
        });
        for (int r = 0; r < mb; r++) T.row_order[r] = (uint8_t)order[r];
    }
    const int ZW = (Z + 31) / 32;
    for (int q = 0; q < pos; q++) {
        const RowEnt &e = T.rows[q];
        if (e.slot >= 0) {
            T.row_off_a[q] = e.slot * 2 * Z + e.shift;
            T.row_off_b[q] = e.id * Z;
        } else {
            T.row_off_a[q] = e.id * Z;
            T.row_off_b[q] = e.id * ZW;
        }
    }

    // Per-heavy-column table in input order.
    pos = 0;
    for (int s = 0; s < n_hcols; s++) {
        T.col_ptr[s] = (uint16_t)pos;
        for (int h = 0; h < n_circ; h++) {
            if (circ_col[h] != T.hcol_base[s]) continue;
            T.cols[pos].shift = circ_shift[h];
            T.cols[pos].id = hid[h];
            T.col_row[pos] = (int16_t)circ_row[h];
            pos++;
        }
    }
    T.col_ptr[n_hcols] = (uint16_t)pos;

    T.k = (int32_t)std::max<int64_t>(n - m, 0);
    code->n = n;
    code->m = m;
    code->k = T.k;
    code->n_edges = (int64_t)n_circ * Z;
    code->graph_cache = nullptr;
    code->last_ws = nullptr;
    code->last_frames = 0;
    code->last_soft = 0;
    // The tables are passed to kernels by value, so building a code needs no
    // device memory. The handle remembers the current device (-1 when no
    // device is visible: the code can then be inspected but not decoded).
    if (cudaGetDevice(&code->device) != cudaSuccess) {
        code->device = -1;
        (void)cudaGetLastError();
    }
    clear_error();
    *out = code;
    return QCLDPC_OK;
}

extern "C" void qcldpc_destroy_code(qcldpc_code *code) {
    if (!code) return;
    qc::destroy_graph_cache(code);
    delete code;
}

extern "C" int qcldpc_code_info(const qcldpc_code *code, int64_t *n, int64_t *m,
                                int64_t *k, int64_t *n_edges) {
    if (!code) return qc::fail(QCLDPC_E_INVAL, "code_info: code is NULL");
    if (n) *n = code->n;
    if (m) *m = code->m;
    if (k) *k = code->k;
    if (n_edges) *n_edges = code->n_edges;
    return QCLDPC_OK;
}
