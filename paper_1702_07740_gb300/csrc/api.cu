// Code construction, status reporting and option defaults of the qcldpc C ABI.
//
// QC expansion (arXiv 1702.07740, Sec. III-C): a base entry holding shift s
// stands for the Z x Z identity shifted right by s, so row i of the block has
// its one at column (i + s) mod Z. The expansion is never materialised: the
// kernels address messages as (circulant, offset) and compute (i + s) mod Z
// on the fly. This file classifies the base columns (degree-1 diagonal
// columns vs heavy columns) and lays out the per-row and per-column circulant
// tables the kernels read.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <new>
#include <type_traits>
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

// ---------------------------------------------------------------------------
// Device table arena: the code tables of every code live in one static device
// array (no device allocation at run time). A code takes a block on its first
// call that launches work and returns it in qcldpc_destroy_code.

namespace {

constexpr size_t kArenaBytes = size_t(64) << 20;
__device__ __align__(256) unsigned char g_table_arena[kArenaBytes];

std::mutex g_arena_mu;
std::vector<std::pair<size_t, size_t>> g_arena_used;  // (offset, bytes), sorted by offset

// First fit; returns false when no gap is large enough.
bool arena_take(size_t bytes, size_t *off) {
    std::lock_guard<std::mutex> lock(g_arena_mu);
    size_t at = 0;
    size_t i = 0;
    for (; i < g_arena_used.size(); i++) {
        if (g_arena_used[i].first - at >= bytes) break;
        at = g_arena_used[i].first + g_arena_used[i].second;
    }
    if (at + bytes > kArenaBytes) return false;
    g_arena_used.insert(g_arena_used.begin() + i, {at, bytes});
    *off = at;
    return true;
}

void arena_give(size_t off) {
    std::lock_guard<std::mutex> lock(g_arena_mu);
    for (size_t i = 0; i < g_arena_used.size(); i++)
        if (g_arena_used[i].first == off) {
            g_arena_used.erase(g_arena_used.begin() + i);
            return;
        }
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

template <typename V>
size_t bytes_of(const V &v) {
    return round256(std::max<size_t>(v.size(), 1) * sizeof(typename V::value_type));
}

}  // namespace

namespace qc {

int upload_tables(qcldpc_code *code) {
    std::lock_guard<std::mutex> lock(code->table_mu);
    if (code->arena_bytes) return QCLDPC_OK;
    const HostTable &H = code->host;
    const size_t total = bytes_of(H.row_ptr) + bytes_of(H.row_nh) + bytes_of(H.row_order) +
                         bytes_of(H.row_desc) + bytes_of(H.row_desc_ord) +
                         bytes_of(H.col_ptr) + bytes_of(H.hcol_base) + bytes_of(H.col_kind) +
                         bytes_of(H.rows) + bytes_of(H.row_off_a) + bytes_of(H.row_off_b) +
                         bytes_of(H.cols) + bytes_of(H.col_row) + bytes_of(H.d1_shift) +
                         bytes_of(H.d1_row) + bytes_of(H.d1_col);
    size_t off;
    if (!arena_take(total, &off))
        return fail(QCLDPC_E_NOMEM, "code tables: the device table arena (64 MiB) is full");
    unsigned char *base = nullptr;
    cudaError_t err = cudaGetSymbolAddress(reinterpret_cast<void **>(&base), g_table_arena);
    if (err != cudaSuccess) {
        arena_give(off);
        return cuda_fail(err, "code tables: cudaGetSymbolAddress");
    }
    // one host staging buffer, one copy
    std::vector<unsigned char> stage(total, 0);
    size_t pos = 0;
    Table &T = code->tab;
    auto put = [&](const auto &v, auto **dst) {
        using E = typename std::decay_t<decltype(v)>::value_type;
        if (!v.empty()) std::memcpy(stage.data() + pos, v.data(), v.size() * sizeof(E));
        *dst = reinterpret_cast<std::remove_pointer_t<decltype(dst)>>(base + off + pos);
        pos += bytes_of(v);
    };
    put(H.row_ptr, &T.row_ptr);
    put(H.row_nh, &T.row_nh);
    put(H.row_order, &T.row_order);
    put(H.row_desc, &T.row_desc);
    put(H.row_desc_ord, &T.row_desc_ord);
    put(H.col_ptr, &T.col_ptr);
    put(H.hcol_base, &T.hcol_base);
    put(H.col_kind, &T.col_kind);
    put(H.rows, &T.rows);
    put(H.row_off_a, &T.row_off_a);
    put(H.row_off_b, &T.row_off_b);
    put(H.cols, &T.cols);
    put(H.col_row, &T.col_row);
    put(H.d1_shift, &T.d1_shift);
    put(H.d1_row, &T.d1_row);
    put(H.d1_col, &T.d1_col);
    err = cudaMemcpy(base + off, stage.data(), total, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
        arena_give(off);
        std::memset(&T.row_ptr, 0, sizeof(T) - offsetof(Table, row_ptr));
        return cuda_fail(err, "code tables: cudaMemcpy");
    }
    code->arena_off = off;
    code->arena_bytes = total;
    return QCLDPC_OK;
}

void release_tables(qcldpc_code *code) {
    std::lock_guard<std::mutex> lock(code->table_mu);
    if (code->arena_bytes) arena_give(code->arena_off);
    code->arena_bytes = 0;
}

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
    p->cn_threads = 0;
    p->vn_nodes = 0;
    p->vn_split = 0;
    p->vn_pass = 0;
    p->frame_groups = 0;
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
    HostTable &H = code->host;
    code->arena_off = code->arena_bytes = 0;
    T.Z = Z;
    T.mb = mb;
    T.nb = nb;
    T.n_circ = n_circ;

    // Column classification: exactly one circulant -> degree-1 column.
    // (A column without circulants counts as heavy with none: its posterior
    // stays its channel LLR.)
    H.col_kind.assign(nb, 0);
    int n_hcols = 0;
    for (int c = 0; c < nb; c++) {
        if (col_count[c] == 1) continue;
        if (n_hcols >= kMaxHeavyCols) {
            delete code;
            return fail(QCLDPC_E_UNSUPPORTED, "create_code: more heavy columns than QCLDPC_MAX_HEAVY_COLS");
        }
        H.hcol_base.push_back(c);
        H.col_kind[c] = n_hcols;
        n_hcols++;
    }
    T.n_hcols = n_hcols;

    // Circulant ids: heavy ones in input order, degree-1 ones in input order.
    std::vector<int> hid(n_circ, -1), did(n_circ, -1);
    int n_h = 0, n_d1 = 0;
    for (int h = 0; h < n_circ; h++) {
        if (col_count[circ_col[h]] == 1) {
            did[h] = n_d1;
            H.d1_shift.push_back(circ_shift[h]);
            H.d1_row.push_back(circ_row[h]);
            H.d1_col.push_back(circ_col[h]);
            H.col_kind[circ_col[h]] = -n_d1 - 2;
            n_d1++;
        } else {
            hid[h] = n_h++;
        }
    }
    T.n_h = n_h;
    T.n_d1 = n_d1;

    // Per-row table: heavy entries first, then degree-1 entries.
    H.row_ptr.assign(mb + 1, 0);
    H.row_nh.assign(mb, 0);
    H.rows.reserve(n_circ);
    {
        std::vector<std::vector<int>> by_row(mb);
        for (int h = 0; h < n_circ; h++) by_row[circ_row[h]].push_back(h);
        int max_deg = 0;
        for (int r = 0; r < mb; r++) {
            H.row_ptr[r] = (int32_t)H.rows.size();
            int nh = 0;
            for (int pass = 0; pass < 2; pass++) {
                for (int h : by_row[r]) {
                    const bool heavy = hid[h] >= 0;
                    if ((pass == 0) != heavy) continue;
                    RowEnt e;
                    e.shift = circ_shift[h];
                    e.slot = heavy ? H.col_kind[circ_col[h]] : -1;
                    e.id = heavy ? hid[h] : did[h];
                    e.col = circ_col[h];
                    H.rows.push_back(e);
                    if (heavy) nh++;
                }
            }
            H.row_nh[r] = nh;
            max_deg = std::max(max_deg, (int)H.rows.size() - H.row_ptr[r]);
        }
        H.row_ptr[mb] = (int32_t)H.rows.size();
        T.max_row_deg = max_deg;
    }
    // Check-node blocks visit rows in this order: rows of one shape (heavy
    // and degree-1 counts) are adjacent, so blocks resident together tend to
    // run the same code.
    {
        std::vector<int> order(mb);
        for (int r = 0; r < mb; r++) order[r] = r;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            const int da = H.row_ptr[a + 1] - H.row_ptr[a], db = H.row_ptr[b + 1] - H.row_ptr[b];
            if (H.row_nh[a] != H.row_nh[b]) return H.row_nh[a] < H.row_nh[b];
            return da < db;
        });
        H.row_order.assign(order.begin(), order.end());
    }
    // Staging footprint of the widest exact-shape row.
    T.stage_rows_max = T.stage_words_max = 0;
    for (int r = 0; r < mb; r++) {
        const int nh = H.row_nh[r], nd = H.row_ptr[r + 1] - H.row_ptr[r] - nh;
        if (!exact_shape(nh, nd)) continue;
        T.stage_rows_max = std::max(T.stage_rows_max, 2 * nh + nd);
        T.stage_words_max = std::max(T.stage_words_max, nd);
    }
    const int ZW = (Z + 31) / 32;
    H.row_off_a.resize(H.rows.size());
    H.row_off_b.resize(H.rows.size());
    for (size_t q = 0; q < H.rows.size(); q++) {
        const RowEnt &e = H.rows[q];
        if (e.slot >= 0) {
            H.row_off_a[q] = e.slot * 2 * Z + e.shift;
            H.row_off_b[q] = e.id * Z;
        } else {
            H.row_off_a[q] = e.id * Z;
            H.row_off_b[q] = e.id * ZW;
        }
    }

    // Row descriptors, natural order and check-pass grid order.
    H.row_desc.resize(mb);
    for (int r = 0; r < mb; r++) {
        RowDesc &d = H.row_desc[r];
        std::memset(&d, 0, sizeof(d));
        d.r = r;
        d.rp = H.row_ptr[r];
        d.nh = H.row_nh[r];
        d.nd = H.row_ptr[r + 1] - H.row_ptr[r] - H.row_nh[r];
        for (int k = 0; k < kDescEnts && k < d.nh + d.nd; k++) {
            d.off_a[k] = H.row_off_a[d.rp + k];
            d.off_b[k] = H.row_off_b[d.rp + k];
        }
    }
    H.row_desc_ord.resize(mb);
    for (int y = 0; y < mb; y++) H.row_desc_ord[y] = H.row_desc[H.row_order[y]];

    // Per-heavy-column table in input order.
    H.col_ptr.assign(n_hcols + 1, 0);
    for (int sl = 0; sl < n_hcols; sl++) {
        H.col_ptr[sl] = (int32_t)H.cols.size();
        for (int h = 0; h < n_circ; h++) {
            if (circ_col[h] != H.hcol_base[sl]) continue;
            ColEnt ce;
            ce.shift = circ_shift[h];
            ce.id = hid[h];
            H.cols.push_back(ce);
            H.col_row.push_back(circ_row[h]);
        }
    }
    H.col_ptr[n_hcols] = (int32_t)H.cols.size();
    ColsInline &CI = code->cols_in;
    std::memset(&CI, 0, sizeof(CI));
    CI.ok = n_hcols <= kInlineHcols && (int)H.cols.size() <= kInlineCols;
    if (CI.ok) {
        for (int sl = 0; sl <= n_hcols; sl++) CI.col_ptr[sl] = H.col_ptr[sl];
        for (size_t q = 0; q < H.cols.size(); q++) CI.cols[q] = H.cols[q];
    }

    T.k = (int32_t)std::max<int64_t>(n - m, 0);
    code->n = n;
    code->m = m;
    code->k = T.k;
    code->n_edges = (int64_t)n_circ * Z;
    code->graph_cache = nullptr;
    code->last_ws = nullptr;
    code->last_frames = 0;
    code->last_soft = 0;
    // Building a code needs no device: the tables go to the device table
    // arena on the first call that launches work. The handle remembers the
    // current device (-1 when no device is visible: the code can then be
    // inspected but not decoded).
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
    qc::purge_multi_graphs(code);
    qc::release_tables(code);
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
