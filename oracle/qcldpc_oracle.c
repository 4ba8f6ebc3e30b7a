/*
 * Plain FP64 CPU oracle for QC multi-edge LDPC reverse reconciliation.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this library. The CUDA
 * decoder never links, calls or reads anything here, and nothing here is
 * taken from the CUDA decoder: the two implementations share no code.
 *
 * Everything is written for clarity, not speed: edge lists are materialised,
 * every exclusive sum and product is recomputed from scratch, and all
 * floating point is IEEE double. Compile with -ffp-contract=off so that the
 * result does not depend on the host's fused multiply-add.
 *
 * Sources (arXiv 1702.07740, "Key reconciliation with LDPC codes for
 * long-distance quantum cryptography"):
 *   - QC expansion: Sec. III-C (quasi-cyclic codes). A base entry of value
 *     i becomes the identity shifted right by i-1; with shift s = i-1 row j
 *     of the block has its one at column (j+s) mod Z.
 *   - Bob's message M_i = (-1)^{C_i} Y_i and its d-dimensional form
 *     M = U Y: Sec. II-C ("Reverse reconciliation algorithm", "Multi-
 *     dimensional reconciliation").
 *   - Alice's division R = M X^{-1} = M X* / |X|^2 and the channel LLR
 *     Q = 2R / sigma_N^2: Sec. II-C and Step 1 of Algorithm 1.
 *   - Sum-product decoding: Algorithm 1 (Steps 1-5) with
 *     Phi(x) = -ln tanh(x/2), in syndrome (Slepian-Wolf) form.
 *
 * Readings where the paper is silent (listed with the design notes):
 *   - several circulants may share one base entry (their shifts differ);
 *   - the d-dim noise variance is d*sigma_Z^2/|X|^2 (|U|^2 = d);
 *   - octonions are built by Cayley-Dickson doubling with
 *     (p,q)(r,s) = (p r - conj(s) q, s p + q conj(r)), conj(p,q) = (conj p, -q);
 *   - syndrome form: every check message carries the extra sign (-1)^{s_c}
 *     and decoding stops when H C = s;
 *   - sgn(0) = +1; messages in both directions are clipped to [-clip, clip]
 *     (clip <= 0 disables clipping); every Phi argument is floored at xmin;
 *   - the stop test runs after iteration t when t >= et_start, and always
 *     after the last iteration;
 *   - layered schedule (not in the paper, which uses flooding): checks are
 *     split into layers visited in order within an iteration; the messages
 *     of one layer are computed together from the state at the layer's
 *     start, so a variable with several edges in one layer sees none of the
 *     layer's own new messages.
 *
 * Parity pins: see the test suite (tree exactness against brute-force MAP,
 * syndrome-sign symmetry, octonion identities, the printed d=2 noise form).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* QC expansion (Sec. III-C)                                                 */
/* ------------------------------------------------------------------------ */

/* Circulant h = (row r, column c, shift s) contributes, for every i in [0,Z),
 * the edge (check r*Z+i, variable c*Z + (i+s) mod Z). Edge number e = h*Z+i.
 * Returns 0, or -1 when an entry is out of range. */
int orc_expand(int mb, int nb, int Z, int nc, const int32_t *row,
               const int32_t *col, const int32_t *shift, int64_t *edge_cn,
               int64_t *edge_vn)
{
    for (int h = 0; h < nc; h++) {
        if (row[h] < 0 || row[h] >= mb || col[h] < 0 || col[h] >= nb ||
            shift[h] < 0 || shift[h] >= Z)
            return -1;
        for (int64_t i = 0; i < Z; i++) {
            int64_t e = (int64_t)h * Z + i;
            edge_cn[e] = (int64_t)row[h] * Z + i;
            edge_vn[e] = (int64_t)col[h] * Z + (i + shift[h]) % Z;
        }
    }
    return 0;
}

/* Syndrome s = H x (mod 2), one byte per bit. */
void orc_syndrome(int64_t m, int64_t n_edges, const int64_t *edge_cn,
                  const int64_t *edge_vn, const uint8_t *bits, uint8_t *syn)
{
    memset(syn, 0, (size_t)m);
    for (int64_t e = 0; e < n_edges; e++)
        syn[edge_cn[e]] ^= (uint8_t)(bits[edge_vn[e]] & 1u);
}

/* ------------------------------------------------------------------------ */
/* Cayley-Dickson algebra (Sec. II-C, multi-dimensional reconciliation)      */
/* ------------------------------------------------------------------------ */

static void cd_conj(const double *a, double *out, int d)
{
    out[0] = a[0];
    for (int i = 1; i < d; i++)
        out[i] = -a[i];
}

/* out = a b for d in {1,2,4,8}; out must not alias a or b. */
static void cd_mul(const double *a, const double *b, double *out, int d)
{
    if (d == 1) {
        out[0] = a[0] * b[0];
        return;
    }
    int h = d / 2;
    const double *p = a, *q = a + h, *r = b, *s = b + h;
    double sc[4], rc[4], t1[4], t2[4];
    cd_conj(s, sc, h);
    cd_conj(r, rc, h);
    /* low half: p r - conj(s) q */
    cd_mul(p, r, t1, h);
    cd_mul(sc, q, t2, h);
    for (int i = 0; i < h; i++)
        out[i] = t1[i] - t2[i];
    /* high half: s p + q conj(r) */
    cd_mul(s, p, t1, h);
    cd_mul(q, rc, t2, h);
    for (int i = 0; i < h; i++)
        out[h + i] = t1[i] + t2[i];
}

/* Exposed for the algebra tests. */
void orc_cd_mul(const double *a, const double *b, double *out, int d)
{
    cd_mul(a, b, out, d);
}

/* Bob's message: per block of d bits, U_j = (-1)^{c_{db+j}} and M = U Y. */
int orc_bob_message(int d, int64_t n, const double *y, const uint8_t *bits,
                    double *m)
{
    if (d != 1 && d != 2 && d != 4 && d != 8)
        return -1;
    if (n % d != 0)
        return -1;
    for (int64_t b = 0; b < n / d; b++) {
        double u[8], out[8];
        for (int j = 0; j < d; j++)
            u[j] = (bits[b * d + j] & 1u) ? -1.0 : 1.0;
        cd_mul(u, y + b * d, out, d);
        for (int j = 0; j < d; j++)
            m[b * d + j] = out[j];
    }
    return 0;
}

/* Alice's channel LLRs: R = (M conj(X)) / |X|^2, sigma_N^2 = d sigma_Z^2 /
 * |X|^2 with sigma_Z^2 = 1/snr, and Q = 2 R / sigma_N^2 (Step 1 of
 * Algorithm 1, extended to d dimensions). */
int orc_llr(int d, int64_t n, const double *x, const double *m, double snr,
            double *q)
{
    if (d != 1 && d != 2 && d != 4 && d != 8)
        return -1;
    if (n % d != 0 || !(snr > 0.0))
        return -1;
    double sigma_z2 = 1.0 / snr;
    for (int64_t b = 0; b < n / d; b++) {
        const double *xb = x + b * d;
        double xc[8], p[8];
        double norm2 = 0.0;
        for (int j = 0; j < d; j++)
            norm2 += xb[j] * xb[j];
        cd_conj(xb, xc, d);
        cd_mul(m + b * d, xc, p, d);
        double sigma_n2 = (double)d * sigma_z2 / norm2;
        for (int j = 0; j < d; j++) {
            double r = p[j] / norm2;
            q[b * d + j] = 2.0 * r / sigma_n2;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sum-product decoding (Algorithm 1), syndrome form, flooding schedule      */
/* ------------------------------------------------------------------------ */

/* Phi(x) = -ln tanh(x/2) = ln coth(x/2) = ln(1 + 2/(e^x - 1)), written as
 * log1p(2/expm1(x)): expm1 keeps small x exact and log1p keeps large x exact
 * (the form ln(1+e^-x) - ln(1-e^-x) loses the second term above x ~ 20). */
double orc_phi(double x)
{
    return log1p(2.0 / expm1(x));
}

static double sgn(double x) { return x < 0.0 ? -1.0 : 1.0; }

static double clip_msg(double x, double clip)
{
    if (clip <= 0.0)
        return x;
    if (x > clip)
        return clip;
    if (x < -clip)
        return -clip;
    return x;
}

/* Adjacency lists in edge order (= circulant order for a fixed node). */
typedef struct {
    int64_t *ptr; /* size count+1 */
    int64_t *edges;
} adj_t;

static int build_adj(int64_t count, int64_t n_edges, const int64_t *node_of,
                     adj_t *a)
{
    a->ptr = (int64_t *)calloc((size_t)count + 1, sizeof(int64_t));
    a->edges = (int64_t *)malloc((size_t)(n_edges > 0 ? n_edges : 1) *
                                 sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)count + 1, sizeof(int64_t));
    if (!a->ptr || !a->edges || !fill) {
        free(a->ptr);
        free(a->edges);
        free(fill);
        return -1;
    }
    for (int64_t e = 0; e < n_edges; e++)
        a->ptr[node_of[e] + 1]++;
    for (int64_t i = 0; i < count; i++)
        a->ptr[i + 1] += a->ptr[i];
    for (int64_t e = 0; e < n_edges; e++) {
        int64_t v = node_of[e];
        a->edges[a->ptr[v] + fill[v]++] = e;
    }
    free(fill);
    return 0;
}

static void free_adj(adj_t *a)
{
    free(a->ptr);
    free(a->edges);
}

/* One frame of syndrome-form sum-product decoding.
 *
 *   q[n]        channel LLRs Q_v = ln P(C_v=0)/P(C_v=1)
 *   syn[m]      syndrome bits s_c (0/1)
 *   max_iter    iterations t = 1..max_iter (0: decisions from Q only)
 *   et_start    the stop test H C = s runs after iteration t when
 *               t >= et_start, and always after the last iteration
 *   clip        clip level for every edge message (<= 0: none)
 *   xmin        floor for every Phi argument
 * Outputs:
 *   post[n]     posteriors L_v of the last iteration run
 *   chat[n]     hard decisions (1 iff L_v < 0)
 *   iters_out   the iteration the decoder stopped at
 *   conv_out    1 if H chat = syn
 * Returns 0, or -1 on allocation failure.
 */
int orc_decode(int64_t n, int64_t m, int64_t n_edges, const int64_t *edge_cn,
               const int64_t *edge_vn, const double *q, const uint8_t *syn,
               int max_iter, int et_start, double clip, double xmin,
               double *post, uint8_t *chat, int32_t *iters_out,
               int32_t *conv_out)
{
    adj_t cn, vn;
    if (build_adj(m, n_edges, edge_cn, &cn))
        return -1;
    if (build_adj(n, n_edges, edge_vn, &vn)) {
        free_adj(&cn);
        return -1;
    }
    size_t ne = (size_t)(n_edges > 0 ? n_edges : 1);
    double *l_vc = (double *)malloc(ne * sizeof(double)); /* VN -> CN */
    double *m_cv = (double *)malloc(ne * sizeof(double)); /* CN -> VN */
    if (!l_vc || !m_cv) {
        free(l_vc);
        free(m_cv);
        free_adj(&cn);
        free_adj(&vn);
        return -1;
    }

    /* Step 1: L_vc^(0) = Q_v on every edge; posterior of iteration 0 is Q. */
    for (int64_t e = 0; e < n_edges; e++)
        l_vc[e] = clip_msg(q[edge_vn[e]], clip);
    for (int64_t v = 0; v < n; v++) {
        post[v] = q[v];
        chat[v] = (uint8_t)(post[v] < 0.0);
    }

    int t = 0;
    int converged = 0;
    for (;;) {
        int test = (t == max_iter) || (t >= 1 && t >= et_start);
        if (test) {
            /* Step 4 (stop test): every check must satisfy
             * s_c + sum_{v in N(c)} chat_v = 0 (mod 2). */
            int ok = 1;
            for (int64_t c = 0; c < m && ok; c++) {
                unsigned par = syn[c] & 1u;
                for (int64_t k = cn.ptr[c]; k < cn.ptr[c + 1]; k++)
                    par ^= chat[edge_vn[cn.edges[k]]];
                if (par)
                    ok = 0;
            }
            if (ok) {
                converged = 1;
                break;
            }
        }
        if (t == max_iter)
            break;
        t++;

        /* Step 2: check-node update. For edge e = (c, v):
         * m_cv = (-1)^{s_c} prod_{v' != v} sgn(L_v'c)
         *        * Phi( max( sum_{v' != v} Phi(max(|L_v'c|, xmin)), xmin ) ). */
        for (int64_t c = 0; c < m; c++) {
            double ssign = (syn[c] & 1u) ? -1.0 : 1.0;
            for (int64_t k = cn.ptr[c]; k < cn.ptr[c + 1]; k++) {
                int64_t e = cn.edges[k];
                double sign = ssign;
                double sum = 0.0;
                for (int64_t k2 = cn.ptr[c]; k2 < cn.ptr[c + 1]; k2++) {
                    if (k2 == k)
                        continue;
                    double l = l_vc[cn.edges[k2]];
                    sign *= sgn(l);
                    sum += orc_phi(fmax(fabs(l), xmin));
                }
                m_cv[e] = clip_msg(sign * orc_phi(fmax(sum, xmin)), clip);
            }
        }

        /* Step 3: variable-node update.
         * L_vc = Q_v + sum_{c' != c} m_c'v,  L_v = Q_v + sum_c m_cv. */
        for (int64_t v = 0; v < n; v++) {
            double total = q[v];
            for (int64_t k = vn.ptr[v]; k < vn.ptr[v + 1]; k++)
                total += m_cv[vn.edges[k]];
            post[v] = total;
            chat[v] = (uint8_t)(total < 0.0); /* Step 4: 0 iff L_v >= 0 */
            for (int64_t k = vn.ptr[v]; k < vn.ptr[v + 1]; k++) {
                int64_t e = vn.edges[k];
                double ext = q[v];
                for (int64_t k2 = vn.ptr[v]; k2 < vn.ptr[v + 1]; k2++)
                    if (k2 != k)
                        ext += m_cv[vn.edges[k2]];
                l_vc[e] = clip_msg(ext, clip);
            }
        }
    }

    *iters_out = t;
    *conv_out = converged;
    free(l_vc);
    free(m_cv);
    free_adj(&cn);
    free_adj(&vn);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Layered schedule (extension; the paper decodes with flooding)            */
/* ------------------------------------------------------------------------ */

/* Sum-product decoding with the checks split into layers, layer[c] in
 * [0, n_layers). Iteration t visits layers 0, 1, ..., n_layers-1; for the
 * checks of layer l:
 *   L_vc = clip(Q_v + sum_{c' != c} m_c'v)   over the messages as they stand
 *          when layer l starts (edges of earlier layers already hold their
 *          iteration-t messages, edges of this and later layers still hold
 *          those of t-1; all messages start at 0);
 *   m_cv = the check rule of Step 2 on those L_vc, for every edge of the
 *          layer, written only after all of the layer's m_cv are computed.
 * After the last layer L_v = Q_v + sum_c m_cv gives the decisions, and the
 * stop test follows the same rule as orc_decode. With one layer this is
 * exactly orc_decode (same sums in the same order). */
int orc_decode_layered(int64_t n, int64_t m, int64_t n_edges, const int64_t *edge_cn,
                       const int64_t *edge_vn, const double *q, const uint8_t *syn,
                       int n_layers, const int32_t *layer, int max_iter, int et_start,
                       double clip, double xmin, double *post, uint8_t *chat,
                       int32_t *iters_out, int32_t *conv_out)
{
    adj_t cn, vn;
    if (n_layers < 1)
        return -1;
    for (int64_t c = 0; c < m; c++)
        if (layer[c] < 0 || layer[c] >= n_layers)
            return -1;
    if (build_adj(m, n_edges, edge_cn, &cn))
        return -1;
    if (build_adj(n, n_edges, edge_vn, &vn)) {
        free_adj(&cn);
        return -1;
    }
    size_t ne = (size_t)(n_edges > 0 ? n_edges : 1);
    double *l_vc = (double *)malloc(ne * sizeof(double));
    double *m_cv = (double *)calloc(ne, sizeof(double));
    double *m_new = (double *)malloc(ne * sizeof(double));
    if (!l_vc || !m_cv || !m_new) {
        free(l_vc);
        free(m_cv);
        free(m_new);
        free_adj(&cn);
        free_adj(&vn);
        return -1;
    }
    for (int64_t v = 0; v < n; v++) {
        post[v] = q[v];
        chat[v] = (uint8_t)(post[v] < 0.0);
    }

    int t = 0;
    int converged = 0;
    for (;;) {
        int test = (t == max_iter) || (t >= 1 && t >= et_start);
        if (test) {
            int ok = 1;
            for (int64_t c = 0; c < m && ok; c++) {
                unsigned par = syn[c] & 1u;
                for (int64_t k = cn.ptr[c]; k < cn.ptr[c + 1]; k++)
                    par ^= chat[edge_vn[cn.edges[k]]];
                if (par)
                    ok = 0;
            }
            if (ok) {
                converged = 1;
                break;
            }
        }
        if (t == max_iter)
            break;
        t++;

        for (int l = 0; l < n_layers; l++) {
            /* variable-to-check messages of the layer's edges */
            for (int64_t c = 0; c < m; c++) {
                if (layer[c] != l)
                    continue;
                for (int64_t k = cn.ptr[c]; k < cn.ptr[c + 1]; k++) {
                    int64_t e = cn.edges[k];
                    int64_t v = edge_vn[e];
                    double ext = q[v];
                    for (int64_t k2 = vn.ptr[v]; k2 < vn.ptr[v + 1]; k2++)
                        if (vn.edges[k2] != e)
                            ext += m_cv[vn.edges[k2]];
                    l_vc[e] = clip_msg(ext, clip);
                }
            }
            /* check-to-variable messages of the layer (Step 2) */
            for (int64_t c = 0; c < m; c++) {
                if (layer[c] != l)
                    continue;
                double ssign = (syn[c] & 1u) ? -1.0 : 1.0;
                for (int64_t k = cn.ptr[c]; k < cn.ptr[c + 1]; k++) {
                    int64_t e = cn.edges[k];
                    double sign = ssign;
                    double sum = 0.0;
                    for (int64_t k2 = cn.ptr[c]; k2 < cn.ptr[c + 1]; k2++) {
                        if (k2 == k)
                            continue;
                        double lv = l_vc[cn.edges[k2]];
                        sign *= sgn(lv);
                        sum += orc_phi(fmax(fabs(lv), xmin));
                    }
                    m_new[e] = clip_msg(sign * orc_phi(fmax(sum, xmin)), clip);
                }
            }
            /* commit the layer */
            for (int64_t c = 0; c < m; c++) {
                if (layer[c] != l)
                    continue;
                for (int64_t k = cn.ptr[c]; k < cn.ptr[c + 1]; k++)
                    m_cv[cn.edges[k]] = m_new[cn.edges[k]];
            }
        }

        /* posteriors and decisions (Steps 3-4) */
        for (int64_t v = 0; v < n; v++) {
            double total = q[v];
            for (int64_t k = vn.ptr[v]; k < vn.ptr[v + 1]; k++)
                total += m_cv[vn.edges[k]];
            post[v] = total;
            chat[v] = (uint8_t)(total < 0.0);
        }
    }

    *iters_out = t;
    *conv_out = converged;
    free(l_vc);
    free(m_cv);
    free(m_new);
    free_adj(&cn);
    free_adj(&vn);
    return 0;
}
