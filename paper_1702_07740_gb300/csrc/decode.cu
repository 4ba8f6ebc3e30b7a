// Syndrome-form sum-product decoding (arXiv 1702.07740, Algorithm 1) on the
// device: flooding schedule, FP32 messages, the iteration loop inside one
// CUDA graph (a conditional WHILE node), no host round trip per iteration.
//
// Data layout per frame f (all in the caller's workspace, frame-major):
//   msg  [n_h][Z]       check-to-variable messages m_cv of every heavy edge,
//                       indexed by (heavy circulant, check offset i)
//   L    [n_hcols][Z]   posterior L_v of every heavy variable node
//   phiq [n_d1][Z]      +-Phi(|Q_p|) of every degree-1 variable node, indexed
//                       by (degree-1 circulant, check offset); its message to
//                       the check never changes (Sec. III-D, long diagonal)
//   bits [2][n_d1][ZW]  hard decisions of the degree-1 nodes, double
//                       buffered by iteration parity (ZW = ceil(Z/32) words)
// Degree-1 edges therefore carry no per-iteration state: a check reads its
// diagonal neighbour's constant Phi value and decides that neighbour's bit
// itself (Step 4 of Algorithm 1 for degree-1 nodes).
//
// One iteration t is two streaming kernels plus a one-block control kernel:
//   cn_kernel   per check c (row r, offset i): L_vc = clip(L_v - m_cv(t-1)) for
//               heavy neighbours v = (col, (i+s) mod Z), Phi-domain exclusive
//               sums, m_cv(t) written back in place; decisions of the degree-1
//               neighbours of iteration t. It also evaluates the stop test of
//               iteration t-1 (H C(t-1) = s) from the L(t-1) values it reads
//               anyway, so the test costs no extra pass over memory.
//   ctrl_kernel freezes frames that passed the test (their L and bits of
//               iteration t-1 are kept: vn_kernel skips them) and sets the
//               graph's loop condition.
//   vn_kernel   per heavy variable v: L_v = Q_v + sum over its ~60 circulants
//               of m_cv, read at offsets (j - s) mod Z (coalesced, one wrap).
// A last pass (t = max_iter + 1) runs cn_kernel as a pure stop test.
//
// Phi(x) = -ln tanh(x/2) is evaluated in FP32 with the hardware ex2/lg2
// approximations and two short polynomials (see phi_f below); the FP32 path
// matches the FP64 oracle's posteriors to ~2e-5 relative after 50 iterations.
#include <algorithm>
#include <cmath>
#include <new>

#include "qcldpc_internal.cuh"

namespace {

using qc::Table;

constexpr int kThreads = 256;
constexpr int kCnVpt = 2;  // checks per thread (interleaved by kThreads)
constexpr int kVnVpt = 2;  // variable nodes per thread
constexpr int kCtrlThreads = 256;

// Per-call arguments and workspace pointers. Written into the workspace by
// the first graph node each call; every other node reads it from there.
struct Work {
    const float *llr;      // [F][n]
    const uint32_t *syn;   // [F][words_m]
    uint32_t *keys;        // [F][words_k]
    int32_t *conv;         // [F]
    int32_t *iters;        // [F]
    float *post;           // [F][n] or nullptr
    int32_t *t;            // iteration counter of the loop
    int32_t *active;       // [F]
    int32_t *fail;         // [F] stop-test failures of the current pass
    float *msg;            // [F][n_h][Z]
    float *L;              // [F][n_hcols][Z]
    float *phiq;           // [F][n_d1][Z]
    uint32_t *bits;        // [2][F][n_d1][ZW]
    float *post1;          // [2][F][n_d1][Z] (soft output only)
    int64_t n, words_m, words_k;
    int32_t n_frames, max_iter, et_start, soft, ZW;
    float clip, xmin;
};

// ---------------------------------------------------------------- Phi

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Polynomial pieces derived by paper_1702_07740_gb300/phi_fit.py.
constexpr float kG0 = 8.333332092e-02f;
constexpr float kG1 = -4.860660061e-03f;
constexpr float kG2 = 3.394155647e-04f;
constexpr float kG3 = -2.243584640e-05f;
constexpr float kA1 = 3.333292305e-01f;
constexpr float kA2 = 2.002381980e-01f;
constexpr float kA3 = 1.380910724e-01f;
constexpr float kA4 = 1.488138288e-01f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kLog2e = 1.4426950408889634f;

// Phi(x) = -ln tanh(x/2) = ln coth(x/2) for x > 0 (callers floor x).
//   x <= 1: ln(2/x) + ln(u coth u), u = x/2; the even second term is w G(w).
//   x >  1: 2 atanh(t), t = e^{-x}; 2 atanh(t) = 2 t A(t^2), A = 1 + v/3 + ...
// Both branches are evaluated (no divergence); max relative error ~4e-7 for
// x <= 30 (ex2/lg2 approximations included).
__device__ __forceinline__ float phi_f(float x) {
    const float w = x * x;
    const float g = fmaf(fmaf(fmaf(kG3, w, kG2), w, kG1), w, kG0);
    const float small = fmaf(w, g, kLn2 - kLn2 * lg2_approx(x));
    const float t = ex2_approx(-x * kLog2e);
    const float v = t * t;
    const float a = fmaf(fmaf(fmaf(fmaf(kA4, v, kA3), v, kA2), v, kA1), v, 1.0f);
    const float large = 2.0f * t * a;
    return x <= 1.0f ? small : large;
}

__device__ __forceinline__ float clampf(float x, float c) { return fminf(fmaxf(x, -c), c); }

// ------------------------------------------------------------ kernels

__global__ void args_kernel(Work w, Work *dst) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = w;
}

// Initial state: L = Q (heavy), phiq = +-Phi(|clip Q|) and the iteration-0
// decisions of the degree-1 nodes, frame flags, loop counter t = 1.
// The message arrays need no initialisation: iteration 1 reads m = 0.
__global__ void __launch_bounds__(kThreads) init_kernel(const __grid_constant__ Table T,
                                                        const Work *__restrict__ Wp) {
    const Work W = *Wp;
    const int Z = T.Z;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    // heavy posteriors
    const int64_t nL = (int64_t)W.n_frames * T.n_hcols * Z;
    for (int64_t e = tid; e < nL; e += nthreads) {
        const int64_t f = e / ((int64_t)T.n_hcols * Z);
        const int64_t rem = e - f * T.n_hcols * Z;
        const int hc = (int)(rem / Z), j = (int)(rem - (int64_t)hc * Z);
        W.L[e] = W.llr[f * W.n + (int64_t)T.hcol_base[hc] * Z + j];
    }
    // degree-1 nodes: one warp per (frame, circulant, 32-check word)
    const int lane = threadIdx.x & 31;
    const int64_t warp = tid >> 5, nwarps = nthreads >> 5;
    const int64_t nwords = (int64_t)W.n_frames * T.n_d1 * W.ZW;
    for (int64_t q = warp; q < nwords; q += nwarps) {
        const int64_t f = q / ((int64_t)T.n_d1 * W.ZW);
        const int64_t rem = q - f * T.n_d1 * W.ZW;
        const int k = (int)(rem / W.ZW), wd = (int)(rem - (int64_t)k * W.ZW);
        const int i = wd * 32 + lane;
        bool neg = false;
        if (i < Z) {
            const int col = T.d1_col[k];
            int vo = i + T.d1_shift[k];
            if (vo >= Z) vo -= Z;
            const float qv = W.llr[f * W.n + (int64_t)col * Z + vo];
            const float a = fmaxf(fminf(fabsf(qv), W.clip), W.xmin);
            const float p = phi_f(a);
            const size_t off = ((size_t)f * T.n_d1 + k) * Z + i;
            W.phiq[off] = qv < 0.0f ? -p : p;
            if (W.soft) W.post1[off] = qv;  // iteration-0 posterior, buffer 0
            neg = qv < 0.0f;
        }
        const uint32_t word = __ballot_sync(0xffffffffu, neg);
        if (lane == 0) W.bits[((size_t)f * T.n_d1 + k) * W.ZW + wd] = word;
    }
    for (int64_t f = tid; f < W.n_frames; f += nthreads) {
        W.active[f] = 1;
        W.fail[f] = 0;
        W.conv[f] = 0;
        W.iters[f] = 0;
    }
    if (tid == 0) *W.t = 1;
}

// Check-node pass of iteration t (see the file comment). MAXD bounds the row
// degree so that every per-edge array stays in registers.
template <int MAXD>
__global__ void __launch_bounds__(kThreads) cn_kernel(const __grid_constant__ Table T,
                                                      const Work *__restrict__ Wp) {
    const int f = blockIdx.y;
    if (Wp->active[f] == 0) return;  // block-uniform
    const int t = *Wp->t;
    const int max_iter = Wp->max_iter;
    const bool update = t <= max_iter;
    const bool check = (t == max_iter + 1) || (t >= 2 && t - 1 >= Wp->et_start);
    const int Z = T.Z;
    const int span = kThreads * kCnVpt;
    const int tiles = (Z + span - 1) / span;
    const int r = blockIdx.x / tiles;
    const int i0 = (blockIdx.x - r * tiles) * span + threadIdx.x;
    const int rp = T.row_ptr[r];
    const int deg = T.row_ptr[r + 1] - rp;
    const int nh = T.row_nh[r];
    const float clip = Wp->clip, xmin = Wp->xmin;
    const int ZW = Wp->ZW;
    const int64_t F = Wp->n_frames;
    float *__restrict__ msg = Wp->msg + (size_t)f * T.n_h * Z;
    const float *__restrict__ L = Wp->L + (size_t)f * T.n_hcols * Z;
    const float *__restrict__ phiq = Wp->phiq + (size_t)f * T.n_d1 * Z;
    uint32_t *__restrict__ bits_cur = Wp->bits + ((size_t)(t & 1) * F + f) * T.n_d1 * ZW;
    const uint32_t *__restrict__ bits_prev =
        Wp->bits + ((size_t)((t - 1) & 1) * F + f) * T.n_d1 * ZW;
    const uint32_t *__restrict__ syn = Wp->syn + (size_t)f * Wp->words_m;
    const bool soft = Wp->soft != 0;
    float *__restrict__ post1 = soft ? Wp->post1 + ((size_t)(t & 1) * F + f) * T.n_d1 * Z : nullptr;
    const float *__restrict__ llr = Wp->llr + (size_t)f * Wp->n;

    bool bad = false;
#pragma unroll 1
    for (int u = 0; u < kCnVpt; u++) {
        const int i = i0 + u * kThreads;
        const bool valid = i < Z;
        float phi[MAXD];
        uint32_t neg = 0;   // bit k: incoming L_vc of edge k is negative
        uint32_t sbit = 0;  // syndrome bit of this check
        uint32_t par = 0;   // parity of iteration t-1's decisions
#pragma unroll
        for (int k = 0; k < MAXD; k++) phi[k] = 0.0f;
        if (valid) {
            const int64_t c = (int64_t)r * Z + i;
            sbit = (__ldg(syn + (c >> 5)) >> (c & 31)) & 1u;
#pragma unroll
            for (int k = 0; k < MAXD; k++) {
                if (k >= deg) break;
                const qc::RowEnt e = T.rows[rp + k];
                if (k < nh) {
                    int vo = i + e.shift;
                    if (vo >= Z) vo -= Z;
                    const float lv = L[(size_t)e.slot * Z + vo];
                    par ^= lv < 0.0f ? 1u : 0u;
                    if (update) {
                        const float mo = t > 1 ? msg[(size_t)e.id * Z + i] : 0.0f;
                        const float lvc = clampf(lv - mo, clip);
                        phi[k] = phi_f(fmaxf(fabsf(lvc), xmin));
                        neg |= (lvc < 0.0f ? 1u : 0u) << k;
                    }
                } else {
                    par ^= (__ldg(bits_prev + (size_t)e.id * ZW + (i >> 5)) >> (i & 31)) & 1u;
                    if (update) {
                        const float p = __ldg(phiq + (size_t)e.id * Z + i);
                        phi[k] = fabsf(p);
                        neg |= (p < 0.0f ? 1u : 0u) << k;
                    }
                }
            }
            if (check && ((par ^ sbit) & 1u)) bad = true;
        }
        if (update) {
            // exclusive Phi sums by prefix/suffix (no subtraction: no cancellation)
            float pre[MAXD + 1], suf[MAXD + 1];
            pre[0] = 0.0f;
#pragma unroll
            for (int k = 0; k < MAXD; k++) pre[k + 1] = pre[k] + phi[k];
            suf[MAXD] = 0.0f;
#pragma unroll
            for (int k = MAXD - 1; k >= 0; k--) suf[k] = suf[k + 1] + phi[k];
            const uint32_t sgn_all = (sbit + __popc(neg)) & 1u;
#pragma unroll
            for (int k = 0; k < MAXD; k++) {
                if (k >= deg) break;
                const qc::RowEnt e = T.rows[rp + k];
                const float ex = fmaxf(pre[k] + suf[k + 1], xmin);
                const uint32_t negk = sgn_all ^ ((neg >> k) & 1u);  // sign of m_cv
                if (k < nh) {
                    if (valid) {
                        const float mag = fminf(phi_f(ex), clip);
                        msg[(size_t)e.id * Z + i] = negk ? -mag : mag;
                    }
                } else {
                    // degree-1 neighbour p: C_p = [Q_p + m_cp < 0]. Phi is
                    // decreasing, so |m_cp| > |Q_p| iff ex < Phi(|Q_p|) = phi[k].
                    const uint32_t qneg = (neg >> k) & 1u;
                    const bool dec = valid && ((ex < phi[k]) ? negk : qneg);
                    const uint32_t word = __ballot_sync(0xffffffffu, dec);
                    if ((threadIdx.x & 31) == 0 && valid)
                        bits_cur[(size_t)e.id * ZW + (i >> 5)] = word;
                    if (soft && valid) {
                        int vo = i + e.shift;
                        if (vo >= Z) vo -= Z;
                        const float mag = fminf(phi_f(ex), clip);
                        post1[(size_t)e.id * Z + i] =
                            llr[(size_t)e.col * Z + vo] + (negk ? -mag : mag);
                    }
                }
            }
        }
    }
    if (check) {
        if (__syncthreads_or(bad) && threadIdx.x == 0) Wp->fail[f] = 1;
    }
}

// Loop control, one block: apply the stop test of iteration t-1, count t up,
// and keep the WHILE node running while any frame is active.
__global__ void __launch_bounds__(kCtrlThreads) ctrl_kernel(const Work *__restrict__ Wp,
                                                            cudaGraphConditionalHandle handle) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    const Work W = *Wp;
    const int t = *W.t;
    const bool last = t == W.max_iter + 1;
    const bool checked = last || (t >= 2 && t - 1 >= W.et_start);
    int mine = 0;
    for (int f = threadIdx.x; f < W.n_frames; f += blockDim.x) {
        if (W.active[f]) {
            if (checked && W.fail[f] == 0) {
                W.conv[f] = 1;
                W.iters[f] = t - 1;
                W.active[f] = 0;
            } else if (last) {
                W.conv[f] = 0;
                W.iters[f] = W.max_iter;
                W.active[f] = 0;
            } else {
                mine = 1;
            }
        }
        W.fail[f] = 0;
    }
    if (mine) atomicOr(&any, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        *W.t = t + 1;
        cudaGraphSetConditional(handle, any ? 1u : 0u);
    }
}

// Variable-node pass: L_v = Q_v + sum_c m_cv for every heavy variable node.
__global__ void __launch_bounds__(kThreads) vn_kernel(const __grid_constant__ Table T,
                                                      const Work *__restrict__ Wp) {
    const int f = blockIdx.y;
    if (Wp->active[f] == 0) return;
    const int Z = T.Z;
    const int span = kThreads * kVnVpt;
    const int tiles = (Z + span - 1) / span;
    const int hc = blockIdx.x / tiles;
    const int j0 = (blockIdx.x - hc * tiles) * span + threadIdx.x;
    const float *__restrict__ msg = Wp->msg + (size_t)f * T.n_h * Z;
    const float *__restrict__ q = Wp->llr + (size_t)f * Wp->n + (size_t)T.hcol_base[hc] * Z;
    float *__restrict__ L = Wp->L + ((size_t)f * T.n_hcols + hc) * Z;
    float acc[kVnVpt];
#pragma unroll
    for (int u = 0; u < kVnVpt; u++) {
        const int j = j0 + u * kThreads;
        acc[u] = j < Z ? __ldg(q + j) : 0.0f;
    }
    const int ce = T.col_ptr[hc + 1];
#pragma unroll 4
    for (int k = T.col_ptr[hc]; k < ce; k++) {
        const qc::ColEnt e = T.cols[k];
        const float *__restrict__ mk = msg + (size_t)e.id * Z;
#pragma unroll
        for (int u = 0; u < kVnVpt; u++) {
            const int j = j0 + u * kThreads;
            int idx = j - e.shift;
            if (idx < 0) idx += Z;
            if (j < Z) acc[u] += mk[idx];
        }
    }
#pragma unroll
    for (int u = 0; u < kVnVpt; u++) {
        const int j = j0 + u * kThreads;
        if (j < Z) L[j] = acc[u];
    }
}

// Outputs: packed key bits C_v (v < k) and, for soft output, every posterior.
__global__ void __launch_bounds__(kThreads) final_kernel(const __grid_constant__ Table T,
                                                         const Work *__restrict__ Wp) {
    const Work W = *Wp;
    const int Z = T.Z;
    const int lane = threadIdx.x & 31;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t warp = tid >> 5, nwarps = nthreads >> 5;
    const int64_t nw = (int64_t)W.n_frames * W.words_k;
    for (int64_t q = warp; q < nw; q += nwarps) {
        const int64_t f = q / W.words_k;
        const int64_t wd = q - f * W.words_k;
        const int64_t v = wd * 32 + lane;
        bool dec = false;
        if (v < T.k) {
            const int c = (int)(v / Z), j = (int)(v - (int64_t)c * Z);
            const int kind = T.col_kind[c];
            if (kind >= 0) {
                dec = W.L[((size_t)f * T.n_hcols + kind) * Z + j] < 0.0f;
            } else {
                const int d = -kind - 2;
                int i = j - T.d1_shift[d];
                if (i < 0) i += Z;
                const int b = W.iters[f] & 1;
                const uint32_t word =
                    W.bits[(((size_t)b * W.n_frames + f) * T.n_d1 + d) * W.ZW + (i >> 5)];
                dec = (word >> (i & 31)) & 1u;
            }
        }
        const uint32_t word = __ballot_sync(0xffffffffu, dec);
        if (lane == 0) W.keys[f * W.words_k + wd] = word;
    }
    if (W.soft) {
        const int64_t total = (int64_t)W.n_frames * W.n;
        for (int64_t e = tid; e < total; e += nthreads) {
            const int64_t f = e / W.n;
            const int64_t v = e - f * W.n;
            const int c = (int)(v / Z), j = (int)(v - (int64_t)c * Z);
            const int kind = T.col_kind[c];
            float val;
            if (kind >= 0) {
                val = W.L[((size_t)f * T.n_hcols + kind) * Z + j];
            } else {
                const int d = -kind - 2;
                int i = j - T.d1_shift[d];
                if (i < 0) i += Z;
                const int b = W.iters[f] & 1;
                val = W.post1[(((size_t)b * W.n_frames + f) * T.n_d1 + d) * Z + i];
            }
            W.post[e] = val;
        }
    }
}

// ------------------------------------------------------------ host side

struct Layout {
    size_t work, t, active, fail, msg, L, phiq, bits, post1, total;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

Layout layout_of(const Table &T, int F, bool soft) {
    Layout o;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    const size_t Z = (size_t)T.Z, ZW = (Z + 31) / 32;
    o.work = take(sizeof(Work));
    o.t = take(sizeof(int32_t));
    o.active = take(sizeof(int32_t) * F);
    o.fail = take(sizeof(int32_t) * F);
    o.msg = take(sizeof(float) * F * T.n_h * Z);
    o.L = take(sizeof(float) * F * T.n_hcols * Z);
    o.phiq = take(sizeof(float) * F * T.n_d1 * Z);
    o.bits = take(sizeof(uint32_t) * 2 * F * T.n_d1 * ZW);
    o.post1 = soft ? take(sizeof(float) * 2 * F * T.n_d1 * Z) : 0;
    o.total = off;
    return o;
}

struct GraphCache {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t args_node = nullptr;
    void *ws = nullptr;
    int n_frames = 0;
    int soft = 0;
};

void free_cache(GraphCache *gc) {
    if (!gc) return;
    if (gc->exec) cudaGraphExecDestroy(gc->exec);
    if (gc->graph) cudaGraphDestroy(gc->graph);
    gc->exec = nullptr;
    gc->graph = nullptr;
}

int cn_blocks_x(const Table &T) {
    const int span = kThreads * kCnVpt;
    return T.mb * ((T.Z + span - 1) / span);
}

int vn_blocks_x(const Table &T) {
    const int span = kThreads * kVnVpt;
    return T.n_hcols * ((T.Z + span - 1) / span);
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

void *cn_kernel_for(int maxdeg) {
    if (maxdeg <= 4) return (void *)cn_kernel<4>;
    if (maxdeg <= 8) return (void *)cn_kernel<8>;
    return (void *)cn_kernel<16>;
}

cudaError_t add_kernel(cudaGraphNode_t *node, cudaGraph_t g, const cudaGraphNode_t *dep,
                       size_t ndep, void *func, dim3 grid, dim3 block, void **args) {
    cudaKernelNodeParams kp = {};
    kp.func = func;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    kp.extra = nullptr;
    return cudaGraphAddKernelNode(node, g, dep, ndep, &kp);
}

// Build and instantiate the decode graph for (code, frames, workspace).
int build_graph(const qcldpc_code *code, GraphCache *gc, int F, void *ws, bool soft,
                const Work &w0) {
    const Table &T = code->tab;
    const Layout lo = layout_of(T, F, soft);
    Work *dwork = reinterpret_cast<Work *>(static_cast<char *>(ws) + lo.work);
    cudaError_t err;
    cudaGraph_t g = nullptr;
    if ((err = cudaGraphCreate(&g, 0)) != cudaSuccess) return qc::cuda_fail(err, "decode: cudaGraphCreate");
    gc->graph = g;

    Work wcopy = w0;
    void *args_args[] = {&wcopy, &dwork};
    cudaGraphNode_t n_args, n_init, n_cond, n_final;
    if ((err = add_kernel(&n_args, g, nullptr, 0, (void *)args_kernel, dim3(1), dim3(32),
                          args_args)) != cudaSuccess)
        return qc::cuda_fail(err, "decode: add args node");

    Table tcopy = T;
    void *tab_args[] = {&tcopy, &dwork};
    const int init_blocks = sm_count() * 4;
    if ((err = add_kernel(&n_init, g, &n_args, 1, (void *)init_kernel, dim3(init_blocks),
                          dim3(kThreads), tab_args)) != cudaSuccess)
        return qc::cuda_fail(err, "decode: add init node");

    cudaGraphConditionalHandle handle;
    if ((err = cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault)) !=
        cudaSuccess)
        return qc::cuda_fail(err, "decode: cudaGraphConditionalHandleCreate");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if ((err = cudaGraphAddNode(&n_cond, g, &n_init, nullptr, 1, &cp)) != cudaSuccess)
        return qc::cuda_fail(err, "decode: add conditional node");
    cudaGraph_t body = cp.conditional.phGraph_out[0];

    cudaGraphNode_t n_cn, n_ctrl, n_vn;
    if ((err = add_kernel(&n_cn, body, nullptr, 0, cn_kernel_for(T.max_row_deg),
                          dim3(cn_blocks_x(T), F), dim3(kThreads), tab_args)) != cudaSuccess)
        return qc::cuda_fail(err, "decode: add check-node kernel");
    void *ctrl_args[] = {&dwork, &handle};
    if ((err = add_kernel(&n_ctrl, body, &n_cn, 1, (void *)ctrl_kernel, dim3(1),
                          dim3(kCtrlThreads), ctrl_args)) != cudaSuccess)
        return qc::cuda_fail(err, "decode: add control kernel");
    if ((err = add_kernel(&n_vn, body, &n_ctrl, 1, (void *)vn_kernel, dim3(vn_blocks_x(T), F),
                          dim3(kThreads), tab_args)) != cudaSuccess)
        return qc::cuda_fail(err, "decode: add variable-node kernel");

    if ((err = add_kernel(&n_final, g, &n_cond, 1, (void *)final_kernel, dim3(init_blocks),
                          dim3(kThreads), tab_args)) != cudaSuccess)
        return qc::cuda_fail(err, "decode: add output kernel");

    cudaGraphExec_t exec = nullptr;
    if ((err = cudaGraphInstantiate(&exec, g, 0)) != cudaSuccess)
        return qc::cuda_fail(err, "decode: cudaGraphInstantiate");
    gc->exec = exec;
    gc->args_node = n_args;
    gc->ws = ws;
    gc->n_frames = F;
    gc->soft = soft ? 1 : 0;
    return QCLDPC_OK;
}

int decode_impl(const qcldpc_code *code_c, const float *llr, const uint32_t *syn, int F,
                int max_iter, const qcldpc_params *p_in, uint32_t *keys, int32_t *conv,
                int32_t *iters, float *post, void *ws, size_t ws_bytes, cudaStream_t stream) {
    using namespace qc;
    qcldpc_code *code = const_cast<qcldpc_code *>(code_c);
    if (!code) return fail(QCLDPC_E_INVAL, "decode: code is NULL");
    qcldpc_params p;
    if (p_in) p = *p_in;
    else qcldpc_params_init(&p);
    const bool soft = post != nullptr;
    if (F < 0 || F > 65535) return fail(QCLDPC_E_INVAL, "decode: n_frames must be in [0, 65535]");
    if (max_iter < 0) return fail(QCLDPC_E_INVAL, "decode: max_iter must be >= 0");
    if (!(p.phi_floor > 0.0f) || p.schedule != 0 || p.msg_format != 0 || p.reserved[0] ||
        p.reserved[1])
        return fail(QCLDPC_E_INVAL, "decode: unsupported option (phi_floor > 0, flooding, FP32)");
    if (soft && p.soft_output != 1)
        return fail(QCLDPC_E_INVAL, "decode_soft: params->soft_output must be 1");
    if (F == 0) return QCLDPC_OK;
    if (!llr || !syn || !keys || !conv || !iters || !ws)
        return fail(QCLDPC_E_INVAL, "decode: NULL buffer");
    if (!aligned(ws, 256)) return fail(QCLDPC_E_ALIGN, "decode: workspace must be 256-byte aligned");
    if (!aligned(llr, 4) || !aligned(syn, 4) || !aligned(keys, 4) || !aligned(conv, 4) ||
        !aligned(iters, 4) || (post && !aligned(post, 4)))
        return fail(QCLDPC_E_ALIGN, "decode: buffers must be 4-byte aligned");
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return cuda_fail(err, "decode: cudaGetDevice");
    if (dev != code->device) return fail(QCLDPC_E_INVAL, "decode: current device differs from the code's device");

    const Table &T = code->tab;
    const Layout lo = layout_of(T, F, soft);
    if (ws_bytes < lo.total) return fail(QCLDPC_E_NOMEM, "decode: workspace too small");
    char *base = static_cast<char *>(ws);
    Work w;
    w.llr = llr;
    w.syn = syn;
    w.keys = keys;
    w.conv = conv;
    w.iters = iters;
    w.post = post;
    w.t = reinterpret_cast<int32_t *>(base + lo.t);
    w.active = reinterpret_cast<int32_t *>(base + lo.active);
    w.fail = reinterpret_cast<int32_t *>(base + lo.fail);
    w.msg = reinterpret_cast<float *>(base + lo.msg);
    w.L = reinterpret_cast<float *>(base + lo.L);
    w.phiq = reinterpret_cast<float *>(base + lo.phiq);
    w.bits = reinterpret_cast<uint32_t *>(base + lo.bits);
    w.post1 = soft ? reinterpret_cast<float *>(base + lo.post1) : nullptr;
    w.n = code->n;
    w.words_m = (code->m + 31) / 32;
    w.words_k = (code->k + 31) / 32;
    w.n_frames = F;
    w.max_iter = max_iter;
    w.et_start = p.et_start;
    w.soft = soft ? 1 : 0;
    w.ZW = (T.Z + 31) / 32;
    w.clip = p.clip > 0.0f ? p.clip : INFINITY;
    w.xmin = p.phi_floor;

    std::lock_guard<std::mutex> lock(code->mu);
    GraphCache *gc = static_cast<GraphCache *>(code->graph_cache);
    if (!gc) {
        gc = new (std::nothrow) GraphCache();
        if (!gc) return fail(QCLDPC_E_NOMEM, "decode: out of host memory");
        code->graph_cache = gc;
    }
    if (!gc->exec || gc->ws != ws || gc->n_frames != F || gc->soft != (soft ? 1 : 0)) {
        free_cache(gc);
        int st = build_graph(code, gc, F, ws, soft, w);
        if (st != QCLDPC_OK) {
            free_cache(gc);
            return st;
        }
    } else {
        Layout l2 = layout_of(T, F, soft);
        Work *dwork = reinterpret_cast<Work *>(base + l2.work);
        void *args_args[] = {&w, &dwork};
        cudaKernelNodeParams kp = {};
        kp.func = (void *)args_kernel;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.kernelParams = args_args;
        if ((err = cudaGraphExecKernelNodeSetParams(gc->exec, gc->args_node, &kp)) != cudaSuccess)
            return cuda_fail(err, "decode: cudaGraphExecKernelNodeSetParams");
    }
    if ((err = cudaGraphLaunch(gc->exec, stream)) != cudaSuccess)
        return cuda_fail(err, "decode: cudaGraphLaunch");
    clear_error();
    return QCLDPC_OK;
}

// Measurement support: put the decoder back into a mid-loop state (t = 2,
// every frame active, at least two iterations) so that a replayed check-node
// pass does a full message update.
__global__ void replay_prep_kernel(Work *Wp) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        *Wp->t = 2;
        if (Wp->max_iter < 2) Wp->max_iter = 2;
    }
    for (int f = tid; f < Wp->n_frames; f += gridDim.x * blockDim.x) Wp->active[f] = 1;
}

}  // namespace

namespace qc {
void destroy_graph_cache(qcldpc_code *code) {
    GraphCache *gc = static_cast<GraphCache *>(code->graph_cache);
    if (!gc) return;
    free_cache(gc);
    delete gc;
    code->graph_cache = nullptr;
}
}  // namespace qc

extern "C" size_t qcldpc_decode_workspace(const qcldpc_code *code, int n_frames,
                                          const qcldpc_params *p) {
    if (!code || n_frames < 0) return 0;
    const bool soft = p && p->soft_output == 1;
    return layout_of(code->tab, n_frames, soft).total;
}

extern "C" int qcldpc_decode(const qcldpc_code *code, const float *llr_dev,
                             const uint32_t *syn_dev, int n_frames, int max_iter,
                             const qcldpc_params *p, uint32_t *key_bits_dev,
                             int32_t *converged_dev, int32_t *iters_dev, void *workspace_dev,
                             size_t workspace_bytes, qcldpc_stream_t stream) {
    return decode_impl(code, llr_dev, syn_dev, n_frames, max_iter, p, key_bits_dev,
                       converged_dev, iters_dev, nullptr, workspace_dev, workspace_bytes,
                       (cudaStream_t)stream);
}

extern "C" int qcldpc_decode_soft(const qcldpc_code *code, const float *llr_dev,
                                  const uint32_t *syn_dev, int n_frames, int max_iter,
                                  const qcldpc_params *p, uint32_t *key_bits_dev,
                                  int32_t *converged_dev, int32_t *iters_dev,
                                  float *posterior_dev, void *workspace_dev,
                                  size_t workspace_bytes, qcldpc_stream_t stream) {
    if (!posterior_dev) return qc::fail(QCLDPC_E_INVAL, "decode_soft: posterior_dev is NULL");
    return decode_impl(code, llr_dev, syn_dev, n_frames, max_iter, p, key_bits_dev,
                       converged_dev, iters_dev, posterior_dev, workspace_dev, workspace_bytes,
                       (cudaStream_t)stream);
}

extern "C" int qcldpc_time_passes(const qcldpc_code *code_c, int n_frames, void *workspace_dev,
                                  size_t workspace_bytes, int reps, float *cn_ms, float *vn_ms,
                                  qcldpc_stream_t stream_) {
    using namespace qc;
    qcldpc_code *code = const_cast<qcldpc_code *>(code_c);
    if (!code || !workspace_dev || !cn_ms || !vn_ms || reps < 1 || n_frames < 1 ||
        n_frames > 65535)
        return fail(QCLDPC_E_INVAL, "time_passes: bad argument");
    cudaStream_t stream = (cudaStream_t)stream_;
    {
        std::lock_guard<std::mutex> lock(code->mu);
        GraphCache *gc = static_cast<GraphCache *>(code->graph_cache);
        if (!gc || !gc->exec || gc->ws != workspace_dev || gc->n_frames != n_frames)
            return fail(QCLDPC_E_INVAL,
                        "time_passes: no decode ran on this workspace with this frame count");
        const Layout lo = layout_of(code->tab, n_frames, gc->soft != 0);
        if (workspace_bytes < lo.total) return fail(QCLDPC_E_NOMEM, "time_passes: workspace too small");
        Work *dwork = reinterpret_cast<Work *>(static_cast<char *>(workspace_dev) + lo.work);
        cudaEvent_t ev[3];
        cudaError_t err = cudaSuccess;
        for (int i = 0; i < 3; i++)
            if ((err = cudaEventCreate(&ev[i])) != cudaSuccess) return cuda_fail(err, "time_passes: cudaEventCreate");
        const Table &T = code->tab;
        replay_prep_kernel<<<1, 256, 0, stream>>>(dwork);
        void *cn = cn_kernel_for(T.max_row_deg);
        void *args[] = {const_cast<Table *>(&T), &dwork};
        cudaEventRecord(ev[0], stream);
        for (int r = 0; r < reps && err == cudaSuccess; r++)
            err = cudaLaunchKernel(cn, dim3(cn_blocks_x(T), n_frames), dim3(kThreads), args, 0, stream);
        cudaEventRecord(ev[1], stream);
        for (int r = 0; r < reps && err == cudaSuccess; r++)
            err = cudaLaunchKernel((void *)vn_kernel, dim3(vn_blocks_x(T), n_frames), dim3(kThreads),
                                   args, 0, stream);
        cudaEventRecord(ev[2], stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(ev[2]);
        float a = 0.f, b = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&a, ev[0], ev[1]);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&b, ev[1], ev[2]);
        for (int i = 0; i < 3; i++) cudaEventDestroy(ev[i]);
        if (err != cudaSuccess) return cuda_fail(err, "time_passes");
        *cn_ms = a / reps;
        *vn_ms = b / reps;
    }
    clear_error();
    return QCLDPC_OK;
}
