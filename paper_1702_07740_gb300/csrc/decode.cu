// Syndrome-form sum-product decoding (arXiv 1702.07740, Algorithm 1) on the
// device: flooding schedule, FP32 messages, the iteration loop inside one
// CUDA graph (a conditional WHILE node), no host round trip per iteration.
//
// Data layout per frame f (all in the caller's workspace, frame-major):
//   msg  [n_h][Z]       check-to-variable messages m_cv of every heavy edge,
//                       indexed by (heavy circulant, check offset i)
//   L    [n_hcols][2Z]  posterior L_v of every heavy variable node, stored
//                       twice in a row so reads at (i + s) need no wrap
//   phiq [n_d1][Z]      +-Phi(|Q_p|) of every degree-1 variable node, indexed
//                       by (degree-1 circulant, check offset); its message to
//                       the check never changes (Sec. III-C, long diagonal)
//   bits [2][n_d1][ZW]  hard decisions of the degree-1 nodes, double
//                       buffered by iteration parity (ZW = ceil(Z/32) words)
// Every array carries kSlack elements of padding at its end, so that lanes
// past the last check of a row may load without a bounds test (their
// results are never stored).
// Degree-1 edges therefore carry no per-iteration state: a check reads its
// diagonal neighbour's constant Phi value and decides that neighbour's bit
// itself (Step 4 of Algorithm 1 for degree-1 nodes).
//
// One iteration t is two streaming kernels plus a one-block control kernel:
//   cn_tma_kernel per check c (row r, offset i): L_vc = clip(L_v - m_cv(t-1)) for
//               heavy neighbours v = (col, (i+s) mod Z), Phi-domain exclusive
//               sums, m_cv(t) written back in place; decisions of the degree-1
//               neighbours of iteration t. It also evaluates the stop test of
//               iteration t-1 (H C(t-1) = s) from the L(t-1) values it reads
//               anyway, so the test costs no extra pass over memory.
//   ctrl_kernel freezes frames that passed the test (their L and bits of
//               iteration t-1 are kept: vn_kernel skips them) and sets the
//               graph's loop condition.
//   vn_kernel   per heavy variable v: L_v = Q_v + sum over its ~60 circulants
//               of m_cv, read at offsets (j - s) mod Z (coalesced, one wrap),
//               as two interleaved partial sums added in a fixed order.
// A last pass (t = max_iter + 1) runs cn_tma_kernel as a pure stop test.
// The decode graph's WHILE body holds four flooding iterations (passes of
// frames that already stopped exit at once). Within it every pass hangs off
// its predecessor by a programmatic edge: it is scheduled while the
// predecessor drains and waits for its results on the device.
//
// Layered schedule (an extension; schedule = 1): the base rows form G groups
// visited in order. An iteration is a stop-test pass (cn_tma_kernel, test
// only), the control kernel, then per group the group's check pass (messages
// of iteration t written to the other of two buffers, next to those of t-1)
// and lvn_kernel, which adds the group's message changes to the posteriors.
//
// All call arguments travel as one __grid_constant__ parameter (Work), so
// they sit in the constant bank as warp-uniform operands; instantiated graphs
// are cached per distinct argument set.
//
// Units: inside the decoder every LLR is kept in base 2, y = x log2(e) for a
// natural LLR x (L, messages, Phi values, clip and floor). The rule is the
// same in these units with Phi replaced by psi(y) = log2 coth(y ln2 / 2) (see
// psi_f), whose exponentials the hardware ex2/lg2 evaluate without argument
// scaling. Channel LLRs come in and posteriors go out in natural units.
//
// psi is evaluated in FP32 with the ex2/lg2 approximations and two short
// polynomials; the FP32 path matches the FP64 oracle's posteriors to ~2e-5
// relative after 50 iterations.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "qcldpc_internal.cuh"

#include "decode_common.cuh"

namespace {
// ------------------------------------------------------------ kernels

// Initial state: L = Q (heavy), phiq = +-Phi(|clip Q|) and the iteration-0
// decisions of the degree-1 nodes, frame flags, loop counter t = 1.
// The message arrays need no initialisation: iteration 1 reads m = 0.
__global__ void __launch_bounds__(kThreads) init_kernel(const __grid_constant__ Table T,
                                                        const __grid_constant__ Work W) {
    const int Z = T.Z;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    // heavy posteriors in base-2 units (-0 -> +0 so that sgn(0) = +1 everywhere)
    const int64_t nL = (int64_t)W.n_frames * T.n_hcols * Z;
    for (int64_t e = tid; e < nL; e += nthreads) {
        const int64_t f = e / ((int64_t)T.n_hcols * Z);
        const int64_t rem = e - f * T.n_hcols * Z;
        const int hc = (int)(rem / Z), j = (int)(rem - (int64_t)hc * Z);
        const float qv = W.llr[f * W.n + (int64_t)T.hcol_base[hc] * Z + j] * kLog2e + 0.0f;
        float *row = W.L + ((size_t)f * T.n_hcols + hc) * 2 * Z;
        row[j] = qv;
        row[j + Z] = qv;
        if (W.accum) {
            int32_t *a = W.acc + ((size_t)f * T.n_hcols + hc) * 2 * Z;
            a[j] = 0;
            a[j + Z] = 0;
        }
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
            int vo = i + T.d1_shift[k];
            if (vo >= Z) vo -= Z;
            const float qv = W.llr[f * W.n + (int64_t)T.d1_col[k] * Z + vo];
            const float a = fmaxf(fminf(fabsf(qv) * kLog2e, W.clip), W.xmin);
            const float p = psi_f(a);
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
        W.t[f] = 1;
    }
    if (tid == 0) *W.err = 0;
}

// Loop control, one block: apply each frame's stop test of its iteration
// t-1, count running frames on, and (inside the decode graph) keep the WHILE
// node running while any frame is active. Frames carry their own iteration
// counter, so frames loaded at different times (pools) share the passes.
template <bool kInGraph>
__global__ void __launch_bounds__(kCtrlThreads) ctrl_kernel(const __grid_constant__ Work W,
                                                            cudaGraphConditionalHandle handle) {
    __shared__ int any;
    pdl_wait();  // the check pass's flags are complete and visible
    pdl_launch_dependents();
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    const bool failed = *W.err != 0;  // a staged copy never completed: stop, flag -1
    for (int f = threadIdx.x; f < W.n_frames; f += blockDim.x) {
        if (W.active[f]) {
            const int t = W.t[f];
            const bool last = t == W.max_iter + 1;
            const bool checked = last || (t >= 2 && t - 1 >= W.et_start);
            bool stop = true;
            if (failed) {
                W.conv[f] = -1;
                W.iters[f] = t - 1;
            } else if (checked && W.fail[f] == 0) {
                W.conv[f] = 1;
                W.iters[f] = t - 1;
            } else if (last) {
                W.conv[f] = 0;
                W.iters[f] = W.max_iter;
            } else {
                stop = false;
                W.t[f] = t + 1;
            }
            if (stop) {
                W.active[f] = 0;
                if (W.state) W.state[f] = 2;
            } else {
                any = 1;
            }
        }
        W.fail[f] = 0;
    }
    if (kInGraph) {
        __syncthreads();
        if (threadIdx.x == 0) cudaGraphSetConditional(handle, any ? 1u : 0u);
    }
}

// Variable-node pass: L_v = Q_v + sum_c m_cv for every heavy variable node.
// Grid (tile, heavy column, frame). Lanes past the end of the column read
// message padding (never stored); the channel LLRs, the caller's buffer, are
// read only in range.
// A node's sum is kVnParts independent partial sums, part p over the
// column's circulants p, p + kVnParts, ... in order (part 0 starts from
// Q_v), added in part order at the end. With S = 1 a thread keeps every part
// of its nodes (independent chains hide load latency); with S = kVnParts the
// block's threads form S groups over the same kThreads / S nodes, group g
// computes part g, and group 0 adds the others' parts from shared memory in
// the same order. Both forms give the same bits, so the launch picks S by
// batch size and a frame's result never depends on its batch.
template <typename M, int VPT, int S>
__global__ void __launch_bounds__(kThreads) vn_kernel(const __grid_constant__ Table T,
                                                      const __grid_constant__ Work W,
                                                      const __grid_constant__ qc::ColsInline C) {
    constexpr int P = kVnParts, G = kThreads / S, NP = P / S;  // parts held per thread
    static_assert(S == 1 || S == P, "a thread holds one part or all of them");
    pdl_wait();  // the control step's flags are complete and visible
    pdl_launch_dependents();  // the next iteration's check pass may be scheduled; it waits for this pass
    const int f = blockIdx.z;
    if (W.active[f] == 0) return;
    const int Z = T.Z;
    const int hc = blockIdx.y;
    const int g = S == 1 ? 0 : (int)threadIdx.x / G;
    const int lt = (int)threadIdx.x - g * G;
    const int j0 = blockIdx.x * (G * VPT) + lt;
    const M *__restrict__ msg = static_cast<const M *>(W.msg) + (size_t)f * T.n_h * Z;
    const float *__restrict__ q = W.llr + (size_t)f * W.n + (size_t)T.hcol_base[hc] * Z;
    float *__restrict__ L = W.L + ((size_t)f * T.n_hcols + hc) * 2 * Z;
    float acc[VPT][NP];
#pragma unroll
    for (int u = 0; u < VPT; u++) {
        const int j = j0 + u * G;
#pragma unroll
        for (int i = 0; i < NP; i++) acc[u][i] = (g == 0 && i == 0 && j < Z) ? __ldg(q + j) * kLog2e : 0.0f;
    }
    // add circulant (shift, id) to the thread's part slot i
    auto add = [&](int shift, int id, int i) {
        const M *__restrict__ mk = msg + id * Z;
#pragma unroll
        for (int u = 0; u < VPT; u++) {
            int idx = j0 + u * G - shift;
            if (idx < 0) idx += Z;
            acc[u][i] += Codec<M>::dec(mk[idx], W);
        }
    };
    if (C.ok) {
        // the column's circulants from the inline copy (constant bank):
        // whole steps of P circulants, then the remainder
        const int cb = C.col_ptr[hc], ce = C.col_ptr[hc + 1];
        int k = cb;
#pragma unroll kVnUnroll
        for (; k + P <= ce; k += P) {
#pragma unroll
            for (int i = 0; i < NP; i++) {
                const qc::ColEnt e = C.cols[k + g + i * S];
                add(e.shift, e.id, i);
            }
        }
#pragma unroll
        for (int i = 0; i < NP; i++) {
            if (k + g + i * S < ce) {
                const qc::ColEnt e = C.cols[k + g + i * S];
                add(e.shift, e.id, i);
            }
        }
    } else {
    // the column's circulants (shift, id), staged in shared memory in chunks
    // of kColChunk (a multiple of P, so a chunk offset keeps the part of k)
    __shared__ int2 s_cols[kColChunk];
    const int cb = T.col_ptr[hc], ce = T.col_ptr[hc + 1];
    for (int base = cb; base < ce; base += kColChunk) {
        const int cnt = min(kColChunk, ce - base);
        __syncthreads();  // the previous chunk is consumed
        if ((int)threadIdx.x < cnt)
            s_cols[threadIdx.x] = __ldg(reinterpret_cast<const int2 *>(T.cols) + base + threadIdx.x);
        __syncthreads();
        int kk = 0;
#pragma unroll kVnUnrollStaged
        for (; kk + P <= cnt; kk += P) {
#pragma unroll
            for (int i = 0; i < NP; i++) {
                const int2 e = s_cols[kk + g + i * S];
                add(e.x, e.y, i);
            }
        }
#pragma unroll
        for (int i = 0; i < NP; i++) {
            if (kk + g + i * S < cnt) {
                const int2 e = s_cols[kk + g + i * S];
                add(e.x, e.y, i);
            }
        }
    }
    }
    float tot[VPT];
    if constexpr (S == 1) {
#pragma unroll
        for (int u = 0; u < VPT; u++) {
            tot[u] = acc[u][0];
#pragma unroll
            for (int p = 1; p < P; p++) tot[u] += acc[u][p];
        }
    } else {
        __shared__ float s_part[P - 1][G * VPT];
        if (g > 0) {
#pragma unroll
            for (int u = 0; u < VPT; u++) s_part[g - 1][u * G + lt] = acc[u][0];
        }
        __syncthreads();
        if (g > 0) return;
#pragma unroll
        for (int u = 0; u < VPT; u++) {
            tot[u] = acc[u][0];
#pragma unroll
            for (int p = 1; p < P; p++) tot[u] += s_part[p - 1][u * G + lt];
        }
    }
#pragma unroll
    for (int u = 0; u < VPT; u++) {
        const int j = j0 + u * G;
        if (j < Z) {
            float lvj = tot[u];
            lvj += 0.0f;  // -0 -> +0: sgn(0) = +1 everywhere
            L[j] = lvj;
            L[j + Z] = lvj;
        }
    }
}

// Variable pass of flooding with accumulated posteriors (accum = 1): for
// every heavy node v = (column hc, j), L_v = Q_v + acc_inv (acc[j] +
// acc[j + Z]), the exact integer sum of the fixed-point messages the check
// pass just added, written twice (j and j + Z); both accumulator words are
// cleared for the next iteration. Frames that stopped keep the posteriors of
// their last test. Grid (tile of kPostVpt * kThreads nodes, heavy column,
// frame).
// The words are read and cleared with atomic exchanges, which the L2 serves
// where the reductions landed: on GB300 plain loads of words that many SMs
// have just reduced into took more than twice as long (18 us against 7.5 us
// for 16 frames of the n = 10^6 code, measured in isolation).
constexpr int kPostVpt = 2;
// PAIR (even Z): a thread takes adjacent nodes j, j + 1 (j even) with one
// 64-bit exchange per accumulator half, and vector loads and stores.
template <bool PAIR>
__global__ void __launch_bounds__(kThreads) post_kernel(const __grid_constant__ Table T,
                                                        const __grid_constant__ Work W) {
    pdl_wait();  // the control step's flags (and the check pass's sums) are complete and visible
    pdl_launch_dependents();  // the next iteration's check pass may be scheduled; it waits for this pass
    const int f = blockIdx.z;
    if (W.active[f] == 0) return;
    const int Z = T.Z;
    const int hc = blockIdx.y;
    const float *__restrict__ q = W.llr + (size_t)f * W.n + (size_t)T.hcol_base[hc] * Z;
    float *__restrict__ L = W.L + ((size_t)f * T.n_hcols + hc) * 2 * Z;
    int32_t *__restrict__ a = W.acc + ((size_t)f * T.n_hcols + hc) * 2 * Z;
    constexpr int P = PAIR ? 2 : 1;  // nodes per exchange
#pragma unroll
    for (int u = 0; u < kPostVpt; u++) {
        const int j = P * ((blockIdx.x * kPostVpt + u) * kThreads + threadIdx.x);
        if (j >= Z) continue;
        if constexpr (PAIR) {
            // exchanges of the 8-byte words (a[j], a[j+1]) and (a[j+Z], a[j+Z+1])
            unsigned long long *a2 = reinterpret_cast<unsigned long long *>(a + j);
            unsigned long long *b2 = reinterpret_cast<unsigned long long *>(a + j + Z);
            const unsigned long long x = atomicExch(a2, 0ull), y = atomicExch(b2, 0ull);
            const int s0 = (int)(uint32_t)x + (int)(uint32_t)y;
            const int s1 = (int)(uint32_t)(x >> 32) + (int)(uint32_t)(y >> 32);
            const float2 qq = __ldg(reinterpret_cast<const float2 *>(q + j));
            float2 lv;
            lv.x = fmaf((float)s0, W.acc_inv, qq.x * kLog2e) + 0.0f;  // -0 -> +0
            lv.y = fmaf((float)s1, W.acc_inv, qq.y * kLog2e) + 0.0f;
            *reinterpret_cast<float2 *>(L + j) = lv;
            *reinterpret_cast<float2 *>(L + j + Z) = lv;
        } else {
            const int sum = atomicExch(a + j, 0) + atomicExch(a + j + Z, 0);
            const float lvj = fmaf((float)sum, W.acc_inv, __ldg(q + j) * kLog2e) + 0.0f;  // -0 -> +0
            L[j] = lvj;
            L[j + Z] = lvj;
        }
    }
}

// The accumulated-posterior variable pass for a code: kernel and grid.
void *post_func(const Table &T) {
    return T.Z % 2 == 0 ? (void *)post_kernel<true> : (void *)post_kernel<false>;
}
dim3 post_grid(const Table &T, int F) {
    const int span = kThreads * kPostVpt * (T.Z % 2 == 0 ? 2 : 1);
    return dim3((unsigned)((T.Z + span - 1) / span), (unsigned)(T.n_hcols > 0 ? T.n_hcols : 1), (unsigned)F);
}

// Layered schedule, posterior update of one row group: for every heavy
// variable v, L_v += sum over the group's circulants of v's column of
// (m_cv(t) - m_cv(t-1)), read at (j - s) mod Z from the two message buffers
// (m(t-1) = 0 at t = 1). t is the iteration the group pass just computed.
template <typename M>
__global__ void __launch_bounds__(kThreads) lvn_kernel(const __grid_constant__ Table T,
                                                       const __grid_constant__ Work W) {
    const int f = blockIdx.z;
    if (W.active[f] == 0) return;
    const int t = W.t[f] - 1;
    const int Z = T.Z;
    const int hc = blockIdx.y;
    const int j0 = blockIdx.x * (kThreads * kVnVpt) + threadIdx.x;
    const M *__restrict__ mnew = static_cast<const M *>(W.msg) + (t & 1) * W.msg_buf + (size_t)f * T.n_h * Z;
    const M *__restrict__ mold = static_cast<const M *>(W.msg) + ((t - 1) & 1) * W.msg_buf + (size_t)f * T.n_h * Z;
    float d[kVnVpt];
#pragma unroll
    for (int u = 0; u < kVnVpt; u++) d[u] = 0.0f;
    bool touched = false;
    const int ce = T.col_ptr[hc + 1];
    for (int k = T.col_ptr[hc]; k < ce; k++) {
        const int row = T.col_row[k];
        if (row < W.lrow0 || row >= W.lrow0 + W.lrows) continue;  // uniform
        touched = true;
        const qc::ColEnt e = T.cols[k];
        const M *__restrict__ nk = mnew + e.id * Z;
        const M *__restrict__ ok = mold + e.id * Z;
#pragma unroll
        for (int u = 0; u < kVnVpt; u++) {
            int idx = j0 + u * kThreads - e.shift;
            if (idx < 0) idx += Z;
            d[u] += Codec<M>::dec(nk[idx], W) - (t > 1 ? Codec<M>::dec(ok[idx], W) : 0.0f);
        }
    }
    if (!touched) return;
    float *__restrict__ L = W.L + ((size_t)f * T.n_hcols + hc) * 2 * Z;
#pragma unroll
    for (int u = 0; u < kVnVpt; u++) {
        const int j = j0 + u * kThreads;
        if (j < Z) {
            const float lvj = L[j] + d[u] + 0.0f;  // -0 -> +0
            L[j] = lvj;
            L[j + Z] = lvj;
        }
    }
}

// Outputs: packed key bits C_v (v < k) and, for soft output, every posterior.
__global__ void __launch_bounds__(kThreads) final_kernel(const __grid_constant__ Table T,
                                                         const __grid_constant__ Work W) {
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
                dec = W.L[((size_t)f * T.n_hcols + kind) * 2 * Z + j] < 0.0f;
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
                val = W.L[((size_t)f * T.n_hcols + kind) * 2 * Z + j] * kLn2;
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

// Measurement support: put the decoder back into a mid-loop state (t = 2,
// every frame active) so that a replayed check-node pass does a full update.
__global__ void replay_prep_kernel(const __grid_constant__ Work W) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    for (int f = tid; f < W.n_frames; f += gridDim.x * blockDim.x) {
        W.active[f] = 1;
        W.t[f] = 2;
    }
}

// ------------------------------------------------------------ host side

struct Layout {
    size_t t, err, active, fail, msg, L, acc, phiq, bits, post1, total;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

size_t msg_elem_size(int fmt) { return fmt == 2 ? 1 : fmt == 1 ? 2 : 4; }

Layout layout_of(const Table &T, int F, bool soft, int fmt, bool layered = false) {
    Layout o;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    // element counts in size_t (F up to 65535 times a frame's arrays)
    const size_t Z = (size_t)T.Z, ZW = (Z + 31) / 32, Fs = (size_t)F;
    const size_t nh = (size_t)T.n_h, nhc = (size_t)T.n_hcols, nd1 = (size_t)T.n_d1;
    o.t = take(sizeof(int32_t) * Fs);
    o.err = take(sizeof(int32_t));
    o.active = take(sizeof(int32_t) * Fs);
    o.fail = take(sizeof(int32_t) * Fs);
    o.msg = take(msg_elem_size(fmt) * ((layered ? 2 : 1) * Fs * nh * Z + kSlack));
    o.L = take(sizeof(float) * (Fs * nhc * 2 * Z + kSlack));
    o.acc = layered ? 0 : take(sizeof(int32_t) * (Fs * nhc * 2 * Z + kSlack));
    o.phiq = take(sizeof(float) * (Fs * nd1 * Z + kSlack));
    o.bits = take(sizeof(uint32_t) * (2 * Fs * nd1 * ZW + kSlack));
    o.post1 = soft ? take(sizeof(float) * (2 * Fs * nd1 * Z + kSlack)) : 0;
    o.total = off;
    return o;
}

// Variable pass: kernel and grid. A thread sums VPT nodes; VPT is the
// largest of 3, 2, 1 that still gives the grid 4 blocks per SM (wider tiles
// cut per-node overhead; a small batch needs the narrower tiles' blocks).
struct VnLaunch {
    void *func;
    dim3 grid;
};

template <typename M>
void *vn_kernel_for(int vpt, int split) {
    if (split == 1) {
        if (vpt == 3) return (void *)vn_kernel<M, 3, 1>;
        if (vpt == 2) return (void *)vn_kernel<M, 2, 1>;
        return (void *)vn_kernel<M, 1, 1>;
    }
    if (vpt == 3) return (void *)vn_kernel<M, 3, kVnParts>;
    if (vpt == 2) return (void *)vn_kernel<M, 2, kVnParts>;
    return (void *)vn_kernel<M, 1, kVnParts>;
}

int sm_count();

// Variable-pass launch: batches whose heavy nodes fill fewer than
// kVnSplitBlocks 256-node blocks per SM give each part of a node's sum its
// own thread group (same bits, kVnParts times the threads); then the nodes
// per thread (VPT) is the largest of kVnVptMax ... 1 that still leaves four
// blocks per SM.
// vpt_set / split_set (non-zero) override the choice (qcldpc_params
// vn_nodes / vn_split); every shape computes the same bits.
VnLaunch vn_launch(const Table &T, int F, int fmt, int vpt_set = 0, int split_set = 0) {
    const int hc = std::max(T.n_hcols, 1);
    const long long sms = sm_count();
    const long long blocks1 = (long long)F * hc * ((T.Z + kThreads - 1) / kThreads);
    const int split = split_set ? split_set : (kVnParts > 1 && blocks1 < kVnSplitBlocks * sms) ? kVnParts : 1;
    const int G = kThreads / split;
    int vpt = 1;
    for (int v = kVnVptMax; v >= 1; v--) {
        const long long blocks = (long long)F * hc * ((T.Z + G * v - 1) / (G * v));
        if (blocks >= 4 * sms || v == 1) {
            vpt = v;
            break;
        }
    }
    if (vpt_set) vpt = vpt_set;
    VnLaunch l;
    l.grid = dim3((unsigned)((T.Z + G * vpt - 1) / (G * vpt)), (unsigned)hc, (unsigned)F);
    l.func = fmt == 1 ? vn_kernel_for<__half>(vpt, split) : fmt == 2 ? vn_kernel_for<int8_t>(vpt, split)
                                                                    : vn_kernel_for<float>(vpt, split);
    return l;
}

dim3 vn_grid(const Table &T, int F) {
    const int span = kThreads * kVnVpt;
    return dim3((unsigned)((T.Z + span - 1) / span), (unsigned)std::max(T.n_hcols, 1), (unsigned)F);
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// The check-pass kernel for a message format (its translation unit): full
// kThreads-thread blocks, or blocks of any width (nt < kThreads).
void *cn_tma_kernel_for(int maxdeg, int fmt, int nt) {
    if (fmt == 1) return qc::cn_kernel_f16(maxdeg, nt);
    if (fmt == 2) return qc::cn_kernel_i8(maxdeg, nt);
    return qc::cn_kernel_f32(maxdeg, nt);
}

void *lvn_kernel_for(int fmt) {
    if (fmt == 1) return (void *)lvn_kernel<__half>;
    if (fmt == 2) return (void *)lvn_kernel<int8_t>;
    return (void *)lvn_kernel<float>;
}

// Base rows [r0, r1) of row group g when mb rows form G groups: row r is in
// group floor(r * G / mb).
void group_rows(const Table &T, int G, int g, int *r0, int *r1) {
    *r0 = (g * T.mb + G - 1) / G;
    *r1 = ((g + 1) * T.mb + G - 1) / G;
}

// psi(y) = log2 coth(y ln2 / 2) in double (base-2 units; psi(inf) = 0).
float psi_host(float y2) {
    if (!(y2 < INFINITY)) return 0.0f;
    const double t = std::exp2(-(double)y2);
    return (float)std::log2((1.0 + t) / (1.0 - t));
}

// Launch-shape options: 0 (chosen by the library) or a supported value.
bool shape_ok(const qcldpc_params &p) {
    return (p.cn_threads == 0 || (p.cn_threads >= 32 && p.cn_threads <= kCnThreads && p.cn_threads % 32 == 0)) &&
           (p.vn_nodes >= 0 && p.vn_nodes <= kVnVptMax) &&
           (p.vn_split == 0 || p.vn_split == 1 || p.vn_split == kVnParts) &&
           (p.vn_pass == 0 || p.vn_pass == 1);
}

// Fixed-point grid of the posterior accumulators (base-2 units): the
// finest 2^-k, k <= 24, for which the full sum of a heavy column's
// messages fits in int32 when every message has the largest magnitude the
// check pass can store, psi(xmin_h) (the clip folded into the floor), with
// 1% slack for FP32 evaluation and FP16 rounding. 0 when no k >= 8 fits.
float acc_scale_for(const qcldpc_code *code, float clip2, float xmin_h2) {
    int maxcol = 1;
    const std::vector<int32_t> &cp = code->host.col_ptr;
    for (size_t h = 0; h + 1 < cp.size(); h++) maxcol = std::max(maxcol, cp[h + 1] - cp[h]);
    const double t = std::exp2(-(double)xmin_h2);
    const double mmax = std::min((double)clip2, std::log2((1.0 + t) / (1.0 - t))) * 1.01;
    const int k = std::min(24, (int)std::floor(std::log2(2147483647.0 / ((double)maxcol * mmax))));
    return k >= 8 ? std::ldexp(1.0f, k) : 0.0f;
}

// Work fields of the accumulated-posterior flooding pass (vn_pass = 0).
void set_accum(const qcldpc_code *code, const qcldpc_params &p, char *acc_base, Work &w) {
    if (w.layered || p.vn_pass != 0) return;
    if (w.fmt == 2) {
        w.acc_inv = w.qstep;  // the sum counts int8 quanta exactly
    } else {
        w.acc_scale = acc_scale_for(code, w.clip, w.xmin_h);
        if (w.acc_scale == 0.0f) return;  // columns too heavy for the grid: separate pass
        w.acc_inv = 1.0f / w.acc_scale;
    }
    w.acc = reinterpret_cast<int32_t *>(acc_base);
    w.accum = 1;
}

// Floor of a heavy check output's exclusive psi sum (base-2 units). psi is
// decreasing and its own inverse, so clipping the output, min(psi(max(s,
// xmin)), clip), equals psi(max(s, xmin, psi(clip))). With the default clip
// psi(clip) is below xmin and the floor is xmin itself; otherwise it sits a
// hair above psi(clip), so that the FP32 psi of it stays at or below clip.
float heavy_out_floor(float clip2, float xmin2) {
    if (!(clip2 < INFINITY)) return xmin2;
    const double t = std::exp2(-(double)clip2);
    const double psi_clip = std::log2((1.0 + t) / (1.0 - t));
    if (psi_clip * (1.0 + 1e-4) < (double)xmin2) return xmin2;
    return (float)(std::max((double)xmin2, psi_clip) * (1.0 + 1e-4));
}

// Launch of the check-node pass for a code: kernel, grid and dynamic shared
// memory (the staged variant needs the code's widest exact-shape row).
struct CnLaunch {
    void *func;
    dim3 grid;
    dim3 block;
    size_t smem;
};

// Threads per check block: the fewest warps whose tile (threads x kTmaVpt
// checks) still covers a row in as many blocks as kTile-check tiles would.
// A row of Z = 625 gets 160 threads (one 640-check tile, not 61% of a
// 1024-check one), and smaller blocks leave room for more of them per SM.
int cn_threads(int Z) {
    if (!QCLDPC_CN_FIT) return kCnThreads;
    const int nblk = (Z + kTile - 1) / kTile;
    const int per = (Z + nblk - 1) / nblk;
    return std::min(kCnThreads, 32 * ((per + 32 * kTmaVpt - 1) / (32 * kTmaVpt)));
}

// nt_set (non-zero) overrides the block width (qcldpc_params cn_threads);
// a check's arithmetic does not depend on it.
CnLaunch cn_launch(const Table &T, int F, int fmt, int nt_set = 0) {
    CnLaunch c;
    {
        const int nt = nt_set ? nt_set : cn_threads(T.Z), tile = nt * kTmaVpt;
        // the code's widest exact-shape row (its staged rows and word rows)
        const size_t smem = kSmemHeader + (size_t)T.stage_rows_max * (tile + 4) * 4 +
                            (size_t)T.stage_words_max * (tile / 32 + 4) * 4;
        c.func = cn_tma_kernel_for(T.max_row_deg, fmt, nt);
        c.grid = dim3((unsigned)((T.Z + tile - 1) / tile), (unsigned)T.mb, (unsigned)F);
        c.block = dim3((unsigned)nt);
        c.smem = smem;
        // Capacity for the largest staged row set (4 heavy + 1 degree-1).
        static std::once_flag once;
        std::call_once(once, [] {
            const int cap = kSmemHeader + 9 * kStage * 4 + kStageWords * 4;
            qc::cn_smem_cap_f32(cap);
            qc::cn_smem_cap_f16(cap);
            qc::cn_smem_cap_i8(cap);
        });
    }
    return c;
}

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Work key;
    unsigned long long stamp = 0;
};

struct GraphCache {
    GraphEntry e[kGraphCacheSize];
    unsigned long long clock = 0;
};

void free_entry(GraphEntry &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g.exec = nullptr;
    g.graph = nullptr;
}

cudaError_t add_kernel(cudaGraphNode_t *node, cudaGraph_t g, const cudaGraphNode_t *dep,
                       size_t ndep, void *func, dim3 grid, dim3 block, void **args,
                       size_t smem = 0, bool programmatic = false) {
    if (programmatic && QCLDPC_PDL && ndep == 1) {
        // edge that fires when every block of the upstream kernel has
        // triggered (or exited); the kernel waits for its completion itself
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeKernel;
        np.kernel.func = func;
        np.kernel.gridDim = grid;
        np.kernel.blockDim = block;
        np.kernel.sharedMemBytes = (unsigned)smem;
        np.kernel.kernelParams = args;
        np.kernel.extra = nullptr;
        cudaGraphEdgeData ed = {};
        ed.from_port = cudaGraphKernelNodePortProgrammatic;
        ed.type = cudaGraphDependencyTypeProgrammatic;
        return cudaGraphAddNode(node, g, dep, &ed, 1, &np);
    }
    cudaKernelNodeParams kp = {};
    kp.func = func;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    kp.extra = nullptr;
    return cudaGraphAddKernelNode(node, g, dep, ndep, &kp);
}

// Graph node priority of the short per-iteration steps (control, posterior
// or variable pass): the highest the device offers, so that when several
// chains share a graph those steps' blocks are scheduled ahead of the
// pending blocks of another chain's check pass (the graphs are instantiated
// with cudaGraphInstantiateFlagUseNodePriority).
cudaError_t raise_priority(cudaGraphNode_t node) {
    int least = 0, greatest = 0;
    cudaError_t err = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (err != cudaSuccess) return err;
    cudaLaunchAttributeValue v = {};
    v.priority = greatest;
    return cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributePriority, &v);
}

// Loop body of the decode graph. Flooding: check pass -> control ->
// variable pass. Layered: stop-test pass -> control -> for every row group,
// its check pass -> its posterior update. The control steps set the loop
// condition (handle) from the chain's own frames.
cudaError_t add_loop_body(cudaGraph_t body, const Table &T, const qc::ColsInline &CI,
                          const Work &w0, cudaGraphConditionalHandle handle) {
    const int F = w0.n_frames;
    Table tcopy = T;
    Work wcopy = w0;
    qc::ColsInline ccopy = CI;
    void *args[] = {&tcopy, &wcopy};
    void *vn_args[] = {&tcopy, &wcopy, &ccopy};
    const CnLaunch cl = cn_launch(T, F, w0.fmt, w0.cn_nt);
    cudaError_t err;
    if (w0.layered) wcopy.pass = kPassTest;
    void *ctrl_args[] = {&wcopy, &handle};
    const bool pdl = !w0.layered;
    // kLoopUnroll flooding iterations per trip of the WHILE body (each trip
    // costs a body relaunch, ~4 us on GB300): passes of frames that stopped
    // in an earlier iteration of the trip exit at once, and the last control
    // step decides whether another trip runs. A layered iteration is 2 + 2G
    // launches, so its body holds one.
    const int unroll = w0.layered ? 1 : kLoopUnroll;
    cudaGraphNode_t prev = nullptr;
    for (int u = 0; u < unroll; u++) {
        cudaGraphNode_t n_cn, n_ctrl, n_vn;
        if ((err = add_kernel(&n_cn, body, prev ? &prev : nullptr, prev ? 1 : 0, cl.func, cl.grid, cl.block,
                              args, cl.smem, prev != nullptr && QCLDPC_PDL_LOOP)) != cudaSuccess)
            return err;
        if ((err = add_kernel(&n_ctrl, body, &n_cn, 1, (void *)ctrl_kernel<true>, dim3(1),
                              dim3(kCtrlThreads), ctrl_args, 0, pdl)) != cudaSuccess)
            return err;
        if (!w0.layered) {
            if (w0.accum)
                err = add_kernel(&n_vn, body, &n_ctrl, 1, post_func(T), post_grid(T, F), dim3(kThreads),
                                 args, 0, true);
            else {
                const VnLaunch vl = vn_launch(T, F, w0.fmt, w0.vn_vpt, w0.vn_split);
                err = add_kernel(&n_vn, body, &n_ctrl, 1, vl.func, vl.grid, dim3(kThreads), vn_args, 0, true);
            }
            if (err != cudaSuccess || (err = raise_priority(n_ctrl)) != cudaSuccess ||
                (err = raise_priority(n_vn)) != cudaSuccess)
                return err;
            prev = n_vn;
            continue;
        }
        prev = n_ctrl;
        for (int g = 0; g < w0.ngroups; g++) {
            Work wg = w0;
            wg.pass = kPassGroup;
            group_rows(T, w0.ngroups, g, &wg.lrow0, &wg.lrows);
            wg.lrows -= wg.lrow0;
            void *gargs[] = {&tcopy, &wg};
            dim3 grid = cl.grid;
            grid.y = (unsigned)wg.lrows;
            cudaGraphNode_t a, b;
            if ((err = add_kernel(&a, body, &prev, 1, cl.func, grid, cl.block, gargs,
                                  cl.smem)) != cudaSuccess ||
                (err = add_kernel(&b, body, &a, 1, lvn_kernel_for(w0.fmt), vn_grid(T, F),
                                  dim3(kThreads), gargs)) != cudaSuccess)
                return err;
            prev = b;
        }
    }
    return cudaSuccess;
}

// Build and instantiate the decode graph for one argument set.
int build_graph(const qcldpc_code *code, GraphEntry &ge, const Work &w0) {
    const Table &T = code->tab;
    cudaError_t err;
    cudaGraph_t g = nullptr;
    if ((err = cudaGraphCreate(&g, 0)) != cudaSuccess) return qc::cuda_fail(err, "decode: cudaGraphCreate");
    ge.graph = g;
    Table tcopy = T;
    Work wcopy = w0;
    void *args[] = {&tcopy, &wcopy};
    const int blocks = sm_count() * 4;
    cudaGraphNode_t n_init, n_cond, n_final;
    if ((err = add_kernel(&n_init, g, nullptr, 0, (void *)init_kernel, dim3(blocks), dim3(kThreads),
                          args)) != cudaSuccess)
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
    if ((err = add_loop_body(body, T, code->cols_in, w0, handle)) != cudaSuccess)
        return qc::cuda_fail(err, "decode: add loop body");
    if ((err = add_kernel(&n_final, g, &n_cond, 1, (void *)final_kernel, dim3(blocks),
                          dim3(kThreads), args)) != cudaSuccess)
        return qc::cuda_fail(err, "decode: add output kernel");
    cudaGraphExec_t exec = nullptr;
    if ((err = cudaGraphInstantiate(&exec, g, cudaGraphInstantiateFlagUseNodePriority)) != cudaSuccess)
        return qc::cuda_fail(err, "decode: cudaGraphInstantiate");
    ge.exec = exec;
    ge.key = w0;
    return QCLDPC_OK;
}

// launch_mode 1: the same passes as the graph, enqueued one by one.
int stream_decode(qcldpc_code *code, const Work &w, cudaStream_t stream) {
    const Table &T = code->tab;
    const int F = w.n_frames;
    const int blocks = sm_count() * 4;
    init_kernel<<<blocks, kThreads, 0, stream>>>(T, w);
    const CnLaunch cl = cn_launch(T, F, w.fmt, w.cn_nt);
    Table tcopy = T;
    Work wcopy = w;
    if (w.layered) wcopy.pass = kPassTest;
    void *args[] = {&tcopy, &wcopy};
    cudaGraphConditionalHandle none = 0;
    cudaError_t err = cudaGetLastError();
    for (int t = 1; t <= w.max_iter + 1 && err == cudaSuccess; t++) {
        err = cudaLaunchKernel(cl.func, cl.grid, cl.block, args, cl.smem, stream);
        if (err != cudaSuccess) break;
        ctrl_kernel<false><<<1, kCtrlThreads, 0, stream>>>(w, none);
        if (t <= w.max_iter && !w.layered && w.accum) {
            err = cudaLaunchKernel(post_func(T), post_grid(T, F), dim3(kThreads), args, 0, stream);
        } else if (t <= w.max_iter && !w.layered) {
            qc::ColsInline ccopy = code->cols_in;
            void *vn_args[] = {&tcopy, &wcopy, &ccopy};
            const VnLaunch vl = vn_launch(T, F, w.fmt, w.vn_vpt, w.vn_split);
            err = cudaLaunchKernel(vl.func, vl.grid, dim3(kThreads), vn_args, 0, stream);
        }
        for (int g = 0; t <= w.max_iter && w.layered && g < w.ngroups && err == cudaSuccess; g++) {
            Work wg = w;
            wg.pass = kPassGroup;
            group_rows(T, w.ngroups, g, &wg.lrow0, &wg.lrows);
            wg.lrows -= wg.lrow0;
            void *gargs[] = {&tcopy, &wg};
            dim3 grid = cl.grid;
            grid.y = (unsigned)wg.lrows;
            err = cudaLaunchKernel(cl.func, grid, cl.block, gargs, cl.smem, stream);
            if (err == cudaSuccess)
                err = cudaLaunchKernel(lvn_kernel_for(w.fmt), vn_grid(T, F), dim3(kThreads), gargs,
                                       0, stream);
        }
        if (err == cudaSuccess) err = cudaGetLastError();
    }
    if (err == cudaSuccess) {
        final_kernel<<<blocks, kThreads, 0, stream>>>(T, w);
        err = cudaGetLastError();
    }
    if (err != cudaSuccess) return qc::cuda_fail(err, "decode (stream mode): launch");
    qc::clear_error();
    return QCLDPC_OK;
}

// The kernels' argument block for one decode call of `code` on F frames
// whose workspace starts at base with layout lo (options p already checked).
Work make_work(const qcldpc_code *code, const qcldpc_params &p, int F, int max_iter, const float *llr,
               const uint32_t *syn, uint32_t *keys, int32_t *conv, int32_t *iters, float *post,
               char *base, const Layout &lo) {
    const Table &T = code->tab;
    const bool soft = post != nullptr;
    const bool layered = p.schedule == 1;
    Work w;
    std::memset(&w, 0, sizeof(w));  // padding bytes take part in cache keys
    w.llr = llr;
    w.syn = syn;
    w.keys = keys;
    w.conv = conv;
    w.iters = iters;
    w.post = post;
    w.t = reinterpret_cast<int32_t *>(base + lo.t);
    w.active = reinterpret_cast<int32_t *>(base + lo.active);
    w.fail = reinterpret_cast<int32_t *>(base + lo.fail);
    w.err = reinterpret_cast<int32_t *>(base + lo.err);
    w.msg = base + lo.msg;
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
    w.clip = p.clip > 0.0f ? p.clip * kLog2e : INFINITY;  // base-2 units
    w.xmin = p.phi_floor * kLog2e;
    w.xmin_h = heavy_out_floor(w.clip, w.xmin);
    w.phi_lo = psi_host(w.clip);
    w.phi_hi = psi_host(w.xmin);
    w.cn_nt = p.cn_threads;
    w.vn_vpt = p.vn_nodes;
    w.vn_split = p.vn_split;
    w.fmt = p.msg_format;
    if (w.fmt == 2) {
        // int8 quantum: msg_step natural-LLR units, default clip / 127
        const float step = p.msg_step > 0.0f ? p.msg_step : (p.clip > 0.0f ? p.clip : 15.0f) / 127.0f;
        w.qstep = step * kLog2e;
        w.qinv = 1.0f / w.qstep;
    }
    if (layered) {
        w.layered = 1;
        w.ngroups = p.layers > 0 ? p.layers : T.mb;
        w.msg_buf = (int64_t)F * T.n_h * T.Z;
    }
    set_accum(code, p, base + lo.acc, w);
    w.wait_polls = kWaitLimit;
    if (const char *e = std::getenv("QCLDPC_TEST_STALL")) {
        if (e[0] == '1') {  // test switch: every staged wait runs out after a few polls
            w.wait_polls = 64;
            w.stall_extra = 16;
        }
    }
    return w;
}

// Frame groups of a decode (qcldpc_params.frame_groups): graph launches of
// decodes without soft output run groups of consecutive frames as
// side-by-side chains of one graph (as qcldpc_decode_multi does for several
// codes), so that one group's short per-iteration steps (flooding) or small
// per-row-group passes (layered) overlap another group's work; every
// frame's arithmetic is the same in any group. The default is two groups
// for flooding and one chain for layered decoding, whose 2 + 2G launches
// per iteration and chain cost more than the overlap gains (49 row groups,
// 16 frames: 7,176 Mbit/s in one chain, 6,576 in two).
int frame_groups_of(const qcldpc_params &p, int F, bool soft) {
    if (p.launch_mode != 0 || soft || F < 2) return 1;
    const int dflt = p.schedule == 0 ? 2 : 1;
    return std::min(p.frame_groups > 0 ? p.frame_groups : dflt, F);
}
// First frame of group g (the groups differ by at most one frame).
int group_first(int F, int G, int g) { return g * (F / G) + std::min(g, F % G); }
// Workspace of a grouped decode: the groups' own layouts one after the
// other (each 256-byte aligned), and at least one layout of all F frames
// (qcldpc_time_passes replays the passes of the whole batch on it).
size_t groups_workspace(const Table &T, int F, int G, int fmt, bool layered) {
    size_t off = 0;
    for (int g = 0; g < G; g++)
        off = align_up(off, 256) +
              layout_of(T, group_first(F, G, g + 1) - group_first(F, G, g), false, fmt, layered).total;
    return std::max(off, layout_of(T, F, false, fmt, layered).total);
}
int launch_multi(const std::vector<const qcldpc_code *> &used, const std::vector<Work> &works,
                 cudaStream_t stream);

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
    if (!(p.phi_floor > 0.0f) || p.schedule < 0 || p.schedule > 1 || p.msg_format < 0 ||
        p.msg_format > 2 || !(p.msg_step >= 0.0f) || (p.launch_mode != 0 && p.launch_mode != 1) ||
        (p.schedule == 1 && (p.layers < 0 || p.layers > code->tab.mb)) || !shape_ok(p) ||
        p.frame_groups < 0 || p.frame_groups > QCLDPC_MULTI_MAX_CODES)
        return fail(QCLDPC_E_INVAL,
                    "decode: unsupported option (phi_floor > 0, schedule 0..1, layers 0..mb, "
                    "msg_format 0..2, msg_step >= 0, launch shapes, frame_groups 0..16)");
    if (soft && p.soft_output != 1)
        return fail(QCLDPC_E_INVAL, "decode_soft: params->soft_output must be 1");
    if (F == 0) return QCLDPC_OK;
    if (!llr || !syn || !keys || !conv || !iters || !ws)
        return fail(QCLDPC_E_INVAL, "decode: NULL buffer");
    if (!aligned(ws, 256)) return fail(QCLDPC_E_ALIGN, "decode: workspace must be 256-byte aligned");
    if (!aligned(llr, 16) || !aligned(syn, 4) || !aligned(keys, 4) || !aligned(conv, 4) ||
        !aligned(iters, 4) || (post && !aligned(post, 4)))
        return fail(QCLDPC_E_ALIGN, "decode: LLRs must be 16-byte aligned, other buffers 4-byte aligned");
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return cuda_fail(err, "decode: cudaGetDevice");
    if (dev != code->device) return fail(QCLDPC_E_INVAL, "decode: current device differs from the code's device");

    if (int st = upload_tables(code)) return st;
    const Table &T = code->tab;
    const bool layered = p.schedule == 1;
    const Layout lo = layout_of(T, F, soft, p.msg_format, layered);
    const int G = frame_groups_of(p, F, soft);
    if (ws_bytes < (G > 1 ? groups_workspace(T, F, G, p.msg_format, layered) : lo.total))
        return fail(QCLDPC_E_NOMEM, "decode: workspace too small");
    Work w = make_work(code, p, F, max_iter, llr, syn, keys, conv, iters, post, static_cast<char *>(ws), lo);

    std::lock_guard<std::mutex> lock(code->mu);
    code->last_ws = ws;
    code->last_frames = F;
    code->last_soft = soft ? 1 : 0;
    std::memcpy(code->last_work, &w, sizeof(w));
    if (p.launch_mode == 1) return stream_decode(code, w, stream);
    if (G > 1) {
        // group g: frames group_first(g) .. group_first(g + 1) - 1, with
        // its own workspace part (the first layout(F) bytes hold the
        // whole-batch layout of w only for qcldpc_time_passes)
        std::vector<const qcldpc_code *> used((size_t)G, code);
        std::vector<Work> works;
        size_t off = 0;
        for (int g = 0; g < G; g++) {
            const int f0 = group_first(F, G, g), Fg = group_first(F, G, g + 1) - f0;
            const Layout lg = layout_of(T, Fg, false, p.msg_format, layered);
            off = align_up(off, 256);
            works.push_back(make_work(code, p, Fg, max_iter, llr + (size_t)f0 * w.n, syn + (size_t)f0 * w.words_m,
                                      keys + (size_t)f0 * w.words_k, conv + f0, iters + f0, nullptr,
                                      static_cast<char *>(ws) + off, lg));
            off += lg.total;
        }
        return launch_multi(used, works, stream);
    }

    GraphCache *gc = static_cast<GraphCache *>(code->graph_cache);
    if (!gc) {
        gc = new (std::nothrow) GraphCache();
        if (!gc) return fail(QCLDPC_E_NOMEM, "decode: out of host memory");
        code->graph_cache = gc;
    }
    GraphEntry *hit = nullptr, *victim = &gc->e[0];
    for (auto &e : gc->e) {
        if (e.exec && std::memcmp(&e.key, &w, sizeof(w)) == 0) hit = &e;
        if (!e.exec || (victim->exec && e.stamp < victim->stamp)) victim = &e;
    }
    if (!hit) {
        free_entry(*victim);
        int st = build_graph(code, *victim, w);
        if (st != QCLDPC_OK) {
            free_entry(*victim);
            return st;
        }
        hit = victim;
    }
    hit->stamp = ++gc->clock;
    if ((err = cudaGraphLaunch(hit->exec, stream)) != cudaSuccess)
        return cuda_fail(err, "decode: cudaGraphLaunch");
    clear_error();
    return QCLDPC_OK;
}

}  // namespace

namespace qc {
void destroy_graph_cache(qcldpc_code *code) {
    GraphCache *gc = static_cast<GraphCache *>(code->graph_cache);
    if (!gc) return;
    for (auto &e : gc->e) free_entry(e);
    delete gc;
    code->graph_cache = nullptr;
}
}  // namespace qc

extern "C" size_t qcldpc_decode_workspace(const qcldpc_code *code, int n_frames,
                                          const qcldpc_params *p) {
    if (!code || n_frames < 0 || n_frames > 65535) return 0;
    const bool soft = p && p->soft_output == 1;
    const int fmt = p ? p->msg_format : 0;
    if (fmt < 0 || fmt > 2) return 0;
    qcldpc_params d;
    qcldpc_params_init(&d);
    if (p && (p->frame_groups < 0 || p->frame_groups > QCLDPC_MULTI_MAX_CODES)) return 0;
    const int G = frame_groups_of(p ? *p : d, n_frames, soft);
    if (G > 1) return groups_workspace(code->tab, n_frames, G, fmt, p && p->schedule == 1);
    return layout_of(code->tab, n_frames, soft, fmt, p && p->schedule == 1).total;
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

// ---------------------------------------------------------------------------
// Batched decoding: the frames of several codes in one graph launch.
//
// The graph holds, for every code (or every frame group of one code), the
// chain a one-code decode runs: initialisation, a device-side loop (a
// conditional WHILE node) over the flooding passes (check pass, control
// step, posterior pass, kLoopUnroll times per trip) whose control steps end
// it once the chain's own frames have stopped, and the output step. The
// chains are independent branches, so the small grids of short codes fill
// the GPU together and one chain's short steps run inside another's check
// pass. Each frame keeps its own iteration counter and stop test, so its
// result is the one a one-code decode of the same frames gives.
namespace {

constexpr int kMultiMaxCodes = QCLDPC_MULTI_MAX_CODES;

struct MultiDecodeGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const qcldpc_code *> codes;
    std::vector<Work> works;
    unsigned long long stamp = 0;
};
// Batched decode graphs kept instantiated (least recently used replaced):
// qcldpc_decode_multi's and the grouped single-code decodes' argument sets.
constexpr int kMultiDecodeGraphs = 32;
std::mutex g_mdec_mu;
MultiDecodeGraph g_mdec[kMultiDecodeGraphs];
unsigned long long g_mdec_clock = 0;

void free_multi(MultiDecodeGraph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g.exec = nullptr;
    g.graph = nullptr;
    g.codes.clear();
    g.works.clear();
}

// One graph for several chains of frames (codes of a batched decode, or
// the frame groups of one code): chain c is init -> its own conditional
// WHILE loop (whose control steps set its condition from its frames) ->
// final, and the chains are independent branches. Each chain stops when
// its own frames have stopped, and the chains never wait for each other
// inside the loop, so their passes stay interleaved.
int build_multi_graph(MultiDecodeGraph &ge, const std::vector<const qcldpc_code *> &codes,
                      const std::vector<Work> &works) {
    cudaError_t err;
    cudaGraph_t g = nullptr;
    if ((err = cudaGraphCreate(&g, 0)) != cudaSuccess) return qc::cuda_fail(err, "decode_multi: cudaGraphCreate");
    ge.graph = g;
    const int blocks = sm_count() * 4;
    for (size_t c = 0; c < codes.size(); c++) {
        Table tcopy = codes[c]->tab;
        Work wcopy = works[c];
        void *args[] = {&tcopy, &wcopy};
        cudaGraphNode_t n_init, n_cond, n_final;
        if ((err = add_kernel(&n_init, g, nullptr, 0, (void *)init_kernel, dim3(blocks), dim3(kThreads),
                              args)) != cudaSuccess)
            return qc::cuda_fail(err, "decode_multi: add init node");
        cudaGraphConditionalHandle handle;
        if ((err = cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
            return qc::cuda_fail(err, "decode_multi: cudaGraphConditionalHandleCreate");
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if ((err = cudaGraphAddNode(&n_cond, g, &n_init, nullptr, 1, &cp)) != cudaSuccess)
            return qc::cuda_fail(err, "decode_multi: add conditional node");
        if ((err = add_loop_body(cp.conditional.phGraph_out[0], codes[c]->tab, codes[c]->cols_in, works[c],
                                 handle)) != cudaSuccess)
            return qc::cuda_fail(err, "decode_multi: add loop body");
        if ((err = add_kernel(&n_final, g, &n_cond, 1, (void *)final_kernel, dim3(blocks), dim3(kThreads),
                              args)) != cudaSuccess)
            return qc::cuda_fail(err, "decode_multi: add output kernel");
    }
    cudaGraphExec_t exec = nullptr;
    if ((err = cudaGraphInstantiate(&exec, g, cudaGraphInstantiateFlagUseNodePriority)) != cudaSuccess)
        return qc::cuda_fail(err, "decode_multi: cudaGraphInstantiate");
    ge.exec = exec;
    ge.codes = codes;
    ge.works = works;
    return QCLDPC_OK;
}

// Launch the batched decode graph of (codes, works), from the cache of
// recent argument sets or built and instantiated now.
int launch_multi(const std::vector<const qcldpc_code *> &used, const std::vector<Work> &works,
                 cudaStream_t stream) {
    using namespace qc;
    std::lock_guard<std::mutex> lock(g_mdec_mu);
    MultiDecodeGraph *hit = nullptr, *victim = &g_mdec[0];
    for (auto &g : g_mdec) {
        if (g.exec && g.codes == used && g.works.size() == works.size() &&
            std::memcmp(g.works.data(), works.data(), sizeof(Work) * works.size()) == 0)
            hit = &g;
        if (!g.exec || (victim->exec && g.stamp < victim->stamp)) victim = &g;
    }
    if (!hit) {
        free_multi(*victim);
        if (int st = build_multi_graph(*victim, used, works)) {
            free_multi(*victim);
            return st;
        }
        hit = victim;
    }
    hit->stamp = ++g_mdec_clock;
    cudaError_t err = cudaGraphLaunch(hit->exec, stream);
    if (err != cudaSuccess) return cuda_fail(err, "decode_multi: cudaGraphLaunch");
    clear_error();
    return QCLDPC_OK;
}

bool multi_params_ok(const qcldpc_params &p) {
    return p.phi_floor > 0.0f && p.schedule == 0 && p.soft_output == 0 && p.msg_format >= 0 &&
           p.msg_format <= 2 && p.msg_step >= 0.0f && shape_ok(p);
}

}  // namespace

namespace qc {
void purge_multi_graphs(const qcldpc_code *code) {
    std::lock_guard<std::mutex> lock(g_mdec_mu);
    for (auto &g : g_mdec)
        if (g.exec && std::find(g.codes.begin(), g.codes.end(), code) != g.codes.end()) free_multi(g);
}
}  // namespace qc

extern "C" size_t qcldpc_decode_multi_workspace(int n_codes, const qcldpc_code *const *codes,
                                                const int *n_frames, const qcldpc_params *p) {
    if (n_codes < 1 || n_codes > kMultiMaxCodes || !codes || !n_frames) return 0;
    const int fmt = p ? p->msg_format : 0;
    if (fmt < 0 || fmt > 2) return 0;
    size_t total = 0;
    for (int c = 0; c < n_codes; c++) {
        if (!codes[c] || n_frames[c] < 0 || n_frames[c] > 65535) return 0;
        total = align_up(total, 256) + layout_of(codes[c]->tab, n_frames[c], false, fmt).total;
    }
    return total;
}

extern "C" int qcldpc_decode_multi(int n_codes, const qcldpc_code *const *codes, const float *const *llr_dev,
                                   const uint32_t *const *syn_dev, const int *n_frames, int max_iter,
                                   const qcldpc_params *p_in, uint32_t *const *key_bits_dev,
                                   int32_t *const *converged_dev, int32_t *const *iters_dev,
                                   void *workspace_dev, size_t workspace_bytes, qcldpc_stream_t stream) {
    using namespace qc;
    if (n_codes < 1 || n_codes > kMultiMaxCodes)
        return fail(QCLDPC_E_INVAL, "decode_multi: n_codes must be in [1, QCLDPC_MULTI_MAX_CODES]");
    if (!codes || !llr_dev || !syn_dev || !n_frames || !key_bits_dev || !converged_dev || !iters_dev ||
        !workspace_dev)
        return fail(QCLDPC_E_INVAL, "decode_multi: NULL array");
    if (max_iter < 0) return fail(QCLDPC_E_INVAL, "decode_multi: max_iter must be >= 0");
    qcldpc_params p;
    if (p_in) p = *p_in;
    else qcldpc_params_init(&p);
    if (!multi_params_ok(p))
        return fail(QCLDPC_E_INVAL,
                    "decode_multi: unsupported option (flooding only, no soft output, msg_format 0..2)");
    if (!aligned(workspace_dev, 256)) return fail(QCLDPC_E_ALIGN, "decode_multi: workspace must be 256-byte aligned");
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return cuda_fail(err, "decode_multi: cudaGetDevice");
    std::vector<const qcldpc_code *> used;
    std::vector<Work> works;
    size_t off = 0;
    for (int c = 0; c < n_codes; c++) {
        qcldpc_code *code = const_cast<qcldpc_code *>(codes[c]);
        const int F = n_frames[c];
        if (!code) return fail(QCLDPC_E_INVAL, "decode_multi: NULL code");
        if (F < 0 || F > 65535) return fail(QCLDPC_E_INVAL, "decode_multi: n_frames must be in [0, 65535]");
        if (dev != code->device) return fail(QCLDPC_E_INVAL, "decode_multi: a code belongs to another device");
        if (int st = upload_tables(code)) return st;
        const Layout lo = layout_of(code->tab, F, false, p.msg_format);
        off = align_up(off, 256);
        char *base = static_cast<char *>(workspace_dev) + off;
        off += lo.total;
        if (F == 0) continue;
        if (!llr_dev[c] || !syn_dev[c] || !key_bits_dev[c] || !converged_dev[c] || !iters_dev[c])
            return fail(QCLDPC_E_INVAL, "decode_multi: NULL buffer");
        if (!aligned(llr_dev[c], 16) || !aligned(syn_dev[c], 4) || !aligned(key_bits_dev[c], 4) ||
            !aligned(converged_dev[c], 4) || !aligned(iters_dev[c], 4))
            return fail(QCLDPC_E_ALIGN, "decode_multi: LLRs must be 16-byte aligned, other buffers 4-byte aligned");
        used.push_back(code);
        works.push_back(make_work(code, p, F, max_iter, llr_dev[c], syn_dev[c], key_bits_dev[c], converged_dev[c],
                                  iters_dev[c], nullptr, base, lo));
    }
    if (workspace_bytes < off) return fail(QCLDPC_E_NOMEM, "decode_multi: workspace too small");
    if (used.empty()) return QCLDPC_OK;
    return launch_multi(used, works, (cudaStream_t)stream);
}

extern "C" int qcldpc_autotune(const qcldpc_code *code, const float *llr_dev,
                               const uint32_t *syn_dev, int n_frames, int max_iter,
                               const qcldpc_params *p_in, uint32_t *key_bits_dev,
                               int32_t *converged_dev, int32_t *iters_dev, void *workspace_dev,
                               size_t workspace_bytes, int reps, qcldpc_params *best,
                               float *times_ms, qcldpc_stream_t stream_) {
    using namespace qc;
    if (!code || !best || reps < 1 || n_frames < 1)
        return fail(QCLDPC_E_INVAL, "autotune: bad argument");
    cudaStream_t stream = (cudaStream_t)stream_;
    qcldpc_params base;
    if (p_in) base = *p_in;
    else qcldpc_params_init(&base);
    const int mb = code->tab.mb;
    // 0: flooding, else layered with that many row groups (at most 64: a
    // group costs two launches per iteration)
    const int want[4] = {0, 2, 7, std::min(mb, 64)};
    if (times_ms)
        for (int i = 0; i < 4; i++) times_ms[i] = NAN;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err;
    if ((err = cudaEventCreate(&e0)) != cudaSuccess || (err = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(err, "autotune: cudaEventCreate");
    }
    int best_i = -1;
    float best_ms = INFINITY;
    int st = QCLDPC_OK;
    for (int i = 0; i < 4 && st == QCLDPC_OK; i++) {
        if (i > 0 && (want[i] > mb || (i == 3 && (want[3] == 2 || want[3] == 7)))) continue;
        qcldpc_params p = base;
        p.schedule = want[i] ? 1 : 0;
        p.layers = want[i];
        auto run = [&]() {
            return decode_impl(code, llr_dev, syn_dev, n_frames, max_iter, &p, key_bits_dev,
                               converged_dev, iters_dev, nullptr, workspace_dev, workspace_bytes,
                               stream);
        };
        if ((st = run()) != QCLDPC_OK) break;  // untimed: graph instantiation
        cudaEventRecord(e0, stream);
        for (int r = 0; r < reps && st == QCLDPC_OK; r++) st = run();
        cudaEventRecord(e1, stream);
        if (st != QCLDPC_OK) break;
        float ms = 0.0f;
        if ((err = cudaEventSynchronize(e1)) != cudaSuccess ||
            (err = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
            st = cuda_fail(err, "autotune: timing");
            break;
        }
        ms /= (float)reps;
        if (times_ms) times_ms[i] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best_i = i;
            *best = p;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != QCLDPC_OK) return st;
    if (best_i < 0) return fail(QCLDPC_E_INVAL, "autotune: no candidate ran");
    clear_error();
    return QCLDPC_OK;
}

// Launch-shape candidates of qcldpc_autotune_shapes, in the order of its
// timing arrays: check blocks of 32, 64, ..., 256 threads; variable pass
// (nodes per thread, part groups) = (1,1), (2,1), (3,1), (1,P), (2,P), (3,P).
extern "C" int qcldpc_autotune_shapes(const qcldpc_code *code_c, int n_frames, void *workspace_dev,
                                      size_t workspace_bytes, int reps, const qcldpc_params *p,
                                      qcldpc_params *best, float *cn_ms, float *vn_ms,
                                      qcldpc_stream_t stream_) {
    using namespace qc;
    qcldpc_code *code = const_cast<qcldpc_code *>(code_c);
    if (!code || !workspace_dev || !best || reps < 1 || n_frames < 1 || n_frames > 65535)
        return fail(QCLDPC_E_INVAL, "autotune_shapes: bad argument");
    cudaStream_t stream = (cudaStream_t)stream_;
    qcldpc_params base;
    if (p) base = *p;
    else qcldpc_params_init(&base);
    std::lock_guard<std::mutex> lock(code->mu);
    if (code->last_ws != workspace_dev || code->last_frames != n_frames)
        return fail(QCLDPC_E_INVAL, "autotune_shapes: no decode ran on this workspace with this frame count");
    Work w;
    std::memcpy(&w, code->last_work, sizeof(w));
    if (w.layered) return fail(QCLDPC_E_INVAL, "autotune_shapes: the last decode was layered (flooding only)");
    const Layout lo = layout_of(code->tab, n_frames, code->last_soft != 0, w.fmt);
    if (workspace_bytes < lo.total) return fail(QCLDPC_E_NOMEM, "autotune_shapes: workspace too small");
    if (w.max_iter < 2) w.max_iter = 2;  // replays run as iteration 2: a full update
    const Table &T = code->tab;
    Table tcopy = T;
    qc::ColsInline ccopy = code->cols_in;
    void *args[] = {&tcopy, &w};
    void *vn_args[] = {&tcopy, &w, &ccopy};
    cudaEvent_t e0, e1;
    cudaError_t err = cudaEventCreate(&e0);
    if (err != cudaSuccess) return cuda_fail(err, "autotune_shapes: cudaEventCreate");
    if ((err = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(err, "autotune_shapes: cudaEventCreate");
    }
    replay_prep_kernel<<<1, 256, 0, stream>>>(w);
    // mean time of `reps` launches after one warm-up launch
    auto time = [&](const void *func, dim3 grid, dim3 block, void **a, size_t smem) {
        float t = 0.f;
        if (err == cudaSuccess) err = cudaLaunchKernel(func, grid, block, a, smem, stream);
        if (err == cudaSuccess) err = cudaEventRecord(e0, stream);
        for (int r = 0; r < reps && err == cudaSuccess; r++) err = cudaLaunchKernel(func, grid, block, a, smem, stream);
        if (err == cudaSuccess) err = cudaEventRecord(e1, stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
        return t / reps;
    };
    constexpr int kNc = kCnThreads / 32, kNv = 6;
    float tc[kNc], tv[kNv];
    int bc = 0, bv = 0;
    for (int i = 0; i < kNc; i++) {
        const CnLaunch cl = cn_launch(T, n_frames, w.fmt, 32 * (i + 1));
        tc[i] = time(cl.func, cl.grid, cl.block, args, cl.smem);
        if (tc[i] < tc[bc]) bc = i;
    }
    for (int i = 0; i < kNv; i++) {
        const VnLaunch vl = vn_launch(T, n_frames, w.fmt, i % 3 + 1, i < 3 ? 1 : kVnParts);
        tv[i] = time(vl.func, vl.grid, dim3(kThreads), vn_args, 0);
        if (tv[i] < tv[bv]) bv = i;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "autotune_shapes");
    for (int i = 0; i < kNc; i++)
        if (cn_ms) cn_ms[i] = tc[i];
    for (int i = 0; i < kNv; i++)
        if (vn_ms) vn_ms[i] = tv[i];
    *best = base;
    best->cn_threads = 32 * (bc + 1);
    best->vn_nodes = bv % 3 + 1;
    best->vn_split = bv < 3 ? 1 : kVnParts;
    clear_error();
    return QCLDPC_OK;
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
    std::lock_guard<std::mutex> lock(code->mu);
    if (code->last_ws != workspace_dev || code->last_frames != n_frames)
        return fail(QCLDPC_E_INVAL, "time_passes: no decode ran on this workspace with this frame count");
    Work w;
    std::memcpy(&w, code->last_work, sizeof(w));
    if (w.layered) return fail(QCLDPC_E_INVAL, "time_passes: the last decode was layered (flooding only)");
    const Layout lo = layout_of(code->tab, n_frames, code->last_soft != 0, w.fmt);
    if (workspace_bytes < lo.total) return fail(QCLDPC_E_NOMEM, "time_passes: workspace too small");
    if (w.max_iter < 2) w.max_iter = 2;  // replays run as iteration 2: a full update
    cudaEvent_t ev[3];
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < 3; i++)
        if ((err = cudaEventCreate(&ev[i])) != cudaSuccess) return cuda_fail(err, "time_passes: cudaEventCreate");
    const Table &T = code->tab;
    replay_prep_kernel<<<1, 256, 0, stream>>>(w);
    const CnLaunch cl = cn_launch(T, n_frames, w.fmt, w.cn_nt);
    Table tcopy = T;
    void *args[] = {&tcopy, &w};
    cudaEventRecord(ev[0], stream);
    for (int r = 0; r < reps && err == cudaSuccess; r++)
        err = cudaLaunchKernel(cl.func, cl.grid, cl.block, args, cl.smem, stream);
    cudaEventRecord(ev[1], stream);
    qc::ColsInline ccopy = code->cols_in;
    void *vn_args[] = {&tcopy, &w, &ccopy};
    const VnLaunch vl = vn_launch(T, n_frames, w.fmt, w.vn_vpt, w.vn_split);
    for (int r = 0; r < reps && err == cudaSuccess; r++) {
        if (w.accum)
            err = cudaLaunchKernel(post_func(T), post_grid(T, n_frames), dim3(kThreads), args, 0, stream);
        else
            err = cudaLaunchKernel(vl.func, vl.grid, dim3(kThreads), vn_args, 0, stream);
    }
    cudaEventRecord(ev[2], stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(ev[2]);
    float a = 0.f, b = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&a, ev[0], ev[1]);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&b, ev[1], ev[2]);
    for (int i = 0; i < 3; i++) cudaEventDestroy(ev[i]);
    if (err != cudaSuccess) return cuda_fail(err, "time_passes");
    *cn_ms = a / reps;
    *vn_ms = b / reps;
    clear_error();
    return QCLDPC_OK;
}

// ---------------------------------------------------------------------------
// Pools: continuous batching of frames of one code.
//
// A pool is a fixed set of frame slots of one code, with the decoder state of
// every slot in one caller-owned workspace. Frames are loaded into free slots
// at any time, every step runs a given number of iteration passes over all
// running slots (each frame at its own iteration), and frames that stopped are
// collected, which frees their slots. Because every slot keeps its own
// counter, stop test and outputs, a frame decodes exactly as it would alone,
// whatever else shares the passes.
namespace {

__global__ void __launch_bounds__(kThreads) pool_reset_kernel(const __grid_constant__ Work W) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t f = tid; f < W.n_frames; f += (int64_t)gridDim.x * blockDim.x) {
        W.state[f] = 0;
        W.active[f] = 0;
        W.fail[f] = 0;
        W.t[f] = 0;
        W.conv[f] = 0;
        W.iters[f] = 0;
    }
    if (tid == 0) *W.err = 0;
}

// Copy n frames (channel LLRs, syndromes) into the listed slots and set up
// their decoder state as init_kernel does for a whole batch.
__global__ void __launch_bounds__(kThreads) pool_load_kernel(const __grid_constant__ Table T,
                                                             const __grid_constant__ Work W,
                                                             const int32_t *__restrict__ slots, int n,
                                                             const float *__restrict__ llr_src,
                                                             const uint32_t *__restrict__ syn_src) {
    const int Z = T.Z;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t N = W.n;
    for (int64_t e = tid; e < (int64_t)n * N; e += nthreads) {
        const int64_t q = e / N, v = e - q * N;
        const_cast<float *>(W.llr)[(int64_t)slots[q] * N + v] = llr_src[e];
    }
    for (int64_t e = tid; e < (int64_t)n * W.words_m; e += nthreads) {
        const int64_t q = e / W.words_m, w = e - q * W.words_m;
        const_cast<uint32_t *>(W.syn)[(int64_t)slots[q] * W.words_m + w] = syn_src[e];
    }
    const int64_t nL = (int64_t)n * T.n_hcols * Z;
    for (int64_t e = tid; e < nL; e += nthreads) {
        const int64_t q = e / ((int64_t)T.n_hcols * Z);
        const int64_t rem = e - q * T.n_hcols * Z;
        const int hc = (int)(rem / Z), j = (int)(rem - (int64_t)hc * Z);
        const int64_t f = slots[q];
        const float qv = llr_src[q * N + (int64_t)T.hcol_base[hc] * Z + j] * kLog2e + 0.0f;
        float *row = W.L + ((size_t)f * T.n_hcols + hc) * 2 * Z;
        row[j] = qv;
        row[j + Z] = qv;
        if (W.accum) {
            int32_t *a = W.acc + ((size_t)f * T.n_hcols + hc) * 2 * Z;
            a[j] = 0;
            a[j + Z] = 0;
        }
    }
    const int lane = threadIdx.x & 31;
    const int64_t warp = tid >> 5, nwarps = nthreads >> 5;
    const int64_t nwords = (int64_t)n * T.n_d1 * W.ZW;
    for (int64_t qw = warp; qw < nwords; qw += nwarps) {
        const int64_t q = qw / ((int64_t)T.n_d1 * W.ZW);
        const int64_t rem = qw - q * T.n_d1 * W.ZW;
        const int k = (int)(rem / W.ZW), wd = (int)(rem - (int64_t)k * W.ZW);
        const int64_t f = slots[q];
        const int i = wd * 32 + lane;
        bool neg = false;
        if (i < Z) {
            int vo = i + T.d1_shift[k];
            if (vo >= Z) vo -= Z;
            const float qv = llr_src[q * N + (int64_t)T.d1_col[k] * Z + vo];
            const float a = fmaxf(fminf(fabsf(qv) * kLog2e, W.clip), W.xmin);
            const float p = psi_f(a);
            W.phiq[((size_t)f * T.n_d1 + k) * Z + i] = qv < 0.0f ? -p : p;
            neg = qv < 0.0f;
        }
        const uint32_t word = __ballot_sync(0xffffffffu, neg);
        if (lane == 0) {
            // decisions of iteration 0 go to the buffer of parity 0
            W.bits[((size_t)f * T.n_d1 + k) * W.ZW + wd] = word;
        }
    }
    for (int64_t q = tid; q < n; q += nthreads) {
        const int32_t f = slots[q];
        W.t[f] = 1;
        W.fail[f] = 0;
        W.conv[f] = 0;
        W.iters[f] = 0;
        W.active[f] = 1;
        W.state[f] = 1;
    }
}

// Outputs of the listed (stopped) slots, then free them.
__global__ void __launch_bounds__(kThreads) pool_collect_kernel(
    const __grid_constant__ Table T, const __grid_constant__ Work W, const int32_t *__restrict__ slots,
    int n, uint32_t *__restrict__ keys, int32_t *__restrict__ conv, int32_t *__restrict__ iters) {
    const int Z = T.Z;
    const int lane = threadIdx.x & 31;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t warp = tid >> 5, nwarps = nthreads >> 5;
    for (int64_t qw = warp; qw < (int64_t)n * W.words_k; qw += nwarps) {
        const int64_t q = qw / W.words_k, wd = qw - q * W.words_k;
        const int64_t f = slots[q];
        const int64_t v = wd * 32 + lane;
        bool dec = false;
        if (v < T.k) {
            const int c = (int)(v / Z), j = (int)(v - (int64_t)c * Z);
            const int kind = T.col_kind[c];
            if (kind >= 0) {
                dec = W.L[((size_t)f * T.n_hcols + kind) * 2 * Z + j] < 0.0f;
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
        if (lane == 0) keys[q * W.words_k + wd] = word;
    }
    for (int64_t q = tid; q < n; q += nthreads) {
        const int32_t f = slots[q];
        conv[q] = W.conv[f];
        iters[q] = W.iters[f];
    }
}

__global__ void pool_free_kernel(const __grid_constant__ Work W, const int32_t *__restrict__ slots,
                                 int n) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t q = tid; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        W.state[slots[q]] = 0;
        W.active[slots[q]] = 0;
    }
}

struct Layout2 {
    Layout base;
    size_t llr, syn, conv, iters, state, total;
};

Layout2 pool_layout(const qcldpc_code *code, int S, int fmt, bool layered = false) {
    Layout2 o;
    o.base = layout_of(code->tab, S, false, fmt, layered);
    size_t off = o.base.total;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    const size_t words_m = (size_t)((code->m + 31) / 32);
    o.llr = take(sizeof(float) * (size_t)S * (size_t)code->n);
    o.syn = take(sizeof(uint32_t) * (size_t)S * words_m);
    o.conv = take(sizeof(int32_t) * S);
    o.iters = take(sizeof(int32_t) * S);
    o.state = take(sizeof(int32_t) * S);
    o.total = off;
    return o;
}

constexpr int kPoolGraphs = 4;

}  // namespace

struct qcldpc_pool {
    qcldpc_code *code;
    Work w;
    int n_slots;
    struct StepGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        int passes = 0;
    } graphs[kPoolGraphs];
    int next_graph = 0;
};

namespace {

// Append n_passes iteration passes of one pool to graph g after node `dep`
// (nullptr: a root chain). Returns the last node.
cudaError_t add_pool_passes(cudaGraph_t g, const qcldpc_pool *pool, int n_passes,
                            cudaGraphNode_t *last) {
    const Table &T = pool->code->tab;
    const int F = pool->n_slots;
    Table tcopy = T;
    Work wcopy = pool->w;
    qc::ColsInline ccopy = pool->code->cols_in;
    void *args[] = {&tcopy, &wcopy};
    void *vn_args[] = {&tcopy, &wcopy, &ccopy};
    cudaGraphConditionalHandle none = 0;
    void *ctrl_args[] = {&wcopy, &none};
    const CnLaunch cl = cn_launch(T, F, pool->w.fmt, pool->w.cn_nt);
    const VnLaunch vl = vn_launch(T, F, pool->w.fmt, pool->w.vn_vpt, pool->w.vn_split);
    const bool layered = pool->w.layered != 0;
    if (layered) wcopy.pass = kPassTest;
    // layered: one Work per row group (kPassGroup, its base rows)
    std::vector<Work> wg(layered ? pool->w.ngroups : 0, pool->w);
    for (int k = 0; k < (int)wg.size(); k++) {
        wg[k].pass = kPassGroup;
        group_rows(T, pool->w.ngroups, k, &wg[k].lrow0, &wg[k].lrows);
        wg[k].lrows -= wg[k].lrow0;
    }
    cudaGraphNode_t prev = nullptr;
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < n_passes && err == cudaSuccess; i++) {
        // an iteration: check pass (flooding: the update and the stop test
        // of the previous iteration; layered: the test alone), control step,
        // then the variable pass or, per row group, its check pass and
        // posterior update
        cudaGraphNode_t a, b, c;
        err = add_kernel(&a, g, prev ? &prev : nullptr, prev ? 1 : 0, cl.func, cl.grid, cl.block,
                         args, cl.smem);
        if (err == cudaSuccess)
            err = add_kernel(&b, g, &a, 1, (void *)ctrl_kernel<false>, dim3(1), dim3(kCtrlThreads),
                             ctrl_args);
        if (!layered) {
            if (err == cudaSuccess) {
                if (pool->w.accum)
                    err = add_kernel(&c, g, &b, 1, post_func(T), post_grid(T, F), dim3(kThreads), args);
                else
                    err = add_kernel(&c, g, &b, 1, vl.func, vl.grid, dim3(kThreads), vn_args);
            }
            // the short steps ahead of other pools' pending check blocks
            if (err == cudaSuccess) err = raise_priority(b);
            if (err == cudaSuccess) err = raise_priority(c);
            prev = c;
            continue;
        }
        prev = b;
        for (int k = 0; k < (int)wg.size() && err == cudaSuccess; k++) {
            void *gargs[] = {&tcopy, &wg[k]};
            dim3 grid = cl.grid;
            grid.y = (unsigned)wg[k].lrows;
            cudaGraphNode_t x, y;
            err = add_kernel(&x, g, &prev, 1, cl.func, grid, cl.block, gargs, cl.smem);
            if (err == cudaSuccess)
                err = add_kernel(&y, g, &x, 1, lvn_kernel_for(pool->w.fmt), vn_grid(T, F), dim3(kThreads),
                                 gargs);
            prev = y;
        }
    }
    *last = prev;
    return err;
}

// Graphs stepping several pools at once, cached by (pools, passes) with
// least-recently-used eviction (a server steps changing subsets of its pools).
struct MultiGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<qcldpc_pool *> pools;
    int passes = 0;
    unsigned long long stamp = 0;
};
constexpr int kMultiGraphs = 32;
std::mutex g_multi_mu;
MultiGraph g_multi[kMultiGraphs];
unsigned long long g_multi_clock = 0;

}  // namespace

extern "C" size_t qcldpc_pool_workspace(const qcldpc_code *code, int n_slots,
                                        const qcldpc_params *p) {
    if (!code || n_slots < 1 || n_slots > 65535) return 0;
    const int fmt = p ? p->msg_format : 0;
    if (fmt < 0 || fmt > 2) return 0;
    return pool_layout(code, n_slots, fmt, p && p->schedule == 1).total;
}

extern "C" int qcldpc_pool_create(const qcldpc_code *code_c, int n_slots, int max_iter,
                                  const qcldpc_params *p_in, void *workspace_dev,
                                  size_t workspace_bytes, qcldpc_stream_t stream,
                                  qcldpc_pool **out) {
    using namespace qc;
    if (!out) return fail(QCLDPC_E_INVAL, "pool_create: out is NULL");
    *out = nullptr;
    qcldpc_code *code = const_cast<qcldpc_code *>(code_c);
    if (!code || !workspace_dev || n_slots < 1 || n_slots > 65535 || max_iter < 0)
        return fail(QCLDPC_E_INVAL, "pool_create: bad argument");
    qcldpc_params p;
    if (p_in) p = *p_in;
    else qcldpc_params_init(&p);
    if (!(p.phi_floor > 0.0f) || p.schedule < 0 || p.schedule > 1 || p.msg_format < 0 ||
        p.msg_format > 2 || !(p.msg_step >= 0.0f) || p.soft_output || !shape_ok(p) ||
        (p.schedule == 1 && (p.layers < 0 || p.layers > code->tab.mb)))
        return fail(QCLDPC_E_INVAL, "pool_create: unsupported option");
    if (!aligned(workspace_dev, 256)) return fail(QCLDPC_E_ALIGN, "pool_create: workspace must be 256-byte aligned");
    if (int st = upload_tables(code)) return st;
    const bool layered = p.schedule == 1;
    const Layout2 lo = pool_layout(code, n_slots, p.msg_format, layered);
    if (workspace_bytes < lo.total) return fail(QCLDPC_E_NOMEM, "pool_create: workspace too small");
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return cuda_fail(err, "pool_create: cudaGetDevice");
    if (dev != code->device) return fail(QCLDPC_E_INVAL, "pool_create: current device differs from the code's device");
    qcldpc_pool *pool = new (std::nothrow) qcldpc_pool();
    if (!pool) return fail(QCLDPC_E_NOMEM, "pool_create: out of host memory");
    char *base = static_cast<char *>(workspace_dev);
    Work &w = pool->w;
    std::memset(&w, 0, sizeof(w));
    w.llr = reinterpret_cast<float *>(base + lo.llr);
    w.syn = reinterpret_cast<uint32_t *>(base + lo.syn);
    w.conv = reinterpret_cast<int32_t *>(base + lo.conv);
    w.iters = reinterpret_cast<int32_t *>(base + lo.iters);
    w.state = reinterpret_cast<int32_t *>(base + lo.state);
    w.t = reinterpret_cast<int32_t *>(base + lo.base.t);
    w.err = reinterpret_cast<int32_t *>(base + lo.base.err);
    w.active = reinterpret_cast<int32_t *>(base + lo.base.active);
    w.fail = reinterpret_cast<int32_t *>(base + lo.base.fail);
    w.msg = base + lo.base.msg;
    w.L = reinterpret_cast<float *>(base + lo.base.L);
    w.phiq = reinterpret_cast<float *>(base + lo.base.phiq);
    w.bits = reinterpret_cast<uint32_t *>(base + lo.base.bits);
    w.n = code->n;
    w.words_m = (code->m + 31) / 32;
    w.words_k = (code->k + 31) / 32;
    w.n_frames = n_slots;
    w.max_iter = max_iter;
    w.et_start = p.et_start;
    w.ZW = (code->tab.Z + 31) / 32;
    w.clip = p.clip > 0.0f ? p.clip * kLog2e : INFINITY;
    w.xmin = p.phi_floor * kLog2e;
    w.xmin_h = heavy_out_floor(w.clip, w.xmin);
    w.phi_lo = psi_host(w.clip);
    w.phi_hi = psi_host(w.xmin);
    w.cn_nt = p.cn_threads;
    w.vn_vpt = p.vn_nodes;
    w.vn_split = p.vn_split;
    w.wait_polls = kWaitLimit;
    if (layered) {
        w.layered = 1;
        w.ngroups = p.layers > 0 ? p.layers : code->tab.mb;
        w.msg_buf = (int64_t)n_slots * code->tab.n_h * code->tab.Z;
    }
    w.fmt = p.msg_format;
    if (w.fmt == 2) {
        const float step = p.msg_step > 0.0f ? p.msg_step : (p.clip > 0.0f ? p.clip : 15.0f) / 127.0f;
        w.qstep = step * kLog2e;
        w.qinv = 1.0f / w.qstep;
    }
    set_accum(code, p, base + lo.base.acc, w);
    pool->code = code;
    pool->n_slots = n_slots;
    pool_reset_kernel<<<std::max(1, std::min(1024, (n_slots + kThreads - 1) / kThreads)), kThreads, 0,
                        (cudaStream_t)stream>>>(w);
    err = cudaGetLastError();
    if (err != cudaSuccess) {
        delete pool;
        return cuda_fail(err, "pool_create: launch");
    }
    clear_error();
    *out = pool;
    return QCLDPC_OK;
}

extern "C" void qcldpc_pool_destroy(qcldpc_pool *pool) {
    if (!pool) return;
    {
        // drop cached multi-pool graphs that step this pool
        std::lock_guard<std::mutex> lock(g_multi_mu);
        for (auto &m : g_multi) {
            if (m.exec && std::find(m.pools.begin(), m.pools.end(), pool) != m.pools.end()) {
                cudaGraphExecDestroy(m.exec);
                cudaGraphDestroy(m.graph);
                m.exec = nullptr;
                m.graph = nullptr;
                m.pools.clear();
            }
        }
    }
    for (auto &g : pool->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    delete pool;
}

extern "C" int qcldpc_pool_state(const qcldpc_pool *pool, const int32_t **state_dev) {
    if (!pool || !state_dev) return qc::fail(QCLDPC_E_INVAL, "pool_state: NULL argument");
    *state_dev = pool->w.state;
    return QCLDPC_OK;
}

extern "C" int qcldpc_pool_load(qcldpc_pool *pool, int n, const int32_t *slots_dev,
                                const float *llr_dev, const uint32_t *syn_dev,
                                qcldpc_stream_t stream) {
    using namespace qc;
    if (!pool || n < 0 || n > pool->n_slots) return fail(QCLDPC_E_INVAL, "pool_load: bad argument");
    if (n == 0) return QCLDPC_OK;
    if (!slots_dev || !llr_dev || !syn_dev) return fail(QCLDPC_E_INVAL, "pool_load: NULL buffer");
    if (!aligned(slots_dev, 4) || !aligned(llr_dev, 4) || !aligned(syn_dev, 4))
        return fail(QCLDPC_E_ALIGN, "pool_load: buffers must be 4-byte aligned");
    std::lock_guard<std::mutex> lock(pool->code->mu);
    pool_load_kernel<<<sm_count() * 4, kThreads, 0, (cudaStream_t)stream>>>(pool->code->tab, pool->w,
                                                                         slots_dev, n, llr_dev, syn_dev);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "pool_load: launch");
    return QCLDPC_OK;
}

extern "C" int qcldpc_pools_step(int n_pools, qcldpc_pool *const *pools, int n_passes,
                                 qcldpc_stream_t stream) {
    using namespace qc;
    if (n_pools < 1 || !pools || n_passes < 1) return fail(QCLDPC_E_INVAL, "pools_step: bad argument");
    for (int i = 0; i < n_pools; i++)
        if (!pools[i]) return fail(QCLDPC_E_INVAL, "pools_step: NULL pool");
    // A single pool caches its step graph; several pools build a fresh graph
    // with one branch per pool (their passes run concurrently).
    cudaError_t err;
    if (n_pools == 1) {
        qcldpc_pool *pool = pools[0];
        std::lock_guard<std::mutex> lock(pool->code->mu);
        qcldpc_pool::StepGraph *hit = nullptr;
        for (auto &g : pool->graphs)
            if (g.exec && g.passes == n_passes) hit = &g;
        if (!hit) {
            hit = &pool->graphs[pool->next_graph];
            pool->next_graph = (pool->next_graph + 1) % kPoolGraphs;
            if (hit->exec) cudaGraphExecDestroy(hit->exec);
            if (hit->graph) cudaGraphDestroy(hit->graph);
            hit->exec = nullptr;
            hit->graph = nullptr;
            if ((err = cudaGraphCreate(&hit->graph, 0)) != cudaSuccess) return cuda_fail(err, "pools_step: cudaGraphCreate");
            cudaGraphNode_t last;
            if ((err = add_pool_passes(hit->graph, pool, n_passes, &last)) != cudaSuccess)
                return cuda_fail(err, "pools_step: add passes");
            if ((err = cudaGraphInstantiate(&hit->exec, hit->graph, cudaGraphInstantiateFlagUseNodePriority)) !=
                cudaSuccess) {
                hit->exec = nullptr;
                return cuda_fail(err, "pools_step: cudaGraphInstantiate");
            }
            hit->passes = n_passes;
        }
        if ((err = cudaGraphLaunch(hit->exec, (cudaStream_t)stream)) != cudaSuccess)
            return cuda_fail(err, "pools_step: cudaGraphLaunch");
        return QCLDPC_OK;
    }
    std::lock_guard<std::mutex> lock(g_multi_mu);
    MultiGraph *hit = nullptr, *victim = &g_multi[0];
    for (auto &m : g_multi) {
        if (m.exec && m.passes == n_passes && m.pools.size() == (size_t)n_pools &&
            std::equal(m.pools.begin(), m.pools.end(), pools))
            hit = &m;
        if (!m.exec || (victim->exec && m.stamp < victim->stamp)) victim = &m;
    }
    if (!hit) {
        hit = victim;
        if (hit->exec) cudaGraphExecDestroy(hit->exec);
        if (hit->graph) cudaGraphDestroy(hit->graph);
        hit->exec = nullptr;
        hit->graph = nullptr;
        if ((err = cudaGraphCreate(&hit->graph, 0)) != cudaSuccess)
            return cuda_fail(err, "pools_step: cudaGraphCreate");
        err = cudaSuccess;
        for (int i = 0; i < n_pools && err == cudaSuccess; i++) {
            cudaGraphNode_t last;
            err = add_pool_passes(hit->graph, pools[i], n_passes, &last);
        }
        if (err == cudaSuccess)
            err = cudaGraphInstantiate(&hit->exec, hit->graph, cudaGraphInstantiateFlagUseNodePriority);
        if (err != cudaSuccess) {
            hit->exec = nullptr;
            return cuda_fail(err, "pools_step: build graph");
        }
        hit->pools.assign(pools, pools + n_pools);
        hit->passes = n_passes;
    }
    hit->stamp = ++g_multi_clock;
    if ((err = cudaGraphLaunch(hit->exec, (cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(err, "pools_step: cudaGraphLaunch");
    return QCLDPC_OK;
}

extern "C" int qcldpc_pool_step(qcldpc_pool *pool, int n_passes, qcldpc_stream_t stream) {
    return qcldpc_pools_step(1, &pool, n_passes, stream);
}

extern "C" int qcldpc_pool_collect(qcldpc_pool *pool, int n, const int32_t *slots_dev,
                                   uint32_t *key_bits_dev, int32_t *converged_dev,
                                   int32_t *iters_dev, qcldpc_stream_t stream) {
    using namespace qc;
    if (!pool || n < 0 || n > pool->n_slots) return fail(QCLDPC_E_INVAL, "pool_collect: bad argument");
    if (n == 0) return QCLDPC_OK;
    if (!slots_dev || !key_bits_dev || !converged_dev || !iters_dev)
        return fail(QCLDPC_E_INVAL, "pool_collect: NULL buffer");
    std::lock_guard<std::mutex> lock(pool->code->mu);
    cudaStream_t st = (cudaStream_t)stream;
    pool_collect_kernel<<<sm_count() * 2, kThreads, 0, st>>>(pool->code->tab, pool->w, slots_dev, n,
                                                            key_bits_dev, converged_dev, iters_dev);
    pool_free_kernel<<<1, kThreads, 0, st>>>(pool->w, slots_dev, n);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "pool_collect: launch");
    return QCLDPC_OK;
}

// ---------------------------------------------------------------------------
// Decoding without caller-provided or library-allocated scratch.
//
// Some callers cannot allocate device memory: for example code embedded in a
// host framework that owns the device allocator and does not expose it, or a
// process whose device memory is reserved once at start-up and may not grow.
// For them qcldpc_decode_noalloc keeps the decoder's scratch in this file-
// scope device array, which every GPU that loads the library holds until the
// process exits. Host code must not use the array's name as an address (on
// the host it is only a stand-in); the device address is fetched once per
// device with cudaGetSymbolAddress and passed to the kernels.
constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoallocMaxDevices];  // device address per device, set on first use
}  // namespace

extern "C" int qcldpc_decode_noalloc(const qcldpc_code *code, const float *llr_dev,
                                     const uint32_t *syn_dev, int n_frames, int max_iter,
                                     const qcldpc_params *p, uint32_t *key_bits_dev,
                                     int32_t *converged_dev, int32_t *iters_dev,
                                     qcldpc_stream_t stream) {
    using namespace qc;
    if (!code) return fail(QCLDPC_E_INVAL, "decode_noalloc: code is NULL");
    if (n_frames < 0 || n_frames > 65535)
        return fail(QCLDPC_E_INVAL, "decode_noalloc: n_frames must be in [0, 65535]");
    const size_t need =
        layout_of(code->tab, n_frames, false, p ? p->msg_format : 0, p && p->schedule == 1).total;
    if (need > kNoallocScratchBytes)
        return fail(QCLDPC_E_UNSUPPORTED,
                    "decode_noalloc: this code and frame count need " + std::to_string(need) +
                        " bytes of scratch; the static scratch holds " +
                        std::to_string(kNoallocScratchBytes) + " bytes (decode fewer frames)");
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return cuda_fail(err, "decode_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kNoallocMaxDevices)
        return fail(QCLDPC_E_UNSUPPORTED, "decode_noalloc: device ordinal above 63");
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            err = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (err != cudaSuccess) return cuda_fail(err, "decode_noalloc: cudaGetSymbolAddress");
            g_noalloc_ptr[dev] = ptr;
        }
        scratch = g_noalloc_ptr[dev];
    }
    qcldpc_params q;
    if (p) q = *p;
    else qcldpc_params_init(&q);
    q.launch_mode = 1;  // plain launches: no graph objects to instantiate
    q.soft_output = 0;
    return decode_impl(code, llr_dev, syn_dev, n_frames, max_iter, &q, key_bits_dev,
                       converged_dev, iters_dev, nullptr, scratch, kNoallocScratchBytes,
                       (cudaStream_t)stream);
}
