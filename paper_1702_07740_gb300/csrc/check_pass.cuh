// Check-node pass of the decoder (Algorithm 1, Steps 2 and 4 for degree-1
// nodes, and the stop test), included once per message storage format by
// check_pass_f32.cu, check_pass_f16.cu and check_pass_i8.cu, which export
// its kernels through qc::cn_kernel_<format>.
//
// Each kernel comes in two block shapes: NT = kCnThreads (compile-time strides,
// rows of Z > (kTile - kTile / 4) checks), and NT = 0, which reads its width
// from blockDim.x (the launch sizes short rows to fit; the run-time strides
// cost registers, so full rows keep the first form).
#pragma once

#include "decode_common.cuh"

namespace {
// ---- check-node pass
//
// Pass modes (uniform per launch): iteration 1 updates without reading old
// messages; later iterations read them; the stop test of iteration t-1 runs
// when t-1 >= et_start; the pass after the last iteration only tests.
enum CnMode { kFirst = 0, kSteady = 1, kSteadyTest = 2, kTestOnly = 3 };

// Any row shape up to MAXD circulants (heavy first), runtime degree with
// predication; used for shapes the exact instantiations do not cover.
template <int MAXD, typename M>
__device__ __forceinline__ bool cn_row_generic(const Table &T, const Work &W, int f, int r, int t,
                                               int mode, int i0, int vpt, int stride) {
    const bool update = mode != kTestOnly;
    const bool read_msg = mode == kSteady || mode == kSteadyTest;
    const bool test = mode == kSteadyTest || mode == kTestOnly;
    const int Z = T.Z, ZW = W.ZW;
    const int rp = T.row_ptr[r];
    const int deg = T.row_ptr[r + 1] - rp;
    const int nh = T.row_nh[r];
    const M *msg_rd = static_cast<const M *>(W.msg) + ((t - 1) & 1) * W.msg_buf + (size_t)f * T.n_h * Z;
    M *msg = static_cast<M *>(W.msg) + (t & 1) * W.msg_buf + (size_t)f * T.n_h * Z;
    const float *L = W.L + (size_t)f * T.n_hcols * 2 * Z;
    int32_t *acc = W.acc + (size_t)f * T.n_hcols * 2 * Z;
    const float *phiq = W.phiq + (size_t)f * T.n_d1 * Z;
    const size_t bstride = (size_t)T.n_d1 * ZW;
    uint32_t *bcur = W.bits + ((size_t)(t & 1) * W.n_frames + f) * bstride;
    const uint32_t *bprev = W.bits + ((size_t)((t - 1) & 1) * W.n_frames + f) * bstride;
    const uint32_t *syn = W.syn + (size_t)f * W.words_m;
    bool bad = false;
    for (int u = 0; u < vpt; u++) {
        const int i = i0 + u * stride;
        const bool valid = i < Z;
        const int cidx = r * Z + i;
        const uint32_t sbit = __ldg(syn + min(cidx >> 5, (int)W.words_m - 1)) << (31 - (cidx & 31));
        float phi[MAXD];
        uint32_t sg[MAXD];
        uint32_t stot = sbit, par = sbit;
#pragma unroll
        for (int k = 0; k < MAXD; k++) {
            phi[k] = 0.0f;
            sg[k] = 0;
            if (k < deg) {
                const int oa = T.row_off_a[rp + k], ob = T.row_off_b[rp + k];
                if (k < nh) {
                    const float lv = L[oa + i];
                    par ^= fbits(lv);
                    const float d = lv - (read_msg ? Codec<M>::dec(msg_rd[ob + i], W) : 0.0f);
                    phi[k] = psi_f(fminf(fmaxf(fabsf(d), W.xmin), W.clip));
                    sg[k] = fbits(d);
                } else {
                    const float p = update ? __ldg(phiq + oa + i) : 0.0f;
                    if (test) par ^= __ldg(bprev + ob + (i >> 5)) << (31 - (i & 31));
                    phi[k] = fabsf(p);
                    sg[k] = fbits(p);
                }
                stot ^= sg[k];
            }
        }
        if (test) bad |= valid && (par & kSign) != 0;
        if (!update) continue;
        float pre[MAXD + 1], suf[MAXD + 1];
        pre[0] = 0.0f;
#pragma unroll
        for (int k = 0; k < MAXD; k++) pre[k + 1] = pre[k] + phi[k];
        suf[MAXD] = 0.0f;
#pragma unroll
        for (int k = MAXD - 1; k >= 0; k--) suf[k] = suf[k + 1] + phi[k];
#pragma unroll
        for (int k = 0; k < MAXD; k++) {
            if (k >= deg) break;
            const qc::RowEnt e = T.rows[rp + k];
            const int oa = T.row_off_a[rp + k], ob = T.row_off_b[rp + k];
            const float ex = fmaxf(pre[k] + suf[k + 1], W.xmin);
            const uint32_t sk = (stot ^ sg[k]) & kSign;
            if (k < nh) {
                const float mag = fminf(psi_f(ex), W.clip);
                const M e = Codec<M>::enc(__uint_as_float(fbits(mag) ^ sk), W);
                if (valid) {
                    msg[ob + i] = e;
                    if (W.accum) red_add(acc + oa + i, acc_value(e, W));
                }
            } else {
                const uint32_t dbits = ex < phi[k] ? sk : (sg[k] & kSign);
                const uint32_t word = __ballot_sync(0xffffffffu, valid && dbits != 0);
                if ((threadIdx.x & 31) == 0 && valid) bcur[ob + (i >> 5)] = word;
                if (W.soft && valid) {
                    int vo = i + e.shift;
                    if (vo >= Z) vo -= Z;
                    const float mag = fminf(psi_f(ex), W.clip);
                    float *post1 = W.post1 + ((size_t)(t & 1) * W.n_frames + f) * T.n_d1 * Z;
                    post1[oa + i] = W.llr[(size_t)f * W.n + (size_t)e.col * Z + vo] +
                                    kLn2 * __uint_as_float(fbits(mag) ^ sk);
                }
            }
        }
    }
    return bad;
}

// ---- check-node pass staged through shared memory by bulk async copies
//
// One block of nt threads (a multiple of 32, chosen per code so that the
// tile nt * kTmaVpt fits Z) owns tile consecutive checks (offsets i0 ..
// i0+tile-1) of one base row of one frame. Thread 0 arms an mbarrier and issues one
// cp.async.bulk per operand row: the heavy posteriors at i0 + shift, the old
// messages and the degree-1 psi values at i0, and the degree-1 decision
// words of iteration t-1. Each source start is rounded down to 16 bytes
// (the copy unit) and the remainder is added when reading. Every thread then
// waits on the barrier (bounded) and evaluates its kTmaVpt checks, i0 + c *
// nt + threadIdx.x, from shared memory: consecutive threads read
// consecutive words, so the reads are free of bank conflicts.

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One bounded test of the barrier's phase. With QCLDPC_WAIT_HINT_NS > 0 the
// waiting thread may be suspended for up to that many nanoseconds (it wakes
// when the phase completes), so a warp re-polls far less often while the
// copies are in flight.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
#if QCLDPC_WAIT_HINT_NS > 0
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "n"(QCLDPC_WAIT_HINT_NS)
        : "memory");
#else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
#endif
    return ok != 0;
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bytes to stage for `count` elements of `esize` bytes starting at `src`
// once the start is rounded down to 16 bytes; *rem receives the offset of
// src[0], in elements, from that rounded start.
__device__ __forceinline__ uint32_t stage_bytes(const void *src, uint32_t count, int esize,
                                                int *rem) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(src);
    *rem = (int)((a & 15u) / (uintptr_t)esize);
    return ((uint32_t)(*rem + count) * (uint32_t)esize + 15u) & ~15u;
}

// Bounded wait for the staged operands. On timeout the block records a
// device error (decoding stops with converged = -1), waits once more
// (bounded) for its copies, and reports failure.
__device__ __forceinline__ bool stage_wait(uint64_t *bar, const Work &W) {
    for (unsigned it = 0; it < W.wait_polls; it++)
        if (mbar_try_wait(bar, 0)) return true;
    atomicOr(W.err, 1);
    for (unsigned it = 0; it < W.wait_polls; it++)
        if (mbar_try_wait(bar, 0)) break;
    return false;
}

// Soft output of a degree-1 neighbour (row entry e, check i) at iteration t:
// its posterior Q_p + m_cp in natural units, where the message has sign sk
// and psi-domain magnitude psi(ex) (clipped).
__device__ __noinline__ void soft_deg1(const Table &T, const Work &W, int f, int t, int e, int i,
                                       float ex, uint32_t sk) {
    const int Z = T.Z;
    const qc::RowEnt re = T.rows[e];
    int vo = i + re.shift;
    if (vo >= Z) vo -= Z;
    const float mag = fminf(psi_f(ex), W.clip);
    float *post1 = W.post1 + ((size_t)(t & 1) * W.n_frames + f) * T.n_d1 * Z;
    post1[T.row_off_a[e] + i] =
        W.llr[(size_t)f * W.n + (size_t)re.col * Z + vo] + kLn2 * __uint_as_float(fbits(mag) ^ sk);
}

// The arithmetic of one tile of checks i0 .. i0 + nt * kTmaVpt - 1 of base
// row r, frame f, from operand rows staged in shared memory (s_off: each
// row's first element, in units of its element type, from `stage`). ob: the
// row entries' output offsets. sy0 / b0: the syndrome word holding check
// r Z + i0 and that check's bit in it (a global pointer, or a staged copy
// when SYN_SMEM). wait() runs after the syndrome loads and reports whether
// the staged rows arrived. Thread tid < nt owns checks i0 + c nt + tid.
template <int NH, int ND, int MODE, typename M, int NT, bool SYN_SMEM, typename Wait>
__device__ __forceinline__ bool cn_compute(const Table &T, const Work &W, int f, int r, int rp, int t,
                                           int i0, const int *oa, const int *ob, const int *s_off,
                                           const float *stage, const uint32_t *sy0, int b0, Wait wait) {
    constexpr int D = NH + ND;
    constexpr int NHa = NH > 0 ? NH : 1;
    constexpr int NDa = ND > 0 ? ND : 1;
    constexpr bool kUpdate = MODE != kTestOnly;
    constexpr bool kReadMsg = MODE == kSteady || MODE == kSteadyTest;
    constexpr bool kTest = MODE == kSteadyTest || MODE == kTestOnly;
    const int Z = T.Z, ZW = W.ZW;
    const int nt = NT ? NT : (int)blockDim.x;  // threads: a multiple of 32, at most kCnThreads
    const int ws = nt >> 5;                    // decision words per check slot
    const int tid = threadIdx.x;
    const size_t bstride = (size_t)T.n_d1 * ZW;
    M *msg = static_cast<M *>(W.msg) + (t & 1) * W.msg_buf + (size_t)f * T.n_h * Z;

    // Per-row pointers for this thread's first check; check c sits at
    // + c * nt elements (or + c * ws words).
    const float *pL[NHa], *pP[NDa];
    const M *pM[NHa];
    const uint32_t *pB[NDa];
    {
        int q = 0;
#pragma unroll
        for (int k = 0; k < NH; k++) pL[k] = stage + s_off[q++] + tid;
        if (kReadMsg) {
#pragma unroll
            for (int k = 0; k < NH; k++) pM[k] = reinterpret_cast<const M *>(stage) + s_off[q++] + tid;
        }
        if (kUpdate) {
#pragma unroll
            for (int k = 0; k < ND; k++) pP[k] = stage + s_off[q++] + tid;
        }
        if (kTest) {
#pragma unroll
            for (int k = 0; k < ND; k++)
                pB[k] = reinterpret_cast<const uint32_t *>(stage) + s_off[q++] + (tid >> 5);
        }
    }
    // Output rows at this thread's first check; oA: the heavy nodes'
    // accumulators at the posterior offsets (node (i + s) mod Z collects at
    // i + s, below 2Z).
    M *oM[NHa];
    uint32_t *oB[NDa];
    {
        uint32_t *bcur = W.bits + ((size_t)(t & 1) * W.n_frames + f) * bstride;
#pragma unroll
        for (int k = 0; k < D; k++) {
            if (k < NH) oM[k] = msg + ob[k] + i0 + tid;
            else oB[k - NH] = bcur + ob[k] + (i0 >> 5) + (tid >> 5);
        }
    }
    // accumulator of heavy entry k for this thread's check c: accb + oa[k] + c nt
    int32_t *accb = W.acc + (size_t)f * T.n_hcols * 2 * Z + i0 + tid;
    const bool accum = W.accum != 0;
    // syndrome words of the owned checks (check c of this thread sits c * ws
    // words after the first), loaded while the copies are in flight
    const int sb = b0 + tid;
    const uint32_t *sy = sy0 + (sb >> 5);
    const int ssh = 31 - (sb & 31);
    const int dsh = 31 - (tid & 31);
    const bool lane0 = (tid & 31) == 0;
    uint32_t sw[kTmaVpt];
#pragma unroll
    for (int c = 0; c < kTmaVpt; c++)
        sw[c] = i0 + c * nt + tid < Z ? ((SYN_SMEM ? sy[c * ws] : __ldg(sy + c * ws)) << ssh) : 0u;

    const bool staged = wait();
    bool bad = false;
    if (staged) {
      if constexpr (QCLDPC_CN_PAIR && kTmaVpt % 2 == 0) {
        // Two checks (c, c + 1) per step, their arithmetic in packed FP32x2
        // operations (per lane identical to the scalar path below).
#pragma unroll kCnUnroll
        for (int c = 0; c < kTmaVpt; c += 2) {
            if (i0 + c * nt + (tid & ~31) >= Z) break;  // warp-uniform: no check of this warp left
            const int ia = i0 + c * nt + tid, ib = ia + nt;
            const bool va = ia < Z, vb = ib < Z;
            float2 lv[NHa], phi[D];
            uint32_t sga[D], sgb[D];
            uint32_t sta = sw[c], stb = sw[c + 1], pa = sw[c], pb = sw[c + 1];
#pragma unroll
            for (int k = 0; k < NH; k++) {
                lv[k] = make_float2(pL[k][c * nt], pL[k][(c + 1) * nt]);
                pa ^= fbits(lv[k].x);
                pb ^= fbits(lv[k].y);
            }
            if (kTest) {
#pragma unroll
                for (int k = 0; k < ND; k++) {
                    pa ^= pB[k][c * ws] << dsh;
                    pb ^= pB[k][(c + 1) * ws] << dsh;
                }
                bad |= (va && (pa & kSign) != 0) || (vb && (pb & kSign) != 0);
            }
            if constexpr (kUpdate) {
#pragma unroll
                for (int k = 0; k < NH; k++) {
                    float2 d = lv[k];
                    if (kReadMsg) {
                        const float2 m = make_float2(Codec<M>::dec(pM[k][c * nt], W),
                                                     Codec<M>::dec(pM[k][(c + 1) * nt], W));
                        d = __ffma2_rn(m, f2(-1.0f), d);  // lv - m, one rounding
                    }
                    phi[k] = psi2_clamped(d, W.phi_lo, W.phi_hi);
                    sga[k] = fbits(d.x);
                    sgb[k] = fbits(d.y);
                    sta ^= sga[k];
                    stb ^= sgb[k];
                }
#pragma unroll
                for (int k = 0; k < ND; k++) {
                    const float qa = pP[k][c * nt], qb = pP[k][(c + 1) * nt];
                    phi[NH + k] = make_float2(fabsf(qa), fabsf(qb));
                    sga[NH + k] = fbits(qa);
                    sgb[NH + k] = fbits(qb);
                    sta ^= sga[NH + k];
                    stb ^= sgb[NH + k];
                }
                // exclusive sums by prefix / suffix (psi >= +0, so 0 + x = x)
                float2 pre[D], suf[D];
                pre[0] = phi[0];
#pragma unroll
                for (int k = 1; k < D; k++) pre[k] = __fadd2_rn(pre[k - 1], phi[k]);
                suf[D - 1] = phi[D - 1];
#pragma unroll
                for (int k = D - 2; k >= 0; k--) suf[k] = __fadd2_rn(suf[k + 1], phi[k]);
#pragma unroll
                for (int k = 0; k < D; k++) {
                    const float2 s2 = k == 0       ? suf[1]
                                      : k == D - 1 ? pre[D - 2]
                                                   : __fadd2_rn(pre[k - 1], suf[k + 1]);
                    const uint32_t ska = (sta ^ sga[k]) & kSign, skb = (stb ^ sgb[k]) & kSign;
                    if (k < NH) {
                        // min(psi(max(s, xmin)), clip) = psi(max(s, xmin_h))
                        const float2 mag = psi2(make_float2(fmaxf(s2.x, W.xmin_h), fmaxf(s2.y, W.xmin_h)));
                        const M ea = Codec<M>::enc(__uint_as_float(fbits(mag.x) ^ ska), W);
                        const M eb = Codec<M>::enc(__uint_as_float(fbits(mag.y) ^ skb), W);
                        if (va) oM[k][c * nt] = ea;
                        if (vb) oM[k][(c + 1) * nt] = eb;
                        if (accum) {
                            if (va) red_add(accb + (oa[k] + c * nt), acc_value(ea, W));
                            if (vb) red_add(accb + (oa[k] + (c + 1) * nt), acc_value(eb, W));
                        }
                    } else {
                        const float2 ex = make_float2(fmaxf(s2.x, W.xmin), fmaxf(s2.y, W.xmin));
                        const uint32_t da = ex.x < phi[k].x ? ska : (sga[k] & kSign);
                        const uint32_t db = ex.y < phi[k].y ? skb : (sgb[k] & kSign);
                        const uint32_t wa = __ballot_sync(0xffffffffu, va && da != 0);
                        const uint32_t wb = __ballot_sync(0xffffffffu, vb && db != 0);
                        if (lane0 && va) oB[k - NH][c * ws] = wa;
                        if (lane0 && vb) oB[k - NH][(c + 1) * ws] = wb;
                        if (W.soft) {
                            if (va) soft_deg1(T, W, f, t, rp + k, ia, ex.x, ska);
                            if (vb) soft_deg1(T, W, f, t, rp + k, ib, ex.y, skb);
                        }
                    }
                }
            }
        }
      } else {
#pragma unroll kCnUnroll
        for (int c = 0; c < kTmaVpt; c++) {
            if (i0 + c * nt + (tid & ~31) >= Z) break;  // warp-uniform: no check of this warp left
            const int i = i0 + c * nt + tid;
            const bool valid = i < Z;
            const uint32_t sb = sw[c];
            float lv[NHa], phi[D];
            uint32_t sg[D];
            uint32_t stot = sb, par = sb;
#pragma unroll
            for (int k = 0; k < NH; k++) {
                lv[k] = pL[k][c * nt];
                par ^= fbits(lv[k]);
            }
            if (kTest) {
#pragma unroll
                for (int k = 0; k < ND; k++) par ^= pB[k][c * ws] << dsh;
                bad |= valid && (par & kSign) != 0;
            }
            if constexpr (kUpdate) {
#pragma unroll
                for (int k = 0; k < NH; k++) {
                    const float d = lv[k] - (kReadMsg ? Codec<M>::dec(pM[k][c * nt], W) : 0.0f);
                    phi[k] = psi_clamped(d, W.phi_lo, W.phi_hi);
                    sg[k] = fbits(d);
                    stot ^= sg[k];
                }
#pragma unroll
                for (int k = 0; k < ND; k++) {
                    const float p = pP[k][c * nt];
                    phi[NH + k] = fabsf(p);
                    sg[NH + k] = fbits(p);
                    stot ^= sg[NH + k];
                }
                float pre[D + 1], suf[D + 1];
                pre[0] = 0.0f;
#pragma unroll
                for (int k = 0; k < D; k++) pre[k + 1] = pre[k] + phi[k];
                suf[D] = 0.0f;
#pragma unroll
                for (int k = D - 1; k >= 0; k--) suf[k] = suf[k + 1] + phi[k];
#pragma unroll
                for (int k = 0; k < D; k++) {
                    const float s1 = pre[k] + suf[k + 1];
                    const uint32_t sk = (stot ^ sg[k]) & kSign;  // sign of m_cv
                    if (k < NH) {
                        const float mag = psi_f(fmaxf(s1, W.xmin_h));
                        const M e = Codec<M>::enc(__uint_as_float(fbits(mag) ^ sk), W);
                        if (valid) {
                            oM[k][c * nt] = e;
                            if (accum) red_add(accb + (oa[k] + c * nt), acc_value(e, W));
                        }
                    } else {
                        const float ex = fmaxf(s1, W.xmin);
                        const uint32_t dbits = ex < phi[k] ? sk : (sg[k] & kSign);
                        const uint32_t word = __ballot_sync(0xffffffffu, valid && dbits != 0);
                        if (lane0 && valid) oB[k - NH][c * ws] = word;
                        if (W.soft && valid) soft_deg1(T, W, f, t, rp + k, i, ex, sk);
                    }
                }
            }
        }
      }
    }
    return bad;
}

template <int NH, int ND, int MODE, typename M, int NT>
__device__ __forceinline__ bool cn_tile(const Table &T, const Work &W, int f, int r, int rp, int t,
                                        const qc::RowDesc *dp, unsigned char *smem) {
    constexpr int NHa = NH > 0 ? NH : 1;
    constexpr int NDa = ND > 0 ? ND : 1;
    constexpr bool kUpdate = MODE != kTestOnly;
    constexpr bool kReadMsg = MODE == kSteady || MODE == kSteadyTest;
    constexpr bool kTest = MODE == kSteadyTest || MODE == kTestOnly;
    const int Z = T.Z, ZW = W.ZW;
    int oa[qc::kDescEnts], ob[qc::kDescEnts];
    load_offsets(dp, oa, ob);
    const int nt = NT ? NT : (int)blockDim.x;  // threads: a multiple of 32, at most kCnThreads
    const int tile = nt * kTmaVpt;     // checks per block
    const int i0 = blockIdx.x * tile;
    const int tid = threadIdx.x;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    int *s_off = reinterpret_cast<int *>(smem + 16);  // per staged row: start of its data
    float *stage = reinterpret_cast<float *>(smem + kSmemHeader);
    const size_t bstride = (size_t)T.n_d1 * ZW;
    // messages of iteration t-1 (read); layered decoding writes those of t
    // to the other buffer
    const M *msg_rd = static_cast<const M *>(W.msg) + ((t - 1) & 1) * W.msg_buf + (size_t)f * T.n_h * Z;

    // Thread 0: arm the barrier, publish each staged row's read offset
    // (row slot * (tile + 4) + 16-byte remainder), then issue the copies.
    // Staged rows: NH posteriors, NH old messages (kReadMsg), ND psi values
    // (kUpdate), then ND decision-word rows of tile / 32 + 4 words (kTest).
    if (tid == 0) {
        const float *L = W.L + (size_t)f * T.n_hcols * 2 * Z;
        const float *phiq = W.phiq + (size_t)f * T.n_d1 * Z;
        const uint32_t *bprev = W.bits + ((size_t)((t - 1) & 1) * W.n_frames + f) * bstride;
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const void *src[2 * NHa + 2 * NDa];
        uint32_t nb[2 * NHa + 2 * NDa];
        int slot_start[2 * NHa + 2 * NDa];
        int ncopy = 0, pos = 0;
        uint32_t total = 0;
        // Each staged row takes row_slots 4-byte slots; s_off holds the row's
        // first element in units of its own element size.
        auto add = [&](const void *p, uint32_t count, int esize, int row_slots) {
            int rem;
            nb[ncopy] = stage_bytes(p, count, esize, &rem);
            src[ncopy] = reinterpret_cast<const char *>(p) - esize * rem;
            slot_start[ncopy] = pos;
            s_off[ncopy] = pos * (4 / esize) + rem;
            total += nb[ncopy];
            pos += row_slots;
            ncopy++;
        };
        // only the tile's checks below Z are copied (the last tile of a row
        // would otherwise pull in its neighbour's data)
        const uint32_t nv = (uint32_t)min(tile, Z - i0);
        const int row_slots = tile + 4, word_slots = tile / 32 + 4;
#pragma unroll
        for (int k = 0; k < NH; k++) add(L + oa[k] + i0, nv, 4, row_slots);
        if (kReadMsg) {
#pragma unroll
            for (int k = 0; k < NH; k++)
                add(msg_rd + ob[k] + i0, nv, (int)sizeof(M), row_slots);
        }
        if (kUpdate) {
#pragma unroll
            for (int k = 0; k < ND; k++) add(phiq + oa[NH + k] + i0, nv, 4, row_slots);
        }
        if (kTest) {
#pragma unroll
            for (int k = 0; k < ND; k++)
                add(bprev + ob[NH + k] + (i0 >> 5), (nv + 31) / 32, 4, word_slots);
        }
        mbar_expect_tx(bar, total + W.stall_extra);
        for (int q = 0; q < ncopy; q++) bulk_g2s(stage + slot_start[q], src[q], nb[q], bar);
    }
    __syncthreads();  // barrier initialised, offsets published

    const int cb0 = r * Z + i0;
    const bool bad = cn_compute<NH, ND, MODE, M, NT, false>(
        T, W, f, r, rp, t, i0, oa, ob, s_off, stage, W.syn + (size_t)f * W.words_m + (cb0 >> 5), cb0 & 31,
        [&] { return stage_wait(bar, W); });
    __syncthreads();
    if (tid == 0) mbar_inval(bar);
    return bad;
}

template <int MODE, typename M, int NT>
__device__ __forceinline__ bool cn_tile_dispatch(const Table &T, const Work &W, int f, int r, int t,
                                                 int rp, int nh, int nd, const qc::RowDesc *dp,
                                                 unsigned char *smem) {
    switch (nh * 4 + nd) {
        case 1 * 4 + 1: return cn_tile<1, 1, MODE, M, NT>(T, W, f, r, rp, t, dp, smem);
        case 2 * 4 + 0: return cn_tile<2, 0, MODE, M, NT>(T, W, f, r, rp, t, dp, smem);
        case 2 * 4 + 1: return cn_tile<2, 1, MODE, M, NT>(T, W, f, r, rp, t, dp, smem);
        case 3 * 4 + 0: return cn_tile<3, 0, MODE, M, NT>(T, W, f, r, rp, t, dp, smem);
        case 3 * 4 + 1: return cn_tile<3, 1, MODE, M, NT>(T, W, f, r, rp, t, dp, smem);
        case 4 * 4 + 0: return cn_tile<4, 0, MODE, M, NT>(T, W, f, r, rp, t, dp, smem);
        case 4 * 4 + 1: return cn_tile<4, 1, MODE, M, NT>(T, W, f, r, rp, t, dp, smem);
        default: return false;
    }
}


// Check-node pass of iteration t, staged variant: grid (ceil(Z / tile), base
// row, frame) with blocks of cn_launch's thread count, dynamic shared memory
// sized by cn_launch for the code's widest exact-shape row. Rows of other
// shapes take the generic path.
template <int MAXD, typename M, int NT>
__global__ void __launch_bounds__(kCnThreads, NT ? QCLDPC_CN_TMA_MINBLOCKS : QCLDPC_CN_FIT_MINBLOCKS)
    cn_tma_kernel(const __grid_constant__ Table T, const __grid_constant__ Work W) {
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_launch_dependents();  // the control step may be scheduled; it waits for this pass
    pdl_wait();  // after a programmatic edge: the previous variable pass is complete
    const int f = blockIdx.z;
    if (W.active[f] == 0) return;  // block-uniform
    const bool group = W.pass == kPassGroup;
    const qc::RowDesc *dp = group ? T.row_desc + (W.lrow0 + (int)blockIdx.y) : T.row_desc_ord + blockIdx.y;
    const int4 head = __ldg(reinterpret_cast<const int4 *>(dp));  // r, rp, nh, nd
    const int r = head.x;
    const int t = W.t[f] - (group ? 1 : 0);
    int mode = t > W.max_iter ? kTestOnly
               : t == 1       ? kFirst
               : (t - 1 >= W.et_start) ? kSteadyTest : kSteady;
    if (W.pass == kPassTest) {
        if (mode != kSteadyTest && mode != kTestOnly) return;  // no test due
        mode = kTestOnly;
    } else if (group) {
        if (mode == kTestOnly) return;
        if (mode == kSteadyTest) mode = kSteady;
    }
    const int rp = head.y, nh = head.z, nd = head.w;
    bool bad;
    if (exact_shape(nh, nd)) {
        switch (mode) {
            case kFirst: bad = cn_tile_dispatch<kFirst, M, NT>(T, W, f, r, t, rp, nh, nd, dp, smem); break;
            case kSteady: bad = cn_tile_dispatch<kSteady, M, NT>(T, W, f, r, t, rp, nh, nd, dp, smem); break;
            case kSteadyTest: bad = cn_tile_dispatch<kSteadyTest, M, NT>(T, W, f, r, t, rp, nh, nd, dp, smem); break;
            default: bad = cn_tile_dispatch<kTestOnly, M, NT>(T, W, f, r, t, rp, nh, nd, dp, smem); break;
        }
    } else {
        bad = cn_row_generic<MAXD, M>(T, W, f, r, t, mode, blockIdx.x * blockDim.x * kTmaVpt + threadIdx.x,
                                      kTmaVpt, (int)blockDim.x);
    }
    if (mode == kSteadyTest || mode == kTestOnly) {
        if (__syncthreads_or(bad) && threadIdx.x == 0) W.fail[f] = 1;
    }
}


template <typename M>
void *cn_kernel_select(int maxdeg, int nt) {
    if (nt == kCnThreads) {
        if (maxdeg <= 5) return (void *)cn_tma_kernel<5, M, kCnThreads>;
        if (maxdeg <= 8) return (void *)cn_tma_kernel<8, M, kCnThreads>;
        return (void *)cn_tma_kernel<16, M, kCnThreads>;
    }
    if (maxdeg <= 5) return (void *)cn_tma_kernel<5, M, 0>;
    if (maxdeg <= 8) return (void *)cn_tma_kernel<8, M, 0>;
    return (void *)cn_tma_kernel<16, M, 0>;
}

template <typename M>
void cn_raise_smem_cap(int cap) {
    const void *k[] = {(const void *)cn_tma_kernel<5, M, kCnThreads>, (const void *)cn_tma_kernel<8, M, kCnThreads>,
                       (const void *)cn_tma_kernel<16, M, kCnThreads>, (const void *)cn_tma_kernel<5, M, 0>,
                       (const void *)cn_tma_kernel<8, M, 0>, (const void *)cn_tma_kernel<16, M, 0>};
    for (const void *f : k) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
}
}  // namespace
