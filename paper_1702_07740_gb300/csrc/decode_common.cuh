// Device-side definitions shared by the decoder's translation units: launch
// constants, the per-call argument block (Work), the psi function, message
// storage codecs. decode.cu holds the host side and every pass but the check
// pass; check_pass.cuh holds the check pass, compiled once per message
// storage format (check_pass_f32.cu, check_pass_f16.cu, check_pass_i8.cu).
#pragma once

#include <cstdint>

#include <cuda_fp16.h>

#include "qcldpc_internal.cuh"

namespace {

using qc::Table;
using qc::exact_shape;

// Launch shapes (overridable at build time for tuning sweeps). Defaults
// from a sweep at Z = 20,000 with 16 frames on GB300.
#ifndef QCLDPC_VN_VPT
#define QCLDPC_VN_VPT 3
#endif
#ifndef QCLDPC_VN_UNROLL
#define QCLDPC_VN_UNROLL 3
#endif
#ifndef QCLDPC_VN_VPT_MAX
#define QCLDPC_VN_VPT_MAX 3
#endif
constexpr int kVnVptMax = QCLDPC_VN_VPT_MAX;
static_assert(kVnVptMax >= 1 && kVnVptMax <= 3, "variable-pass nodes per thread: 1 to 3");
constexpr int kThreads = 256;
constexpr int kVnVpt = QCLDPC_VN_VPT;  // variable nodes per thread
constexpr int kVnUnroll = QCLDPC_VN_UNROLL;
// Variable pass: each node's sum is kVnParts interleaved partial sums
// (independent chains, added in a fixed order); the loop over a column's
// circulants is unrolled kVnUnroll steps of kVnParts circulants
// (kVnUnrollStaged when the column lists are staged in shared memory).
#ifndef QCLDPC_VN_PARTS
#define QCLDPC_VN_PARTS 2
#endif
constexpr int kVnParts = QCLDPC_VN_PARTS;
static_assert(kThreads % (32 * kVnParts) == 0, "variable-pass part groups must be whole warps");
// Batches below this many 256-node variable-pass blocks per SM split each
// node's parts over thread groups.
#ifndef QCLDPC_VN_SPLIT_BLOCKS
#define QCLDPC_VN_SPLIT_BLOCKS 8
#endif
constexpr int kVnSplitBlocks = QCLDPC_VN_SPLIT_BLOCKS;
#ifndef QCLDPC_VN_UNROLL_STAGED
#define QCLDPC_VN_UNROLL_STAGED 6
#endif
constexpr int kVnUnrollStaged = QCLDPC_VN_UNROLL_STAGED;
constexpr int kColChunk = 128;  // heavy-column circulants staged per chunk by the variable pass
static_assert(kColChunk % kVnParts == 0, "column chunks must keep each circulant's part");
constexpr int kCtrlThreads = 256;
constexpr int kGraphCacheSize = 8;
// Check-node pass with bulk-copy staging: one block stages up to kTile
// consecutive checks of one base row (kTmaVpt per thread) into shared memory.
#ifndef QCLDPC_CN_TVPT
#define QCLDPC_CN_TVPT 4
#endif
constexpr int kTmaVpt = QCLDPC_CN_TVPT;
// Threads of a full check block.
#ifndef QCLDPC_CN_THREADS
#define QCLDPC_CN_THREADS 256
#endif
constexpr int kCnThreads = QCLDPC_CN_THREADS;
// Resident full check blocks per SM the staged pass is compiled for (caps
// registers).
#ifndef QCLDPC_CN_TMA_MINBLOCKS
#define QCLDPC_CN_TMA_MINBLOCKS 5
#endif
// Programmatic dependent launch inside a flooding iteration: the control and
// variable passes are scheduled while their predecessor drains and wait for
// it on the device (griddepcontrol), hiding the launch gaps.
#ifndef QCLDPC_PDL
#define QCLDPC_PDL 1
#endif
// Inside a trip, the next iteration's check pass hangs off the variable pass
// by a programmatic edge (scheduled while the variable pass drains).
#ifndef QCLDPC_PDL_LOOP
#define QCLDPC_PDL_LOOP 1
#endif
// Flooding iterations per trip of the decode graph's WHILE body.
#ifndef QCLDPC_LOOP_UNROLL
#define QCLDPC_LOOP_UNROLL 4
#endif
constexpr int kLoopUnroll = QCLDPC_LOOP_UNROLL;
// Evaluate a thread's checks two at a time in packed FP32x2 arithmetic.
#ifndef QCLDPC_CN_PAIR
#define QCLDPC_CN_PAIR 1
#endif
#ifndef QCLDPC_CN_UNROLL
#define QCLDPC_CN_UNROLL 4
#endif
constexpr int kCnUnroll = QCLDPC_CN_UNROLL;
// Size check blocks to Z (cn_threads); 0 keeps kCnThreads for every code.
#ifndef QCLDPC_CN_FIT
#define QCLDPC_CN_FIT 1
#endif
// Register cap of the variable-width check kernel, as resident full-width
// blocks per SM (its narrower blocks fit more).
#ifndef QCLDPC_CN_FIT_MINBLOCKS
#define QCLDPC_CN_FIT_MINBLOCKS QCLDPC_CN_TMA_MINBLOCKS
#endif
constexpr int kTile = kCnThreads * kTmaVpt;    // checks per block, at most
constexpr int kStage = kTile + 4;              // staged floats per row (16-byte realignment)
constexpr int kStageWords = kTile / 32 + 4;    // staged decision words per row
constexpr int kSmemHeader = 128;               // mbarrier, then 16-byte aligned rows
// Suspend-time hint of the staged check pass's barrier polls, in ns (0: none).
#ifndef QCLDPC_WAIT_HINT_NS
#define QCLDPC_WAIT_HINT_NS 0
#endif
// bounded mbarrier polls before giving up (fewer when each poll may suspend)
#if QCLDPC_WAIT_HINT_NS > 0
constexpr unsigned kWaitLimit = 1u << 14;
#else
constexpr unsigned kWaitLimit = 1u << 22;
#endif
// Padding elements after every workspace array: lanes and staged copies that
// run past a row's end read here (results unused), and never past the array.
constexpr int kSlack = 4096;

// Per-call arguments and workspace pointers (by value in every kernel).
struct Work {
    const float *llr;      // [F][n]
    const uint32_t *syn;   // [F][words_m]
    uint32_t *keys;        // [F][words_k]
    int32_t *conv;         // [F]
    int32_t *iters;        // [F]
    float *post;           // [F][n] or nullptr
    int32_t *t;            // [F] iteration each frame is at
    int32_t *state;        // [F] slot state for pools (0 free, 1 running, 2 stopped) or null
    int32_t *active;       // [F]
    int32_t *fail;         // [F] stop-test failures of the current pass
    int32_t *err;          // device error word (a bounded wait gave up)
    void *msg;             // [F][n_h][Z] messages in the storage format fmt (layered:
                           // two such buffers msg_buf elements apart, by iteration parity)
    float *L;              // [F][n_hcols][2Z]
    float *phiq;           // [F][n_d1][Z]
    uint32_t *bits;        // [2][F][n_d1][ZW]
    float *post1;          // [2][F][n_d1][Z] (soft output only)
    int64_t n, words_m, words_k;
    int32_t n_frames, max_iter, et_start, soft, ZW, fmt;
    float clip, xmin;      // base-2 units
    float xmin_h;          // floor of a heavy output's exclusive sum: max(xmin, psi(clip)),
                           // so that psi of it needs no clip (psi decreases, psi(psi(y)) = y)
    float phi_lo, phi_hi;  // psi(clip) and psi(xmin): psi(clamp(y, xmin, clip)) =
                           // clamp(psi(y), phi_lo, phi_hi)
    float qstep, qinv;     // int8 message quantum and its inverse (base-2 units)
    int64_t msg_buf;       // layered: elements per message buffer; 0 for flooding
    int32_t layered;       // schedule: 0 flooding, 1 layered
    int32_t ngroups;       // layered: row groups per iteration
    int32_t pass;          // check-pass kind (kPassFlood, kPassTest, kPassGroup)
    int32_t lrow0, lrows;  // kPassGroup and the group's posterior update: its base rows
    int32_t cn_nt;         // check-block threads, 0 = chosen from Z (launch shape only)
    int32_t vn_vpt, vn_split;  // variable pass nodes per thread / part groups, 0 = chosen
    // Flooding with accumulated posteriors (accum = 1): the check pass adds
    // every new heavy message, as the integer acc_value() of its stored form,
    // into acc at the posterior's own offset (slot 2Z + shift + i, so a
    // column's node j collects at j and j + Z); post_kernel turns the sums
    // into L = Q + acc_inv (acc[j] + acc[j + Z]) and clears them. Integer
    // addition is exact and order-free: the sum, and so every posterior bit,
    // is the same whatever order the blocks and their reductions run in.
    int32_t *acc;          // [F][n_hcols][2Z]
    float acc_scale;       // FP32 / FP16 messages: fixed-point scale 2^k (int8: unused)
    float acc_inv;         // 2^-k, or the int8 quantum (the sum then counts quanta)
    int32_t accum;         // 1: accumulated posteriors; 0: separate summing variable pass
    // Bounded waits of the staged check pass: polls before giving up, and a
    // test switch (QCLDPC_TEST_STALL=1 in the environment) under which each
    // block expects 16 bytes more than it copies, so that its wait runs out
    // and the decode reports converged = -1 without any fault.
    uint32_t wait_polls;
    uint32_t stall_extra;  // bytes expected beyond the copies (0, or 16 under the switch)
};
// Kinds of check pass. kPassFlood: flooding iteration t (stop test of t-1
// when due, then the update). kPassTest: the stop test of iteration t-1
// alone, when due (layered). kPassGroup: the update of one row group for the
// iteration the control step just counted on (layered, no test).
enum CnPass { kPassFlood = 0, kPassTest = 1, kPassGroup = 2 };
static_assert(sizeof(Work) <= sizeof(((qcldpc_code *)nullptr)->last_work), "Work too large");

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
constexpr float kC = 1.528766394e+00f;  // 1 - log2(ln 2)
constexpr float kG0 = 5.776225403e-02f;
constexpr float kG1 = -1.618719543e-03f;
constexpr float kG2 = 5.430740566e-05f;
constexpr float kG3 = -1.724728236e-06f;
constexpr float kA0 = 2.885390043e+00f;
constexpr float kA1 = 9.617848396e-01f;
constexpr float kA2 = 5.777652860e-01f;
constexpr float kA3 = 3.984466195e-01f;
constexpr float kA4 = 4.293859601e-01f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kLog2e = 1.4426950408889634f;

// psi(y) = log2 coth(y ln2 / 2) = log2(e) Phi(y ln 2), for y > 0 (callers
// floor y); Phi(x) = -ln tanh(x/2) is Algorithm 1's check-node function.
//   small y: psi = 1 - log2(ln 2) - log2(y) + w G(w), w = y^2;
//   large y: psi = (2/ln 2) atanh(t) = t A(t^2), t = 2^-y.
// Both pieces are evaluated (no divergence) and combined with a max: each
// piece underestimates psi outside its own range (split at y = 1/ln 2), so
// the max picks the accurate piece; they differ only near the split, where
// both are accurate. Max relative error 2e-7 for y in [1e-6, 60] (ex2/lg2
// approximations included).
__device__ __forceinline__ float psi_f(float y) {
    const float w = y * y;
    const float g = fmaf(fmaf(fmaf(kG3, w, kG2), w, kG1), w, kG0);
    const float small = fmaf(w, g, kC - lg2_approx(y));
    const float t = ex2_approx(-y);
    const float v = t * t;
    const float a = fmaf(fmaf(fmaf(fmaf(kA4, v, kA3), v, kA2), v, kA1), v, kA0);
    return fmaxf(small, t * a);
}

// psi_f on two arguments at once with the packed FP32x2 multiply-adds of
// sm_100-class GPUs. Every packed operation rounds each lane exactly as the
// scalar fmaf / multiply of psi_f does, so psi2(y).x == psi_f(y.x) bit for
// bit (kC - lg2 is formed as fma(lg2, -1, kC), the same single rounding).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 psi2(float2 y) {
    const float2 w = __fmul2_rn(y, y);
    float2 g = __ffma2_rn(f2(kG3), w, f2(kG2));
    g = __ffma2_rn(g, w, f2(kG1));
    g = __ffma2_rn(g, w, f2(kG0));
    const float2 lc = __ffma2_rn(make_float2(lg2_approx(y.x), lg2_approx(y.y)), f2(-1.0f), f2(kC));
    const float2 small = __ffma2_rn(w, g, lc);
    const float2 t = make_float2(ex2_approx(-y.x), ex2_approx(-y.y));
    const float2 v = __fmul2_rn(t, t);
    float2 a = __ffma2_rn(f2(kA4), v, f2(kA3));
    a = __ffma2_rn(a, v, f2(kA2));
    a = __ffma2_rn(a, v, f2(kA1));
    a = __ffma2_rn(a, v, f2(kA0));
    const float2 ta = __fmul2_rn(t, a);
    return make_float2(fmaxf(small.x, ta.x), fmaxf(small.y, ta.y));
}

// max of three (sm_100-class three-input form)
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// psi(clamp(|y|, xmin, clip)) for a message difference y, as
// clamp(psi(|y|), lo, hi) with lo = psi(clip), hi = psi(xmin): psi decreases,
// so the clamp moves past it, and its lower bound merges with the max of the
// two pieces (|y| = 0 gives +inf before the clamp, never NaN).
__device__ __forceinline__ float psi_clamped(float y, float lo, float hi) {
    const float a = fabsf(y);
    const float w = a * a;
    const float g = fmaf(fmaf(fmaf(kG3, w, kG2), w, kG1), w, kG0);
    const float small = fmaf(w, g, kC - lg2_approx(a));
    const float t = ex2_approx(-a);
    const float v = t * t;
    const float p = fmaf(fmaf(fmaf(fmaf(kA4, v, kA3), v, kA2), v, kA1), v, kA0);
    return fminf(fmax3(small, t * p, lo), hi);
}
__device__ __forceinline__ float2 psi2_clamped(float2 y, float lo, float hi) {
    const float2 a = make_float2(fabsf(y.x), fabsf(y.y));
    const float2 w = __fmul2_rn(a, a);
    float2 g = __ffma2_rn(f2(kG3), w, f2(kG2));
    g = __ffma2_rn(g, w, f2(kG1));
    g = __ffma2_rn(g, w, f2(kG0));
    const float2 lc = __ffma2_rn(make_float2(lg2_approx(a.x), lg2_approx(a.y)), f2(-1.0f), f2(kC));
    const float2 small = __ffma2_rn(w, g, lc);
    const float2 t = make_float2(ex2_approx(-a.x), ex2_approx(-a.y));
    const float2 v = __fmul2_rn(t, t);
    float2 p = __ffma2_rn(f2(kA4), v, f2(kA3));
    p = __ffma2_rn(p, v, f2(kA2));
    p = __ffma2_rn(p, v, f2(kA1));
    p = __ffma2_rn(p, v, f2(kA0));
    const float2 tp = __fmul2_rn(t, p);
    return make_float2(fminf(fmax3(small.x, tp.x, lo), hi), fminf(fmax3(small.y, tp.y, lo), hi));
}

// Programmatic dependent launch: let the next kernel of the graph be
// scheduled now / wait until the previous kernel's results are visible.
// Without a programmatic edge both are no-ops.
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

constexpr uint32_t kSign = 0x80000000u;

// The off_a / off_b of a row's entries from its descriptor (three 16-byte
// read-only loads; the first 16 bytes, r / rp / nh / nd, the caller has).
__device__ __forceinline__ void load_offsets(const qc::RowDesc *dp, int (&oa)[qc::kDescEnts],
                                             int (&ob)[qc::kDescEnts]) {
    const int4 *q = reinterpret_cast<const int4 *>(dp);
    const int4 q1 = __ldg(q + 1), q2 = __ldg(q + 2), q3 = __ldg(q + 3);
    oa[0] = q1.x; oa[1] = q1.y; oa[2] = q1.z; oa[3] = q1.w; oa[4] = q2.x; oa[5] = q2.y;
    ob[0] = q2.z; ob[1] = q2.w; ob[2] = q3.x; ob[3] = q3.y; ob[4] = q3.z; ob[5] = q3.w;
}
__device__ __forceinline__ uint32_t fbits(float x) { return __float_as_uint(x); }

// Storage formats of the check-to-variable messages (computation is FP32):
// FP32, FP16 (round to nearest), or int8 codes q with m = q * qstep,
// |q| <= 127 (values beyond saturate; the quantum is one scale for the one
// stored edge type, heavy check-to-variable edges).
template <typename M>
struct Codec;
template <>
struct Codec<float> {
    __device__ static float dec(float v, const Work &) { return v; }
    __device__ static float enc(float v, const Work &) { return v; }
};
template <>
struct Codec<__half> {
    __device__ static float dec(__half v, const Work &) { return __half2float(v); }
    __device__ static __half enc(float v, const Work &) { return __float2half_rn(v); }
};
template <>
struct Codec<int8_t> {
    __device__ static float dec(int8_t v, const Work &W) { return (float)v * W.qstep; }
    __device__ static int8_t enc(float v, const Work &W) {
        return (int8_t)__float2int_rn(fminf(fmaxf(v * W.qinv, -127.0f), 127.0f));
    }
};

// The integer a stored message adds to its node's accumulator: the stored
// value in units of acc_inv (the int8 code itself; FP32 and FP16 values
// rounded to the fixed-point grid 2^-k).
__device__ __forceinline__ int acc_value(float v, const Work &W) { return __float2int_rn(v * W.acc_scale); }
__device__ __forceinline__ int acc_value(__half v, const Work &W) {
    return __float2int_rn(__half2float(v) * W.acc_scale);
}
__device__ __forceinline__ int acc_value(int8_t v, const Work &) { return (int)v; }

// Reduction into an accumulator (no return value: the add runs in L2).
__device__ __forceinline__ void red_add(int32_t *p, int v) {
    asm volatile("red.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

}  // namespace

namespace qc {
// Check-pass kernels of one storage format (FP32, FP16, int8) for codes whose
// rows have at most maxdeg circulants: the full-block kernel when nt ==
// kCnThreads, else the one that takes its width from the launch.
void *cn_kernel_f32(int maxdeg, int nt);
void *cn_kernel_f16(int maxdeg, int nt);
void *cn_kernel_i8(int maxdeg, int nt);
// Raise the dynamic shared-memory cap of that format's check-pass kernels.
void cn_smem_cap_f32(int cap);
void cn_smem_cap_f16(int cap);
void cn_smem_cap_i8(int cap);
}  // namespace qc
