/*
 * qcldpc — GB300 (sm_103a) decoder for quasi-cyclic multi-edge LDPC codes used
 * in long-distance CV-QKD reverse reconciliation (arXiv 1702.07740).
 *
 * C ABI. Every device buffer is owned by the caller; the library never
 * allocates device memory at run time (code tables and the no-alloc scratch
 * are static device arrays of the library), never frees or synchronises
 * caller memory, and
 * every call that takes a stream only enqueues work on it. Calls return 0 on success or a
 * negative QCLDPC_E_* status; qcldpc_last_error() then describes the failure
 * (thread-local text, valid until the next failing call on the same thread).
 * A frame that does not converge is not an error: its converged flag is 0.
 *
 * Bit packing: bit v of a frame is bit (v % 32) of 32-bit word v / 32
 * (LSB first). Frames of a batch are stored back to back; each packed frame
 * occupies ceil(bits / 32) words. Float arrays are frame-major, n floats per
 * frame.
 *
 * LLR sign convention: Q_v = ln P(C_v = 0) / P(C_v = 1) (Algorithm 1, Step 1).
 */
#ifndef QCLDPC_H
#define QCLDPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *qcldpc_stream_t; /* = cudaStream_t; NULL = legacy default stream */

enum {
    QCLDPC_OK = 0,
    QCLDPC_E_INVAL = -1,       /* bad argument (null pointer, size, range) */
    QCLDPC_E_SHIFT_RANGE = -2, /* circulant shift outside [0, Z) */
    QCLDPC_E_DUP_SHIFT = -3,   /* two circulants with equal shift in one base entry */
    QCLDPC_E_ALIGN = -4,       /* pointer not aligned as required */
    QCLDPC_E_NOMEM = -5,       /* host allocation failed, workspace too small, or
                                  the device table arena is full */
    QCLDPC_E_CUDA = -6,        /* a CUDA runtime call failed */
    QCLDPC_E_TIMEOUT = -7,     /* reserved: a bounded device wait gave up */
    QCLDPC_E_UNSUPPORTED = -8  /* code exceeds a compile-time table limit */
};

/* Table limits (checked by qcldpc_create_code). The tables of
 * all live codes share a 64 MiB static device arena inside the library (about
 * 60 bytes per circulant plus 128 bytes per base row: 0.4 MB for a
 * 1568 x 1600 base matrix); a code takes its block on the first call that
 * launches work and returns it in qcldpc_destroy_code. */
#define QCLDPC_MAX_BASE_ROWS 16384
#define QCLDPC_MAX_BASE_COLS 32768
#define QCLDPC_MAX_CIRCULANTS 65536
#define QCLDPC_MAX_HEAVY_COLS 4096
#define QCLDPC_MAX_ROW_DEGREE 16
#define QCLDPC_MAX_Z (1 << 24)

typedef struct qcldpc_code qcldpc_code; /* opaque, library-owned */

/*
 * Build a QC code from its base-matrix circulant list (QC expansion, Sec.
 * III-C). Each circulant is a Z x Z permutation block given by its shift
 * s in [0, Z): row i of the block has its single one in column (i + s) mod Z.
 * Circulant h = (circ_row[h], circ_col[h], circ_shift[h]) puts, for every
 * i in [0, Z), a one at (check circ_row*Z + i, variable circ_col*Z +
 * (i + circ_shift) mod Z). Several circulants may share a base entry if their
 * shifts differ (equal shifts would cancel over GF(2): QCLDPC_E_DUP_SHIFT).
 *
 *   mb, nb      base rows / columns; n = nb*Z bits, m = mb*Z checks, k = n-m
 *   Z           expansion factor (lifting size), 1 <= Z <= QCLDPC_MAX_Z
 *   n_circ      number of circulants (1..QCLDPC_MAX_CIRCULANTS)
 *   circ_*      HOST arrays of n_circ int32; copied, caller keeps ownership
 *   out         receives the new handle (set to NULL on failure)
 *
 * Columns holding exactly one circulant are degree-1 ("diagonal") columns:
 * their variable nodes never need per-iteration messages (the unshifted
 * diagonal of Sec. III-C). All other columns are heavy columns. Host-only:
 * no device memory is allocated here; the tables are copied into the
 * library's static device table arena on the first call that launches work
 * with the code, and their block is returned by qcldpc_destroy_code. The handle
 * remembers the CUDA device current at creation (decoding on another device
 * fails with QCLDPC_E_INVAL). Errors: QCLDPC_E_INVAL, _SHIFT_RANGE,
 * _DUP_SHIFT, _UNSUPPORTED, _NOMEM.
 */
int qcldpc_create_code(int mb, int nb, int Z, int n_circ,
                       const int32_t *circ_row, const int32_t *circ_col,
                       const int32_t *circ_shift, qcldpc_code **out);

/* Release a handle (NULL is ignored). Work already enqueued that uses it
 * must have completed. */
void qcldpc_destroy_code(qcldpc_code *code);

/* Sizes of a code: n bits, m checks, k = n - m key bits, n_edges ones in H.
 * Any output pointer may be NULL. Errors: QCLDPC_E_INVAL. */
int qcldpc_code_info(const qcldpc_code *code, int64_t *n, int64_t *m,
                     int64_t *k, int64_t *n_edges);

/*
 * Syndrome s = H x (mod 2) of n_frames frames (the Slepian-Wolf form of
 * reverse reconciliation, Sec. II-C: Bob publishes s for his bits).
 *   bits_dev   DEVICE uint32[n_frames * ceil(n/32)], packed frames
 *   syn_dev    DEVICE uint32[n_frames * ceil(m/32)], packed output
 * Bit-exact. Errors: QCLDPC_E_INVAL, _ALIGN (4-byte), _CUDA (launch).
 */
int qcldpc_syndrome(const qcldpc_code *code, const uint32_t *bits_dev,
                    uint32_t *syn_dev, int n_frames, qcldpc_stream_t stream);

/*
 * Bob's side of 8-dimensional reconciliation (Sec. II-C): per block b of
 * eight positions, U_j = (-1)^{C_{8b+j}} and M = U Y, the octonion product
 * (Cayley-Dickson doubling, (p,q)(r,s) = (pr - conj(s) q, sp + q conj(r))).
 *   y_dev     DEVICE float[n], Bob's normalised Gaussian samples
 *   bits_dev  DEVICE uint32[ceil(n/32)], packed bits C
 *   n         total length, n % 8 == 0 (frames may be concatenated if each
 *             frame length is a multiple of 8 and of 32)
 *   m_dev     DEVICE float[n], the public message M
 * FP32 arithmetic. Errors: QCLDPC_E_INVAL, _ALIGN (16-byte floats), _CUDA.
 */
int qcldpc_bob_message_8d(const float *y_dev, const uint32_t *bits_dev,
                          int64_t n, float *m_dev, qcldpc_stream_t stream);

/*
 * Alice's channel LLRs for 8-dimensional reconciliation (Sec. II-C and
 * Step 1 of Algorithm 1): R = M X^{-1} = (M conj(X)) / |X|^2 and the virtual
 * BIAWGN noise variance sigma_N^2 = 8 sigma_Z^2 / |X|^2 with sigma_Z^2 =
 * 1/snr, so Q = 2 R / sigma_N^2 = (M conj(X)) * snr / 4.
 *   x_dev, m_dev   DEVICE float[n] (Alice's X, Bob's message M)
 *   n              n % 8 == 0
 *   snr            > 0
 *   llr_dev        DEVICE float[n] output Q
 * FP32 arithmetic. Errors: QCLDPC_E_INVAL, _ALIGN (16-byte), _CUDA.
 */
int qcldpc_llr_8d(const float *x_dev, const float *m_dev, int64_t n, float snr,
                  float *llr_dev, qcldpc_stream_t stream);

/*
 * The d-dimensional maps for d in {1, 2, 4, 8} (Sec. II-C, multi-dimensional
 * reconciliation): groups of d consecutive positions share one virtual
 * BIAWGN channel. Bob: M = U Y with U_j = (-1)^{C_j} (reals, complex
 * numbers, quaternions, octonions by Cayley-Dickson doubling). Alice:
 * R = M conj(X) / |X|^2, sigma_N^2 = d sigma_Z^2 / |X|^2, Q = 2R / sigma_N^2
 * = (M conj(X)) 2 snr / d; for d = 1 this is Step 1 of Algorithm 1 with
 * sigma_N^2 = sigma_Z^2 / X^2. d = 8 calls the 8-D entry points above.
 * Arrays as for the 8-D calls (n % d == 0); 4-byte alignment suffices for
 * d < 8. Errors: QCLDPC_E_INVAL, _ALIGN, _CUDA.
 */
int qcldpc_bob_message(int d, const float *y_dev, const uint32_t *bits_dev, int64_t n,
                       float *m_dev, qcldpc_stream_t stream);
int qcldpc_llr(int d, const float *x_dev, const float *m_dev, int64_t n, float snr,
               float *llr_dev, qcldpc_stream_t stream);

/* Decoder options. Initialise with qcldpc_params_init. */
typedef struct qcldpc_params {
    float clip;          /* every edge message is clipped to [-clip, clip];
                            <= 0 disables clipping. Default 15 */
    float phi_floor;     /* every Phi argument is floored at this value
                            (Phi(x) = -ln tanh(x/2)). Default 1e-6 */
    int32_t et_start;    /* the stop test H C = s runs after iteration t when
                            t >= et_start, and always after the last
                            iteration (delayed early termination, Sec. IV-A).
                            Default 1 */
    int32_t schedule;    /* 0 = flooding (Algorithm 1, default); 1 = layered:
                            the base rows are split into `layers` contiguous
                            groups (row r in group floor(r * layers / mb)),
                            visited in order within an iteration; a group's
                            messages are computed from the state at the
                            group's start and its posteriors updated before
                            the next group (an extension of the paper's
                            flooding decoder). Pools accept both */
    int32_t msg_format;  /* storage of the check-to-variable messages, all
                            arithmetic FP32: 0 = FP32 (default), 1 = FP16
                            (round to nearest), 2 = int8 codes q with
                            m = q * msg_step, |q| <= 127 (saturating) */
    int32_t soft_output; /* 1: reserve workspace for qcldpc_decode_soft */
    int32_t launch_mode; /* 0: the iteration loop runs inside one CUDA graph
                            (a conditional WHILE node; no host work per
                            iteration). 1: the host enqueues max_iter + 1
                            iteration passes as ordinary kernel launches on
                            the stream (passes after every frame stopped exit
                            at once); same results, meant for profilers that
                            cannot look inside conditional graphs. Default 0 */
    float msg_step;      /* int8 quantum in natural-LLR units; 0 (default)
                            means clip / 127. Ignored for other formats */
    int32_t layers;      /* layered schedule: number of row groups, 1..mb;
                            0 (default) = one group per base row. Ignored by
                            flooding. layers = 1 computes what flooding does */
    /* Launch shapes; 0 (default) lets the library choose. None of them
       changes a result bit (qcldpc_autotune_shapes picks them by time). */
    int32_t cn_threads;  /* threads per check-pass block: a multiple of 32,
                            32..256; a block evaluates 4 checks per thread of
                            one base row */
    int32_t vn_nodes;    /* variable pass: heavy nodes per thread, 1..3 */
    int32_t vn_split;    /* variable pass: 1 = a thread adds both partial sums
                            of its nodes, 2 = two thread groups, one per
                            partial sum (added in the same order) */
    int32_t vn_pass;     /* how flooding forms the posteriors L_v = Q_v +
                            sum_c m_cv (Algorithm 1, Step 3). 0 (default):
                            the check pass adds every new heavy message,
                            rounded to a fixed-point grid (2^-20 for the
                            rate-0.02 codes; the int8 quantum for int8
                            storage), into exact integer per-node sums, so
                            one iteration reads and writes each message once;
                            the sums do not depend on the order of the adds.
                            1: a separate variable pass re-reads every message
                            and adds them in FP32 (vn_nodes and vn_split
                            apply). Layered decoding ignores it */
    int32_t frame_groups; /* graph launches (launch_mode 0) of decodes
                            without soft output: the frames are split into
                            this many groups of consecutive frames, each
                            iterating in its own chain of passes inside the
                            one decode graph. Flooding: a group's short
                            per-iteration steps (stop test, posterior pass)
                            run at high priority while other groups' check
                            passes fill the GPU; layered: the groups' small
                            per-row-group passes run side by side. 0
                            (default): 2 groups for flooding when n_frames
                            >= 2, one chain for layered decoding (its many
                            small launches gain less than they cost); 1: one
                            chain; at most QCLDPC_MULTI_MAX_CODES (and at
                            most n_frames). No result bit depends on it */
} qcldpc_params;

void qcldpc_params_init(qcldpc_params *p);

/* Bytes of device workspace qcldpc_decode needs for n_frames frames
 * (p may be NULL for defaults). Returns 0 on invalid arguments. */
size_t qcldpc_decode_workspace(const qcldpc_code *code, int n_frames,
                               const qcldpc_params *p);

/*
 * Syndrome-form sum-product decoding (Algorithm 1, flooding schedule) of
 * n_frames independent frames, the whole loop on the device.
 *
 * For every frame: L_vc^(0) = Q_v. Iteration t: check nodes send
 *   m_cv = (-1)^{s_c} prod_{v' != v} sgn(L_v'c) Phi(sum_{v' != v} Phi(|L_v'c|)),
 * variable nodes form L_v = Q_v + sum_c m_cv and L_vc = L_v - m_cv, and the
 * hard decision is C_v = 1 iff L_v < 0 (sgn(0) = +1). After iteration t the
 * stop test H C = s runs when t >= et_start or t = max_iter; a frame that
 * passes stops there. Messages are clipped to [-clip, clip], Phi arguments
 * floored at phi_floor, all arithmetic FP32.
 *
 *   llr_dev        DEVICE float[n_frames * n], channel LLRs Q (16-byte aligned)
 *   syn_dev        DEVICE uint32[n_frames * ceil(m/32)], packed syndromes s
 *   max_iter       >= 0 (0: the channel decisions are tested and returned)
 *   p              options, NULL for defaults
 *   key_bits_dev   DEVICE uint32[n_frames * ceil(k/32)]: decisions C_v for
 *                  v < k (the key S-hat, Step 5: parity bits discarded)
 *   converged_dev  DEVICE int32[n_frames]: 1 if H C = s at the stop
 *   iters_dev      DEVICE int32[n_frames]: iteration the frame stopped at
 *   workspace_dev  DEVICE scratch of at least qcldpc_decode_workspace()
 *                  bytes, 256-byte aligned; contents are overwritten
 * Enqueues on `stream`; returns without waiting. Concurrent calls on one code
 * handle are serialised on the host. By default (p->frame_groups = 0) a
 * graph-launched flooding decode of n_frames >= 2 runs its frames as two
 * groups of consecutive frames in side-by-side chains of one graph (the
 * instantiated graphs of recent argument sets are kept); the workspace
 * size accounts for it. Errors: QCLDPC_E_INVAL, _ALIGN, _NOMEM (workspace
 * too small), _CUDA.
 */
int qcldpc_decode(const qcldpc_code *code, const float *llr_dev,
                  const uint32_t *syn_dev, int n_frames, int max_iter,
                  const qcldpc_params *p, uint32_t *key_bits_dev,
                  int32_t *converged_dev, int32_t *iters_dev,
                  void *workspace_dev, size_t workspace_bytes,
                  qcldpc_stream_t stream);

/*
 * As qcldpc_decode, and also writes the posterior LLR L_v of every bit at
 * the stopping iteration (Algorithm 1, Step 3) to posterior_dev
 * (DEVICE float[n_frames * n]). Requires p != NULL with p->soft_output = 1
 * for both this call and qcldpc_decode_workspace.
 */
int qcldpc_decode_soft(const qcldpc_code *code, const float *llr_dev,
                       const uint32_t *syn_dev, int n_frames, int max_iter,
                       const qcldpc_params *p, uint32_t *key_bits_dev,
                       int32_t *converged_dev, int32_t *iters_dev,
                       float *posterior_dev, void *workspace_dev,
                       size_t workspace_bytes, qcldpc_stream_t stream);

/*
 * Batched decoding of the frames of several codes in one graph launch (frame
 * batching across codes; the paper decodes one frame of one code per GPU).
 * Code c's n_frames[c] frames run the rule of qcldpc_decode (flooding,
 * Algorithm 1) with their own stop test; each code's frames iterate in
 * their own device-side loop, the loops of all codes side by side in the
 * one graph (each ends when its own frames have stopped). The
 * results (key bits, flags, iterations) are the ones one qcldpc_decode call
 * per code with the same frames and options returns.
 *
 *   n_codes         1..QCLDPC_MULTI_MAX_CODES
 *   codes           HOST array of n_codes code handles (distinct or not)
 *   llr_dev, syn_dev, key_bits_dev, converged_dev, iters_dev
 *                   HOST arrays of n_codes DEVICE pointers, each laid out
 *                   as for qcldpc_decode with that code and frame count
 *                   (LLRs 16-byte aligned); entries of codes with no frame
 *                   may be NULL
 *   n_frames        HOST int[n_codes], each 0..65535
 *   p               options as for qcldpc_decode; schedule must be 0
 *                   (flooding) and soft_output 0
 *   workspace_dev   DEVICE scratch of qcldpc_decode_multi_workspace() bytes,
 *                   256-byte aligned
 * Enqueues on `stream`; the instantiated graph is cached per argument set.
 * Errors: QCLDPC_E_INVAL, _ALIGN, _NOMEM (workspace too small), _CUDA.
 */
#define QCLDPC_MULTI_MAX_CODES 16
size_t qcldpc_decode_multi_workspace(int n_codes, const qcldpc_code *const *codes,
                                     const int *n_frames, const qcldpc_params *p);
int qcldpc_decode_multi(int n_codes, const qcldpc_code *const *codes,
                        const float *const *llr_dev, const uint32_t *const *syn_dev,
                        const int *n_frames, int max_iter, const qcldpc_params *p,
                        uint32_t *const *key_bits_dev, int32_t *const *converged_dev,
                        int32_t *const *iters_dev, void *workspace_dev,
                        size_t workspace_bytes, qcldpc_stream_t stream);

/*
 * Pools: continuous batching of frames of one code (serving). A pool is a
 * fixed set of n_slots frame slots with all decoder state in one caller-owned
 * workspace (qcldpc_pool_workspace bytes, 256-byte aligned). Frames are loaded
 * into free slots at any time; each step runs n_passes iteration passes over
 * all running slots, every frame at its own iteration and with its own stop
 * test (the rule of qcldpc_decode, max_iter and options fixed per pool);
 * frames that stopped are collected, which frees their slots. A frame's
 * result does not depend on the other frames sharing the passes.
 *
 *   qcldpc_pool_create   max_iter >= 0; p as for qcldpc_decode (soft_output
 *                        must be 0); all slots start free. Enqueues a reset on
 *                        `stream`. Host handle, library-owned.
 *   qcldpc_pool_state    device pointer to int32[n_slots] slot states:
 *                        0 free, 1 running, 2 stopped (result ready)
 *   qcldpc_pool_load     n frames: slots_dev int32[n] (free or stopped slots,
 *                        distinct), llr_dev float[n * code n] (natural LLRs),
 *                        syn_dev uint32[n * ceil(m/32)]; inputs are copied, so
 *                        the caller may reuse them once the load has run
 *   qcldpc_pool_step     n_passes >= 1 passes; the graph is cached per count
 *   qcldpc_pools_step    one graph stepping several pools concurrently (e.g.
 *                        codes of different rates), cached per pool list
 *   qcldpc_pool_collect  for n stopped slots: key bits uint32[n * ceil(k/32)],
 *                        converged int32[n] (1, 0, or -1 if a device wait
 *                        timed out), iterations int32[n]; frees the slots
 * All calls only enqueue work on `stream`. Calls on one pool are serialised
 * on the host; GPU work of one pool must stay on one stream (or be ordered by
 * the caller). Errors: QCLDPC_E_INVAL, _ALIGN, _NOMEM, _CUDA.
 */
typedef struct qcldpc_pool qcldpc_pool;
size_t qcldpc_pool_workspace(const qcldpc_code *code, int n_slots, const qcldpc_params *p);
int qcldpc_pool_create(const qcldpc_code *code, int n_slots, int max_iter, const qcldpc_params *p,
                       void *workspace_dev, size_t workspace_bytes, qcldpc_stream_t stream,
                       qcldpc_pool **out);
void qcldpc_pool_destroy(qcldpc_pool *pool);
int qcldpc_pool_state(const qcldpc_pool *pool, const int32_t **state_dev);
int qcldpc_pool_load(qcldpc_pool *pool, int n, const int32_t *slots_dev, const float *llr_dev,
                     const uint32_t *syn_dev, qcldpc_stream_t stream);
int qcldpc_pool_step(qcldpc_pool *pool, int n_passes, qcldpc_stream_t stream);
int qcldpc_pools_step(int n_pools, qcldpc_pool *const *pools, int n_passes,
                      qcldpc_stream_t stream);
int qcldpc_pool_collect(qcldpc_pool *pool, int n, const int32_t *slots_dev,
                        uint32_t *key_bits_dev, int32_t *converged_dev, int32_t *iters_dev,
                        qcldpc_stream_t stream);

/*
 * Schedule autotuner; an extension (the paper fixes flooding). Decodes the
 * caller's sample batch once per candidate schedule: flooding, then layered
 * with 2, 7 and min(mb, 64) row groups (those in [1, mb], without repeats). Every
 * other option comes from p. Each candidate runs once untimed (its graph is
 * instantiated), then `reps` times between CUDA events on `stream`; the
 * fastest candidate's options are written to *best. What is timed is the
 * time to decode the sample, including the iterations each schedule needs,
 * so the sample should look like the frames to come (code, SNR, batch size).
 *   llr_dev .. iters_dev   as qcldpc_decode; the outputs of the last sample
 *                          decode are left there
 *   workspace_dev          at least qcldpc_decode_workspace(code, n_frames,
 *                          p with schedule = 1) bytes (the larger layout)
 *   reps                   >= 1 timed decodes per candidate
 *   best                   HOST qcldpc_params, written on success
 *   times_ms               optional HOST float[4]: mean decode time per
 *                          candidate (flooding, 2, 7, min(mb, 64) groups), NAN where
 *                          a candidate was not tried
 * Blocks the calling thread until the timings are known. Errors as
 * qcldpc_decode.
 */
int qcldpc_autotune(const qcldpc_code *code, const float *llr_dev, const uint32_t *syn_dev,
                    int n_frames, int max_iter, const qcldpc_params *p,
                    uint32_t *key_bits_dev, int32_t *converged_dev, int32_t *iters_dev,
                    void *workspace_dev, size_t workspace_bytes, int reps,
                    qcldpc_params *best, float *times_ms, qcldpc_stream_t stream);

/*
 * Launch-shape autotuner; the paper has no counterpart. On the workspace of
 * a previous flooding qcldpc_decode / qcldpc_decode_soft call with the same
 * code and n_frames (read as qcldpc_time_passes reads it), replays the
 * check-node pass with
 * blocks of 32, 64, ..., 256 threads, and the separate variable-node pass
 * (the one vn_pass = 1 selects) with (nodes per thread, vn_split) = (1,1),
 * (2,1), (3,1), (1,2), (2,2), (3,2), each `reps` times after one warm-up
 * launch (CUDA events on `stream`). The accumulated-posterior pass of
 * vn_pass = 0 has one shape and is not tuned.
 *   p        options the shapes are tuned for (NULL = defaults)
 *   best     out: *p with cn_threads, vn_nodes and vn_split set to the
 *            fastest candidates
 *   cn_ms    out (may be NULL): 8 mean check-pass times, ms, in that order
 *   vn_ms    out (may be NULL): 6 mean variable-pass times, ms
 * Every shape computes the same bits. Overwrites the decoder state in the
 * workspace as qcldpc_time_passes does; blocks the calling thread.
 * Errors: QCLDPC_E_INVAL (no matching previous flooding decode), _NOMEM,
 * _CUDA.
 */
int qcldpc_autotune_shapes(const qcldpc_code *code, int n_frames, void *workspace_dev,
                           size_t workspace_bytes, int reps, const qcldpc_params *p,
                           qcldpc_params *best, float *cn_ms, float *vn_ms, qcldpc_stream_t stream);

/*
 * Measurement helper; the paper has no counterpart. Replays the check-node
 * pass and then the variable-node pass of the decoder (with vn_pass = 0 the
 * light pass that turns the accumulated sums into posteriors) `reps` times
 * each, with
 * the launch configuration qcldpc_decode uses for the whole batch, on the
 * workspace of a previous qcldpc_decode / qcldpc_decode_soft call with the
 * same code and n_frames, and returns each pass's mean duration in
 * milliseconds (CUDA events on `stream`). The replays run as iteration 2 of
 * a decode with every frame active, so each moves a full iteration's data.
 * After a decode that ran its frames in groups (frame_groups), the replays
 * read the workspace through the whole batch's layout: the same kernels,
 * launch shapes and bytes, on values that are not that decode's state.
 * Overwrites the decoder state in the workspace (the last decode's outputs
 * are untouched). Blocks the calling thread until the replays finish.
 * Errors: QCLDPC_E_INVAL (no matching previous decode), _NOMEM, _CUDA.
 */
int qcldpc_time_passes(const qcldpc_code *code, int n_frames, void *workspace_dev,
                       size_t workspace_bytes, int reps, float *cn_ms, float *vn_ms,
                       qcldpc_stream_t stream);

/*
 * Decoding for callers that cannot allocate device memory; the paper has no
 * counterpart. Some callers have no way to allocate device memory: code
 * embedded in a host framework that owns the device allocator and does not
 * expose it, or a process whose device memory is reserved once at start-up
 * and may not grow. This entry point computes exactly what qcldpc_decode
 * computes (same kernels, passes enqueued one by one on `stream`, no graph
 * objects), but keeps its scratch in a static 16 MiB device array inside the
 * library instead of a caller workspace. Every GPU that loads the library
 * holds that array until the process exits. The caller still passes the
 * inputs and outputs described at qcldpc_decode; the array is never exposed.
 *
 * Limit: the code's workspace for n_frames (qcldpc_decode_workspace with
 * default options) must fit in 16 MiB, e.g. one frame of the rate-0.02,
 * n = 10^6 code; larger requests return QCLDPC_E_UNSUPPORTED and a message
 * naming both sizes. p->soft_output and p->launch_mode are ignored.
 *
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * All calls on a device share the one array and every call re-initialises
 * all decoder state it reads, so consecutive calls are independent; calls
 * whose work overlaps on the GPU (e.g. on two streams at once) race on the
 * array and must be serialised by the caller. Allocates nothing.
 * Errors: QCLDPC_E_INVAL, _ALIGN, _UNSUPPORTED, _CUDA.
 */
int qcldpc_decode_noalloc(const qcldpc_code *code, const float *llr_dev,
                          const uint32_t *syn_dev, int n_frames, int max_iter,
                          const qcldpc_params *p, uint32_t *key_bits_dev,
                          int32_t *converged_dev, int32_t *iters_dev,
                          qcldpc_stream_t stream);

/* Description of the last failure on this thread ("" if none). */
const char *qcldpc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QCLDPC_H */
