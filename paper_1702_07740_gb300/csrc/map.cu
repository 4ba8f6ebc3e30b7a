// Syndrome and 8-dimensional reconciliation kernels.
//
// * qcldpc_syndrome: s = H x over GF(2) for the QC expansion of Sec. III-C,
//   one thread per check node, results packed with a warp ballot.
// * qcldpc_bob_message_8d / qcldpc_llr_8d: Sec. II-C. Bob sends M = U Y with
//   U_j = (-1)^{C_j}; Alice divides, R = M X^{-1} = M conj(X) / |X|^2, and
//   with sigma_N^2 = 8 sigma_Z^2 / |X|^2 the channel LLR of Step 1 of
//   Algorithm 1 becomes Q = 2R / sigma_N^2 = (M conj(X)) snr / 4: |X|^2
//   cancels, so the kernel needs one octonion product per block of eight.
//
// Octonions are pairs of quaternions with Cayley-Dickson doubling
// (p,q)(r,s) = (p r - conj(s) q, s p + q conj(r)); quaternions multiply by
// Hamilton's rule. One thread owns one block of eight floats, loaded and
// stored as two 16-byte vectors; the work is a pure stream (12 bytes per bit
// for the LLR map), bounded by HBM bandwidth.
#include "qcldpc_internal.cuh"

namespace {

struct Quat {
    float w, x, y, z;
};

__device__ __forceinline__ Quat qmul(Quat a, Quat b) {
    Quat r;
    r.w = a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z;
    r.x = a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y;
    r.y = a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x;
    r.z = a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w;
    return r;
}

__device__ __forceinline__ Quat qconj(Quat a) { return Quat{a.w, -a.x, -a.y, -a.z}; }
__device__ __forceinline__ Quat qadd(Quat a, Quat b) {
    return Quat{a.w + b.w, a.x + b.x, a.y + b.y, a.z + b.z};
}
__device__ __forceinline__ Quat qsub(Quat a, Quat b) {
    return Quat{a.w - b.w, a.x - b.x, a.y - b.y, a.z - b.z};
}
__device__ __forceinline__ Quat q4(float4 v) { return Quat{v.x, v.y, v.z, v.w}; }
__device__ __forceinline__ float4 f4(Quat q) { return make_float4(q.w, q.x, q.y, q.z); }

// (p, q)(r, s) = (p r - conj(s) q, s p + q conj(r))
__device__ __forceinline__ void omul(Quat p, Quat q, Quat r, Quat s, Quat &lo, Quat &hi) {
    lo = qsub(qmul(p, r), qmul(qconj(s), q));
    hi = qadd(qmul(s, p), qmul(q, qconj(r)));
}

__global__ void __launch_bounds__(256) syndrome_kernel(const __grid_constant__ qc::Table T,
                                                       const uint32_t *__restrict__ bits,
                                                       uint32_t *__restrict__ syn,
                                                       int64_t words_n, int64_t words_m) {
    const int f = blockIdx.y;
    const int64_t m = (int64_t)T.mb * T.Z;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t *fb = bits + (int64_t)f * words_n;
    uint32_t par = 0;
    if (c < m) {
        const int r = (int)(c / T.Z);
        const int i = (int)(c - (int64_t)r * T.Z);
        for (int k = T.row_ptr[r]; k < T.row_ptr[r + 1]; k++) {
            const qc::RowEnt e = T.rows[k];
            int j = i + e.shift;
            if (j >= T.Z) j -= T.Z;
            const int64_t v = (int64_t)e.col * T.Z + j;
            par ^= (__ldg(fb + (v >> 5)) >> (v & 31)) & 1u;
        }
    }
    const uint32_t word = __ballot_sync(0xffffffffu, par);
    if ((threadIdx.x & 31) == 0 && c < m) syn[(int64_t)f * words_m + (c >> 5)] = word;
}

__global__ void __launch_bounds__(256) bob8_kernel(const float4 *__restrict__ y,
                                                   const uint32_t *__restrict__ bits,
                                                   float4 *__restrict__ out, int64_t n_blocks) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t byte = (__ldg(bits + (b >> 2)) >> (8 * (b & 3))) & 0xffu;
        float u[8];
#pragma unroll
        for (int j = 0; j < 8; j++) u[j] = ((byte >> j) & 1u) ? -1.0f : 1.0f;
        const Quat up{u[0], u[1], u[2], u[3]}, uq{u[4], u[5], u[6], u[7]};
        const Quat yr = q4(__ldg(y + 2 * b)), ys = q4(__ldg(y + 2 * b + 1));
        Quat lo, hi;
        omul(up, uq, yr, ys, lo, hi);
        out[2 * b] = f4(lo);
        out[2 * b + 1] = f4(hi);
    }
}

__global__ void __launch_bounds__(256) llr8_kernel(const float4 *__restrict__ x,
                                                   const float4 *__restrict__ m,
                                                   float4 *__restrict__ llr, float scale,
                                                   int64_t n_blocks) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        const Quat mp = q4(__ldg(m + 2 * b)), mq = q4(__ldg(m + 2 * b + 1));
        const Quat xp = q4(__ldg(x + 2 * b)), xq = q4(__ldg(x + 2 * b + 1));
        // conj of the octonion (xp, xq) is (conj xp, -xq)
        const Quat cp = qconj(xp);
        const Quat cq{-xq.w, -xq.x, -xq.y, -xq.z};
        Quat lo, hi;
        omul(mp, mq, cp, cq, lo, hi);
        llr[2 * b] = make_float4(lo.w * scale, lo.x * scale, lo.y * scale, lo.z * scale);
        llr[2 * b + 1] = make_float4(hi.w * scale, hi.x * scale, hi.y * scale, hi.z * scale);
    }
}

// d in {1, 2, 4}: reals, complex numbers (Cayley-Dickson doubling of the
// reals) and quaternions (Hamilton's rule), one thread per block of d.
// Bob: M = U Y. Alice: Q = (M conj(X)) * 2 snr / d (sigma_N^2 = d sigma_Z^2 /
// |X|^2, so |X|^2 cancels as in the 8-D map).
template <int D>
__global__ void __launch_bounds__(256) bob_d_kernel(const float *__restrict__ y,
                                                    const uint32_t *__restrict__ bits,
                                                    float *__restrict__ out, int64_t n_blocks) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v0 = b * D;
        float u[D], yy[D];
#pragma unroll
        for (int j = 0; j < D; j++) {
            const int64_t v = v0 + j;
            u[j] = ((__ldg(bits + (v >> 5)) >> (v & 31)) & 1u) ? -1.0f : 1.0f;
            yy[j] = __ldg(y + v);
        }
        if constexpr (D == 1) {
            out[v0] = u[0] * yy[0];
        } else if constexpr (D == 2) {  // (a + ib)(c + id)
            out[v0] = u[0] * yy[0] - u[1] * yy[1];
            out[v0 + 1] = u[0] * yy[1] + u[1] * yy[0];
        } else {
            const Quat r = qmul(Quat{u[0], u[1], u[2], u[3]}, Quat{yy[0], yy[1], yy[2], yy[3]});
            out[v0] = r.w;
            out[v0 + 1] = r.x;
            out[v0 + 2] = r.y;
            out[v0 + 3] = r.z;
        }
    }
}

template <int D>
__global__ void __launch_bounds__(256) llr_d_kernel(const float *__restrict__ x,
                                                    const float *__restrict__ m,
                                                    float *__restrict__ llr, float scale,
                                                    int64_t n_blocks) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v0 = b * D;
        if constexpr (D == 1) {
            llr[v0] = __ldg(m + v0) * __ldg(x + v0) * scale;
        } else if constexpr (D == 2) {  // M conj(X) = (a + ib)(c - id)
            const float a = __ldg(m + v0), bb = __ldg(m + v0 + 1);
            const float c = __ldg(x + v0), d = __ldg(x + v0 + 1);
            llr[v0] = (a * c + bb * d) * scale;
            llr[v0 + 1] = (bb * c - a * d) * scale;
        } else {
            const Quat mq{__ldg(m + v0), __ldg(m + v0 + 1), __ldg(m + v0 + 2), __ldg(m + v0 + 3)};
            const Quat xq{__ldg(x + v0), __ldg(x + v0 + 1), __ldg(x + v0 + 2), __ldg(x + v0 + 3)};
            const Quat r = qmul(mq, qconj(xq));
            llr[v0] = r.w * scale;
            llr[v0 + 1] = r.x * scale;
            llr[v0 + 2] = r.y * scale;
            llr[v0 + 3] = r.z * scale;
        }
    }
}

int stream_grid(int64_t n_blocks) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    int64_t g = (n_blocks + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;  // 8 resident blocks of 256 per SM
    if (g > cap) g = cap;
    return (int)(g > 0 ? g : 1);
}

}  // namespace

extern "C" int qcldpc_syndrome(const qcldpc_code *code, const uint32_t *bits_dev,
                               uint32_t *syn_dev, int n_frames, qcldpc_stream_t stream) {
    using namespace qc;
    if (!code || !bits_dev || !syn_dev || n_frames < 0)
        return fail(QCLDPC_E_INVAL, "syndrome: NULL argument or negative frame count");
    if (!aligned(bits_dev, 4) || !aligned(syn_dev, 4))
        return fail(QCLDPC_E_ALIGN, "syndrome: buffers must be 4-byte aligned");
    if (n_frames > 65535) return fail(QCLDPC_E_INVAL, "syndrome: more than 65535 frames");
    if (n_frames == 0) return QCLDPC_OK;
    if (int st = upload_tables(const_cast<qcldpc_code *>(code))) return st;
    const int64_t words_n = (code->n + 31) / 32, words_m = (code->m + 31) / 32;
    dim3 grid((unsigned)((code->m + 255) / 256), (unsigned)n_frames);
    syndrome_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(code->tab, bits_dev, syn_dev,
                                                           words_n, words_m);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "syndrome: launch");
    return QCLDPC_OK;
}

extern "C" int qcldpc_bob_message_8d(const float *y_dev, const uint32_t *bits_dev, int64_t n,
                                     float *m_dev, qcldpc_stream_t stream) {
    using namespace qc;
    if (!y_dev || !bits_dev || !m_dev || n < 0 || n % 8 != 0)
        return fail(QCLDPC_E_INVAL, "bob_message_8d: NULL argument or n not a multiple of 8");
    if (!aligned(y_dev, 16) || !aligned(m_dev, 16) || !aligned(bits_dev, 4))
        return fail(QCLDPC_E_ALIGN, "bob_message_8d: floats must be 16-byte aligned");
    if (n == 0) return QCLDPC_OK;
    const int64_t nb = n / 8;
    bob8_kernel<<<stream_grid(nb), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4 *>(y_dev), bits_dev, reinterpret_cast<float4 *>(m_dev), nb);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "bob_message_8d: launch");
    return QCLDPC_OK;
}

extern "C" int qcldpc_llr_8d(const float *x_dev, const float *m_dev, int64_t n, float snr,
                             float *llr_dev, qcldpc_stream_t stream) {
    using namespace qc;
    if (!x_dev || !m_dev || !llr_dev || n < 0 || n % 8 != 0 || !(snr > 0.0f))
        return fail(QCLDPC_E_INVAL, "llr_8d: NULL argument, n not a multiple of 8, or snr <= 0");
    if (!aligned(x_dev, 16) || !aligned(m_dev, 16) || !aligned(llr_dev, 16))
        return fail(QCLDPC_E_ALIGN, "llr_8d: buffers must be 16-byte aligned");
    if (n == 0) return QCLDPC_OK;
    const int64_t nb = n / 8;
    llr8_kernel<<<stream_grid(nb), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4 *>(x_dev), reinterpret_cast<const float4 *>(m_dev),
        reinterpret_cast<float4 *>(llr_dev), snr * 0.25f, nb);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "llr_8d: launch");
    return QCLDPC_OK;
}

extern "C" int qcldpc_bob_message(int d, const float *y_dev, const uint32_t *bits_dev, int64_t n,
                                  float *m_dev, qcldpc_stream_t stream) {
    using namespace qc;
    if (d == 8) return qcldpc_bob_message_8d(y_dev, bits_dev, n, m_dev, stream);
    if ((d != 1 && d != 2 && d != 4) || !y_dev || !bits_dev || !m_dev || n < 0 || n % d != 0)
        return fail(QCLDPC_E_INVAL, "bob_message: d must be 1, 2, 4 or 8 and n a multiple of d");
    if (!aligned(y_dev, 4) || !aligned(m_dev, 4) || !aligned(bits_dev, 4))
        return fail(QCLDPC_E_ALIGN, "bob_message: buffers must be 4-byte aligned");
    if (n == 0) return QCLDPC_OK;
    const int64_t nb = n / d;
    cudaStream_t st = (cudaStream_t)stream;
    if (d == 1) bob_d_kernel<1><<<stream_grid(nb), 256, 0, st>>>(y_dev, bits_dev, m_dev, nb);
    else if (d == 2) bob_d_kernel<2><<<stream_grid(nb), 256, 0, st>>>(y_dev, bits_dev, m_dev, nb);
    else bob_d_kernel<4><<<stream_grid(nb), 256, 0, st>>>(y_dev, bits_dev, m_dev, nb);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "bob_message: launch");
    return QCLDPC_OK;
}

extern "C" int qcldpc_llr(int d, const float *x_dev, const float *m_dev, int64_t n, float snr,
                          float *llr_dev, qcldpc_stream_t stream) {
    using namespace qc;
    if (d == 8) return qcldpc_llr_8d(x_dev, m_dev, n, snr, llr_dev, stream);
    if ((d != 1 && d != 2 && d != 4) || !x_dev || !m_dev || !llr_dev || n < 0 || n % d != 0 ||
        !(snr > 0.0f))
        return fail(QCLDPC_E_INVAL, "llr: d must be 1, 2, 4 or 8, n a multiple of d, snr > 0");
    if (!aligned(x_dev, 4) || !aligned(m_dev, 4) || !aligned(llr_dev, 4))
        return fail(QCLDPC_E_ALIGN, "llr: buffers must be 4-byte aligned");
    if (n == 0) return QCLDPC_OK;
    const int64_t nb = n / d;
    const float scale = 2.0f * snr / (float)d;
    cudaStream_t st = (cudaStream_t)stream;
    if (d == 1) llr_d_kernel<1><<<stream_grid(nb), 256, 0, st>>>(x_dev, m_dev, llr_dev, scale, nb);
    else if (d == 2) llr_d_kernel<2><<<stream_grid(nb), 256, 0, st>>>(x_dev, m_dev, llr_dev, scale, nb);
    else llr_d_kernel<4><<<stream_grid(nb), 256, 0, st>>>(x_dev, m_dev, llr_dev, scale, nb);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "llr: launch");
    return QCLDPC_OK;
}
