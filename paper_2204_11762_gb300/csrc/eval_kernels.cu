// mfadvr_eval_points: value and first derivatives of the MFA model at
// arbitrary parameter points (queryValueMFA + queryGradientMFA of
// Algorithm 1, computed together as Sec. 3.1 describes).
//
// One thread per point, grid-stride over a grid sized to the SM count.  The
// span index is exact integer work (see span_exact); basis and contraction
// run in FP32 on the FMA pipe; control points come through the read-only
// cache (the lattices of the point workloads are L2-resident).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mfa_basis.cuh"
#include "mfa_internal.h"

namespace mfadvr {
namespace {

template <int P, typename T>
__global__ void __launch_bounds__(256) eval_points_kernel(ModelView mv, const float *__restrict__ params,
                                                          int64_t n, float4 *__restrict__ out,
                                                          int32_t *__restrict__ spans)
{
    const T *__restrict__ cp = static_cast<const T *>(mv.cp);
    const float mf0 = static_cast<float>(mv.m[0]);
    const float mf1 = static_cast<float>(mv.m[1]);
    const float mf2 = static_cast<float>(mv.m[2]);
    const int64_t sj = mv.n[0];
    const int64_t sk = static_cast<int64_t>(mv.n[0]) * mv.n[1];
    const float s0 = mv.scale * mf0, s1 = mv.scale * mf1, s2 = mv.scale * mf2;

    for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < n;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        // fminf/fmaxf return the non-NaN operand: NaN clamps to 0.
        const float u = fminf(fmaxf(params[3 * idx + 0], 0.0f), 1.0f);
        const float v = fminf(fmaxf(params[3 * idx + 1], 0.0f), 1.0f);
        const float w = fminf(fmaxf(params[3 * idx + 2], 0.0f), 1.0f);
        const int k0 = span_exact(u, mv.m[0], mf0);
        const int k1 = span_exact(v, mv.m[1], mf1);
        const int k2 = span_exact(w, mv.m[2], mf2);
        float Nu[P + 1], dNu[P + 1], Nv[P + 1], dNv[P + 1], Nw[P + 1], dNw[P + 1];
        basis<P>(fmaf(u, mf0, -static_cast<float>(k0)), k0, mv.m[0], Nu, dNu);
        basis<P>(fmaf(v, mf1, -static_cast<float>(k1)), k1, mv.m[1], Nv, dNv);
        basis<P>(fmaf(w, mf2, -static_cast<float>(k2)), k2, mv.m[2], Nw, dNw);

        const T *base = cp + (k0 + sj * k1 + sk * k2);
        float r[4];
        contract<P>(Nu, dNu, Nv, dNv, Nw, dNw,
                    [&](int i, int j, int k) { return load_cp<T>(base + i + sj * j + sk * k); }, r);
        out[idx] = make_float4(r[0] * mv.scale, r[1] * s0, r[2] * s1, r[3] * s2);
        if (spans) {
            spans[3 * idx + 0] = k0 + P;
            spans[3 * idx + 1] = k1 + P;
            spans[3 * idx + 2] = k2 + P;
        }
    }
}

template <int P, typename T>
cudaError_t launch_eval_t(const ModelView &mv, const float *params, int64_t n, float4 *out, int32_t *spans,
                          cudaStream_t stream)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eval_points_kernel<P, T>, 256, 0);
    if (per_sm < 1) per_sm = 1;
    const int64_t need = (n + 255) / 256;
    const int64_t cap = static_cast<int64_t>(sms) * per_sm;
    const int blocks = static_cast<int>(need < cap ? need : cap);
    eval_points_kernel<P, T><<<blocks, 256, 0, stream>>>(mv, params, n, out, spans);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_eval_dtype(const ModelView &mv, const float *params, int64_t n, float4 *out, int32_t *spans,
                              cudaStream_t stream)
{
    switch (mv.p) {
    case 1: return launch_eval_t<1, T>(mv, params, n, out, spans, stream);
    case 2: return launch_eval_t<2, T>(mv, params, n, out, spans, stream);
    case 3: return launch_eval_t<3, T>(mv, params, n, out, spans, stream);
    case 4: return launch_eval_t<4, T>(mv, params, n, out, spans, stream);
    case 5: return launch_eval_t<5, T>(mv, params, n, out, spans, stream);
    default: return cudaErrorInvalidValue;
    }
}

__device__ __forceinline__ void store_q(__half *d, float v) { *d = __float2half_rn(v); }
__device__ __forceinline__ void store_q(__nv_bfloat16 *d, float v) { *d = __float2bfloat16_rn(v); }

template <typename T>
__global__ void quantize_kernel(const float *__restrict__ src, T *__restrict__ dst, int64_t count, float inv_scale)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        store_q(dst + i, src[i] * inv_scale);
}

}  // namespace

cudaError_t launch_eval_points(const ModelView &mv, const float *params, int64_t n, float4 *out, int32_t *spans,
                               cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    switch (mv.dtype) {
    case MFADVR_F32: return launch_eval_dtype<float>(mv, params, n, out, spans, stream);
    case MFADVR_F16: return launch_eval_dtype<__half>(mv, params, n, out, spans, stream);
    case MFADVR_BF16: return launch_eval_dtype<__nv_bfloat16>(mv, params, n, out, spans, stream);
    default: return cudaErrorInvalidValue;
    }
}

// P / s rounded to nearest in the storage type.
cudaError_t launch_quantize(const float *src, void *dst, int64_t count, int dtype, float inv_scale,
                            cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    const int blocks = static_cast<int>((count + 255) / 256 < 152 * 16 ? (count + 255) / 256 : 152 * 16);
    if (dtype == MFADVR_F16)
        quantize_kernel<__half><<<blocks, 256, 0, stream>>>(src, static_cast<__half *>(dst), count, inv_scale);
    else if (dtype == MFADVR_BF16)
        quantize_kernel<__nv_bfloat16>
            <<<blocks, 256, 0, stream>>>(src, static_cast<__nv_bfloat16 *>(dst), count, inv_scale);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace mfadvr
