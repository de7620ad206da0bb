// mfadvr_eval_points' launcher (picks the per-degree instantiation of the
// kernel in eval_kernels.cuh) and the kernels that build a model's row array
// and its span polynomials.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "eval_kernels.cuh"
#include "mfa_internal.h"

namespace mfadvr {
namespace {

__device__ __forceinline__ unsigned pack2(float a, float b, __half)
{
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const unsigned *>(&h);
}
__device__ __forceinline__ unsigned pack2(float a, float b, __nv_bfloat16)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const unsigned *>(&h);
}

// One thread per lattice point (i, j, k): gathers P(i..i+3, j..j+1, k)
// (FP32) or P(i..i+3, j..j+3, k) (FP16/BF16) as (j, j+1) pairs in the entry
// order of mfa_basis.cuh, zero past the lattice, scaled by inv_scale and
// rounded to the storage type.
template <typename T>
__global__ void build_rows_kernel(const float *__restrict__ src, void *__restrict__ dst, int n0, int n1, int n2,
                                  float inv_scale)
{
    constexpr int H = sizeof(T) == 4 ? 1 : 2;  // j pairs per entry
    const int64_t total = static_cast<int64_t>(n0) * n1 * n2;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e % n0);
        const int j = static_cast<int>((e / n0) % n1);
        float v[H][4][2];  // [h][d][j + 2h + c]
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
            for (int d = 0; d < 4; ++d)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const bool in = i + d < n0 && j + 2 * h + c < n1;
                    v[h][d][c] = in ? src[e + d + static_cast<int64_t>(2 * h + c) * n0] * inv_scale : 0.0f;
                }
        if constexpr (sizeof(T) == 4) {
            float4 *q = static_cast<float4 *>(dst) + 2 * e;
            q[0] = make_float4(v[0][0][0], v[0][0][1], v[0][1][0], v[0][1][1]);
            q[1] = make_float4(v[0][2][0], v[0][2][1], v[0][3][0], v[0][3][1]);
        } else {
            uint4 *q = static_cast<uint4 *>(dst) + 2 * e;
            q[0] = make_uint4(pack2(v[0][0][0], v[0][0][1], T()), pack2(v[0][1][0], v[0][1][1], T()),
                              pack2(v[0][2][0], v[0][2][1], T()), pack2(v[0][3][0], v[0][3][1], T()));
            q[1] = make_uint4(pack2(v[H - 1][0][0], v[H - 1][0][1], T()), pack2(v[H - 1][1][0], v[H - 1][1][1], T()),
                              pack2(v[H - 1][2][0], v[H - 1][2][1], T()), pack2(v[H - 1][3][0], v[H - 1][3][1], T()));
        }
    }
}

// One thread per span cell (i, j, k) of an FP32 model of degree P: the
// coefficients of the cell's polynomial about its centre (PolyCell in
// mfa_basis.cuh), A = (Cu x Cv x Cw) applied to the (P+1)^3 control points
// P(i.., j.., k..) one axis at a time, in FP64, each rounded once to FP32.
// cp0..cp2: each axis's span pieces about the span centres (FP64, m x (P+1)
// x (P+1), the host's centred_axis_pieces).
template <int P>
__global__ void build_poly_kernel(const float *__restrict__ src, float2 *__restrict__ poly, int n0, int n1, int n2,
                                  const double *__restrict__ cp0, const double *__restrict__ cp1,
                                  const double *__restrict__ cp2)
{
    constexpr int K = P + 1, S = PolyCell<P>::kSectors;
    const int m0 = n0 - P, m1 = n1 - P, m2 = n2 - P;
    const int64_t cells = static_cast<int64_t>(m0) * m1 * m2;
    for (int64_t cell = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; cell < cells;
         cell += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(cell % m0);
        const int j = static_cast<int>((cell / m0) % m1);
        const int k = static_cast<int>(cell / (static_cast<int64_t>(m0) * m1));
        double cu[K][K], cv[K][K], cw[K][K];
        for (int r = 0; r < K; ++r)
            for (int e = 0; e < K; ++e) {
                cu[r][e] = cp0[(static_cast<int64_t>(i) * K + r) * K + e];
                cv[r][e] = cp1[(static_cast<int64_t>(j) * K + r) * K + e];
                cw[r][e] = cp2[(static_cast<int64_t>(k) * K + r) * K + e];
            }
        double t[K][K][K];  // t[a][s][q] = sum_r cu[r][a] P(i+r, j+s, k+q)
        for (int q = 0; q < K; ++q)
            for (int s = 0; s < K; ++s) {
                const float *row = src + i + static_cast<int64_t>(n0) * (j + s + static_cast<int64_t>(n1) * (k + q));
                for (int a = 0; a < K; ++a) {
                    double acc = 0.0;
                    for (int r = 0; r < K; ++r) acc += cu[r][a] * static_cast<double>(row[r]);
                    t[a][s][q] = acc;
                }
            }
        double w[K][K][K];  // w[a][b][q] = sum_s cv[s][b] t[a][s][q]
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b)
                for (int q = 0; q < K; ++q) {
                    double acc = 0.0;
                    for (int s = 0; s < K; ++s) acc += cv[s][b] * t[a][s][q];
                    w[a][b][q] = acc;
                }
        float2 *out = poly + cell * (4 * S);
        for (int f = 0; f < 4 * S; ++f) {
            const int g = f / (K * K), b = (f / K) % K, a = f % K;
            float2 pr = make_float2(0.0f, 0.0f);
            if (f < PolyCell<P>::kPairs) {
                double lo = 0.0, hi = 0.0;  // A[a][b][2g], A[a][b][2g+1]
                for (int q = 0; q < K; ++q) {
                    lo += cw[q][2 * g] * w[a][b][q];
                    if (2 * g + 1 < K) hi += cw[q][2 * g + 1] * w[a][b][q];
                }
                pr = make_float2(static_cast<float>(lo), static_cast<float>(hi));
            }
            out[f] = pr;
        }
    }
}

}  // namespace

cudaError_t launch_eval_points(const ModelView &mv, const float *params, int64_t n, float *out, int query,
                               int32_t *spans, cudaStream_t stream, int max_blocks)
{
    if (n <= 0) return cudaSuccess;
    switch (mv.p) {
    case 1: return launch_eval_p1(mv, params, n, out, query, spans, stream, max_blocks);
    case 2: return launch_eval_p2(mv, params, n, out, query, spans, stream, max_blocks);
    case 3: return launch_eval_p3(mv, params, n, out, query, spans, stream, max_blocks);
    case 4: return launch_eval_p4(mv, params, n, out, query, spans, stream, max_blocks);
    case 5: return launch_eval_p5(mv, params, n, out, query, spans, stream, max_blocks);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_build_poly(const float *src, void *poly, int p, int n0, int n1, int n2,
                              const double *const pieces[3], cudaStream_t stream)
{
    const int64_t cells = static_cast<int64_t>(n0 - p) * (n1 - p) * (n2 - p);
    if (cells <= 0) return cudaSuccess;
    const int blocks = static_cast<int>((cells + 127) / 128 < 152 * 32 ? (cells + 127) / 128 : 152 * 32);
    float2 *dst = static_cast<float2 *>(poly);
    switch (p) {
    case 1:
        build_poly_kernel<1><<<blocks, 128, 0, stream>>>(src, dst, n0, n1, n2, pieces[0], pieces[1], pieces[2]);
        break;
    case 2:
        build_poly_kernel<2><<<blocks, 128, 0, stream>>>(src, dst, n0, n1, n2, pieces[0], pieces[1], pieces[2]);
        break;
    case 3:
        build_poly_kernel<3><<<blocks, 128, 0, stream>>>(src, dst, n0, n1, n2, pieces[0], pieces[1], pieces[2]);
        break;
    case 4:
        build_poly_kernel<4><<<blocks, 128, 0, stream>>>(src, dst, n0, n1, n2, pieces[0], pieces[1], pieces[2]);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_build_rows(const float *src, void *rows, int n0, int n1, int n2, int dtype, float inv_scale,
                              cudaStream_t stream)
{
    const int64_t total = static_cast<int64_t>(n0) * n1 * n2;
    if (total <= 0) return cudaSuccess;
    const int blocks = static_cast<int>((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
    switch (dtype) {
    case MFADVR_F32:
        build_rows_kernel<float><<<blocks, 256, 0, stream>>>(src, rows, n0, n1, n2, inv_scale);
        break;
    case MFADVR_F16:
        build_rows_kernel<__half><<<blocks, 256, 0, stream>>>(src, rows, n0, n1, n2, inv_scale);
        break;
    case MFADVR_BF16:
        build_rows_kernel<__nv_bfloat16><<<blocks, 256, 0, stream>>>(src, rows, n0, n1, n2, inv_scale);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace mfadvr
