// mfadvr_eval_points / mfadvr_query_points: the value, the first
// derivatives, both (queryValueMFA + queryGradientMFA of Algorithm 1,
// computed together as Sec. 3.1 describes) or the second derivatives too
// (Sec. 3.1's higher-order query) at arbitrary parameter points.  The kernel
// template lives here; eval_p1.cu .. eval_p5.cu instantiate one degree each
// and eval_kernels.cu picks the degree and builds the row arrays.
//
// One thread per point, grid-stride over a grid sized to the SM count.  The
// span index is exact integer work (span_exact on uniform knots, span_search
// on general ones); basis and contraction run in FP32 on the FMA pipe; the
// span block is gathered from the row array, one 32-byte sector per entry
// (8 entries at degree 3 in FP32, 4 in 16 bits).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mfa_basis.cuh"
#include "mfa_internal.h"

namespace mfadvr {
namespace {

// Points whose parameters a thread loads ahead of the one it evaluates: one
// (measured: 3-10% faster), except in the FP32 Hessian query, whose 2^24-point
// run took 1.08 ms with it and 0.88 ms without.
template <typename T, int Q>
struct PointsAhead {
    static constexpr int value = (Q == kQueryHessian && sizeof(T) == 4) ? 0 : 1;
};

// NU: general knots (span search, per-span pieces); otherwise uniform knots
// (exact floor, uniform pieces or the clamped-pattern table).  R: rational
// model, rows hold w P and wrows w; f = A / W and grad f = (grad A - f grad W)
// / W from the two contractions (the weights' gradient only when the
// gradient is queried).
template <int P, typename T, int Q, bool NU, bool R>
__global__ void __launch_bounds__(256) eval_points_kernel(ModelView mv, const float *__restrict__ params,
                                                          int64_t n, float *__restrict__ out,
                                                          int32_t *__restrict__ spans)
{
    const float mf0 = static_cast<float>(mv.m[0]);
    const float mf1 = static_cast<float>(mv.m[1]);
    const float mf2 = static_cast<float>(mv.m[2]);
    constexpr float bs = BasisScale<P>::value;
    // value scale of a contraction: storage scale / basis scale^3 (a rational
    // model's A / W carries neither)
    const float sv = R ? 1.0f : mv.scale / (bs * bs * bs);
    const int n0 = mv.n[0], n01 = mv.n01;
    // a rational query needs W always and A's value for the gradient too
    constexpr int QA = R ? (Q == kQueryValue ? kQueryValue : kQueryBoth) : Q;

    // Points and outputs stream through once: loaded and stored with the
    // evict-first hint so that they do not push the row array out of L2.  A
    // thread keeps the parameters of its next kPointsAhead points in flight
    // while it evaluates the current one (the points may sit in host memory,
    // a few microseconds away).
    constexpr int kPointsAhead = PointsAhead<T, Q>::value;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    float ahead[kPointsAhead + 1][3];
#pragma unroll
    for (int q = 0; q < kPointsAhead; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            ahead[q][c] = idx + q * stride < n ? __ldcs(params + 3 * (idx + q * stride) + c) : 0.0f;
    for (; idx < n; idx += stride) {
        {
            const int64_t j = idx + kPointsAhead * stride;
#pragma unroll
            for (int c = 0; c < 3; ++c) ahead[kPointsAhead][c] = j < n ? __ldcs(params + 3 * j + c) : 0.0f;
        }
        // fminf/fmaxf return the non-NaN operand: NaN clamps to 0.
        const float u = fminf(fmaxf(ahead[0][0], 0.0f), 1.0f);
        const float v = fminf(fmaxf(ahead[0][1], 0.0f), 1.0f);
        const float w = fminf(fmaxf(ahead[0][2], 0.0f), 1.0f);
#pragma unroll
        for (int q = 0; q < kPointsAhead; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) ahead[q][c] = ahead[q + 1][c];
        int k0, k1, k2;
        float x0, x1, x2;
        float d0 = mf0, d1 = mf1, d2 = mf2;  // d/du = d * d/dx (1 / span width)
        if constexpr (NU) {
            k0 = span_search(mv.brk[0], mv.cell[0], mv.grid[0], u);
            k1 = span_search(mv.brk[1], mv.cell[1], mv.grid[1], v);
            k2 = span_search(mv.brk[2], mv.cell[2], mv.grid[2], w);
            d0 = __ldg(mv.ih[0] + k0);
            d1 = __ldg(mv.ih[1] + k1);
            d2 = __ldg(mv.ih[2] + k2);
            x0 = (u - __ldg(mv.brk[0] + k0)) * d0;
            x1 = (v - __ldg(mv.brk[1] + k1)) * d1;
            x2 = (w - __ldg(mv.brk[2] + k2)) * d2;
        } else {
            k0 = span_exact(u, mv.m[0], mf0);
            k1 = span_exact(v, mv.m[1], mf1);
            k2 = span_exact(w, mv.m[2], mf2);
            x0 = fmaf(u, mf0, -static_cast<float>(k0));
            x1 = fmaf(v, mf1, -static_cast<float>(k1));
            x2 = fmaf(w, mf2, -static_cast<float>(k2));
        }
        const int base = k0 + n0 * k1 + n01 * k2;
        if constexpr (Q == kQueryHessian) {
            // value, gradient and the six second partials (Sec. 3.1's
            // higher-order query); order (a, b, c) scales by d0^a d1^b d2^c
            float Bu[3][P + 1], Bv[3][P + 1], Bw[3][P + 1];
            if constexpr (NU) {
                basis_pieces_d2<P>(x0, mv.pieces[0], k0, Bu[0], Bu[1], Bu[2]);
                basis_pieces_d2<P>(x1, mv.pieces[1], k1, Bv[0], Bv[1], Bv[2]);
                basis_pieces_d2<P>(x2, mv.pieces[2], k2, Bw[0], Bw[1], Bw[2]);
            } else {
                basis_d2<P>(x0, k0, mv.m[0], Bu[0], Bu[1], Bu[2]);
                basis_d2<P>(x1, k1, mv.m[1], Bv[0], Bv[1], Bv[2]);
                basis_d2<P>(x2, k2, mv.m[2], Bw[0], Bw[1], Bw[2]);
            }
            float h[10];
            contract_hessian<P>(Bu, Bv, Bw,
                                [&](int k, int jp, int i) { return row_pair<T>(mv.rows, base, n0, n01, k, jp, i); }, h);
            if constexpr (R) {
                float g[10];
                contract_hessian<P>(
                    Bu, Bv, Bw, [&](int k, int jp, int i) { return row_pair<T>(mv.wrows, base, n0, n01, k, jp, i); },
                    g);
                // f = A / W, f_i = (A_i - f W_i) / W,
                // f_ij = (A_ij - f_i W_j - f_j W_i - f W_ij) / W
#pragma unroll
                for (int o = 0; o < 10; ++o) {
                    h[o] *= mv.scale;
                    g[o] *= mv.wscale;
                }
                const float W = g[0], f = h[0] / W;
                float f1[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) f1[d] = (h[1 + d] - f * g[1 + d]) / W;
                constexpr int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
                for (int o = 0; o < 6; ++o)
                    h[4 + o] = (h[4 + o] - f1[pi[o]] * g[1 + pj[o]] - f1[pj[o]] * g[1 + pi[o]] - f * g[4 + o]) / W;
                h[0] = f;
#pragma unroll
                for (int d = 0; d < 3; ++d) h[1 + d] = f1[d];
            }
            const float dd[3] = {d0, d1, d2};
#pragma unroll
            for (int o = 0; o < 10; ++o) {
                float sc = sv;
#pragma unroll
                for (int axis = 0; axis < 3; ++axis)
#pragma unroll
                    for (int e = 0; e < hessian_order(o, axis); ++e) sc *= dd[axis];
                __stcs(out + 10 * idx + o, h[o] * sc);
            }
            if (spans) {
                __stcs(spans + 3 * idx + 0, k0 + P);
                __stcs(spans + 3 * idx + 1, k1 + P);
                __stcs(spans + 3 * idx + 2, k2 + P);
            }
            continue;
        }
        float r[4];
        float Nu[P + 1], dNu[P + 1], Nv[P + 1], dNv[P + 1], Nw[P + 1], dNw[P + 1];
        auto basis3 = [&]() {
            if constexpr (NU) {
                basis_pieces<P>(x0, mv.pieces[0], k0, Nu, dNu);
                basis_pieces<P>(x1, mv.pieces[1], k1, Nv, dNv);
                basis_pieces<P>(x2, mv.pieces[2], k2, Nw, dNw);
            } else {
                basis<P>(x0, k0, mv.m[0], Nu, dNu);
                basis<P>(x1, k1, mv.m[1], Nv, dNv);
                basis<P>(x2, k2, mv.m[2], Nw, dNw);
            }
        };
        if constexpr (P <= 3 && !R) {
            // the whole block in flight before the basis is evaluated
            typename Entries<P, T>::E q[P + 1][Entries<P, T>::JE][Block<P>::IR];
            load_block<P, T>(mv.rows, base, n0, n01, q);
            basis3();
            contract<P, Q>(Nu, dNu, Nv, dNv, Nw, dNw,
                           [&](int k, int jp, int i) { return block_pair<P, T>(q, k, jp, i); }, r);
        } else {
            basis3();
            contract<P, QA>(Nu, dNu, Nv, dNv, Nw, dNw,
                            [&](int k, int jp, int i) { return row_pair<T>(mv.rows, base, n0, n01, k, jp, i); }, r);
        }
        if constexpr (R) {
            float rw[4];
            contract<P, QA>(Nu, dNu, Nv, dNv, Nw, dNw,
                            [&](int k, int jp, int i) { return row_pair<T>(mv.wrows, base, n0, n01, k, jp, i); }, rw);
            // the basis scale cancels in A / W; the storage scales do not
            const float W = rw[0] * mv.wscale, f = (r[0] * mv.scale) / W;
            if constexpr (QA == kQueryBoth) {
#pragma unroll
                for (int d = 1; d < 4; ++d) r[d] = (r[d] * mv.scale - f * (rw[d] * mv.wscale)) / W;
            }
            r[0] = f;
        }
        const float g0 = sv * d0, g1 = sv * d1, g2 = sv * d2;
        if constexpr (Q == kQueryBoth) {
            __stcs(reinterpret_cast<float4 *>(out) + idx, make_float4(r[0] * sv, r[1] * g0, r[2] * g1, r[3] * g2));
        } else if constexpr (Q == kQueryValue) {
            __stcs(out + idx, r[0] * sv);
        } else {
            __stcs(out + 3 * idx + 0, r[1] * g0);
            __stcs(out + 3 * idx + 1, r[2] * g1);
            __stcs(out + 3 * idx + 2, r[3] * g2);
        }
        if (spans) {
            __stcs(spans + 3 * idx + 0, k0 + P);
            __stcs(spans + 3 * idx + 1, k1 + P);
            __stcs(spans + 3 * idx + 2, k2 + P);
        }
    }
}

template <int P, typename T, int Q, bool NU, bool R>
cudaError_t launch_eval_k(const ModelView &mv, const float *params, int64_t n, float *out, int32_t *spans,
                          cudaStream_t stream, int max_blocks)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eval_points_kernel<P, T, Q, NU, R>, 256, 0);
    if (per_sm < 1) per_sm = 1;
    const int64_t need = (n + 255) / 256;
    int64_t cap = static_cast<int64_t>(sms) * per_sm;
    if (max_blocks > 0 && max_blocks < cap) cap = max_blocks;
    const int blocks = static_cast<int>(need < cap ? need : cap);
    eval_points_kernel<P, T, Q, NU, R><<<blocks, 256, 0, stream>>>(mv, params, n, out, spans);
    return cudaGetLastError();
}

template <int P, typename T, int Q>
cudaError_t launch_eval_q(const ModelView &mv, const float *params, int64_t n, float *out, int32_t *spans,
                          cudaStream_t stream, int max_blocks)
{
    if (mv.rational)
        return mv.nu ? launch_eval_k<P, T, Q, true, true>(mv, params, n, out, spans, stream, max_blocks)
                     : launch_eval_k<P, T, Q, false, true>(mv, params, n, out, spans, stream, max_blocks);
    return mv.nu ? launch_eval_k<P, T, Q, true, false>(mv, params, n, out, spans, stream, max_blocks)
                 : launch_eval_k<P, T, Q, false, false>(mv, params, n, out, spans, stream, max_blocks);
}

template <int P, typename T>
cudaError_t launch_eval_t(const ModelView &mv, const float *params, int64_t n, float *out, int query,
                          int32_t *spans, cudaStream_t stream, int max_blocks)
{
    switch (query) {
    case kQueryValue: return launch_eval_q<P, T, kQueryValue>(mv, params, n, out, spans, stream, max_blocks);
    case kQueryGradient:
        return launch_eval_q<P, T, kQueryGradient>(mv, params, n, out, spans, stream, max_blocks);
    case kQueryBoth: return launch_eval_q<P, T, kQueryBoth>(mv, params, n, out, spans, stream, max_blocks);
    case kQueryHessian:
        return launch_eval_q<P, T, kQueryHessian>(mv, params, n, out, spans, stream, max_blocks);
    default: return cudaErrorInvalidValue;
    }
}

template <int P, typename T>
cudaError_t launch_eval_dtype_p(const ModelView &mv, const float *params, int64_t n, float *out, int query,
                                int32_t *spans, cudaStream_t stream, int max_blocks)
{
    return launch_eval_t<P, T>(mv, params, n, out, query, spans, stream, max_blocks);
}

}  // namespace

// The per-degree launcher one eval_pN.cu defines.
#define MFADVR_EVAL_DEGREE(PP)                                                                               \
    cudaError_t launch_eval_p##PP(const ModelView &mv, const float *params, int64_t n, float *out, int query, \
                                  int32_t *spans, cudaStream_t stream, int max_blocks)                       \
    {                                                                                                        \
        switch (mv.dtype) {                                                                                  \
        case MFADVR_F32:                                                                                     \
            return launch_eval_dtype_p<PP, float>(mv, params, n, out, query, spans, stream, max_blocks);     \
        case MFADVR_F16:                                                                                     \
            return launch_eval_dtype_p<PP, __half>(mv, params, n, out, query, spans, stream, max_blocks);    \
        case MFADVR_BF16:                                                                                    \
            return launch_eval_dtype_p<PP, __nv_bfloat16>(mv, params, n, out, query, spans, stream,          \
                                                          max_blocks);                                       \
        default: return cudaErrorInvalidValue;                                                               \
        }                                                                                                    \
    }

cudaError_t launch_eval_p1(const ModelView &, const float *, int64_t, float *, int, int32_t *, cudaStream_t, int);
cudaError_t launch_eval_p2(const ModelView &, const float *, int64_t, float *, int, int32_t *, cudaStream_t, int);
cudaError_t launch_eval_p3(const ModelView &, const float *, int64_t, float *, int, int32_t *, cudaStream_t, int);
cudaError_t launch_eval_p4(const ModelView &, const float *, int64_t, float *, int, int32_t *, cudaStream_t, int);
cudaError_t launch_eval_p5(const ModelView &, const float *, int64_t, float *, int, int32_t *, cudaStream_t, int);

}  // namespace mfadvr
