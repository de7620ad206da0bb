// Device-side pieces of the MFA query (Sec. 2.3 model; queryValueMFA /
// queryGradientMFA of Algorithm 1): knot-span lookup, B-spline basis and
// first derivatives, control-point loads.
//
// Everything works in span-local coordinates.  With clamped uniform knots
// t_{p+j} = j/m, span s = p + k (k = 0..m-1) covers [k/m, (k+1)/m), and the
// local coordinate x = u*m - k lies in [0, 1].  In units of 1/m, the knots
// around the span sit at the integers kappa(j) = clamp(k + j, 0, m) - k, so
// the Cox-de Boor denominators are small integers and the first control
// point touched by the span is index k.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace mfadvr {

// ---------------------------------------------------------------------------
// Uniform pieces: on a span whose 2p surrounding knots are all distinct
// (kappa(j) = j), the p+1 non-zero basis functions are fixed polynomials of
// the local coordinate.  Their monomial coefficients are computed at compile
// time by running the Cox-de Boor recurrence on polynomials.
// ---------------------------------------------------------------------------
template <int P>
struct UniformPieces {
    float c[P + 1][P + 1];  // N_r(x)  = sum_e c[r][e] x^e
    float d[P + 1][P + 1];  // N'_r(x) = sum_e d[r][e] x^e  (d/dx, d[r][P] = 0)
};

template <int P>
constexpr UniformPieces<P> make_uniform_pieces()
{
    // B[q][r][e]: coefficient of x^e of N_{s-q+r, q}, knots kappa(j) = j.
    double B[P + 1][P + 1][P + 2] = {};
    B[0][0][0] = 1.0;
    for (int q = 1; q <= P; ++q) {
        for (int r = 0; r <= q; ++r) {
            const int i = r - q;  // N_{s+i,q}
            const double den = q; // kappa(i+q) - kappa(i) = kappa(i+q+1) - kappa(i+1) = q
            for (int e = 0; e <= P; ++e) {
                if (r > 0) {      // (x - i)/q * N_{s+i, q-1}
                    B[q][r][e + 1] += B[q - 1][r - 1][e] / den;
                    B[q][r][e] -= i * B[q - 1][r - 1][e] / den;
                }
                if (r < q) {      // (i + q + 1 - x)/q * N_{s+i+1, q-1}
                    B[q][r][e] += (i + q + 1) * B[q - 1][r][e] / den;
                    B[q][r][e + 1] -= B[q - 1][r][e] / den;
                }
            }
        }
    }
    UniformPieces<P> out{};
    for (int r = 0; r <= P; ++r) {
        for (int e = 0; e <= P; ++e) {
            out.c[r][e] = static_cast<float>(B[P][r][e]);
            out.d[r][e] = (e < P) ? static_cast<float>((e + 1) * B[P][r][e + 1]) : 0.0f;
        }
    }
    return out;
}

// Values and local derivatives of the uniform pieces by Horner's rule.
template <int P>
__device__ __forceinline__ void basis_uniform(float x, float N[P + 1], float dN[P + 1])
{
    constexpr UniformPieces<P> U = make_uniform_pieces<P>();
#pragma unroll
    for (int r = 0; r <= P; ++r) {
        float v = U.c[r][P];
#pragma unroll
        for (int e = P - 1; e >= 0; --e) v = fmaf(v, x, U.c[r][e]);
        N[r] = v;
        float dv = U.d[r][P - 1];
#pragma unroll
        for (int e = P - 2; e >= 0; --e) dv = fmaf(dv, x, U.d[r][e]);
        dN[r] = dv;
    }
}

// Any span (including the clamped ones near the ends): the Cox-de Boor
// triangle with left/right differences (the published form, Piegl & Tiller,
// The NURBS Book, Sec. 2.2-2.3) on the integer knots kappa(j).
template <int P>
__device__ __forceinline__ void basis_general(float x, int k, int m, float N[P + 1], float dN[P + 1])
{
    float left[P + 1], right[P + 1];
#pragma unroll
    for (int j = 1; j <= P; ++j) {
        left[j] = x - static_cast<float>(min(max(k + 1 - j, 0), m) - k);
        right[j] = static_cast<float>(min(max(k + j, 0), m) - k) - x;
    }
    float Nq[P + 1];
    float Nlow[P + 1];  // degree P-1 values, for the derivatives
    Nq[0] = 1.0f;
#pragma unroll
    for (int q = 1; q <= P; ++q) {
        if (q == P) {
#pragma unroll
            for (int r = 0; r < P; ++r) Nlow[r] = Nq[r];
        }
        float saved = 0.0f;
#pragma unroll
        for (int r = 0; r < q; ++r) {
            const float tmp = Nq[r] * __frcp_rn(right[r + 1] + left[q - r]);
            Nq[r] = fmaf(right[r + 1], tmp, saved);
            saved = left[q - r] * tmp;
        }
        Nq[q] = saved;
    }
    // N'_{i,P} = P (N_{i,P-1}/(t_{i+P}-t_i) - N_{i+1,P-1}/(t_{i+P+1}-t_{i+1}))
    // for i = s-P+r, r = 0..P.  In kappa units the two knot differences are
    // kappa(r) - kappa(r-P) and kappa(r+1) - kappa(r+1-P); N_{i,P-1} is
    // Nlow[r-1] and N_{i+1,P-1} is Nlow[r].
#pragma unroll
    for (int r = 0; r <= P; ++r) {
        float dv = 0.0f;
        if (r > 0) {
            const float den = static_cast<float>(min(max(k + r, 0), m) - min(max(k + r - P, 0), m));
            dv = Nlow[r - 1] * __frcp_rn(den);
        }
        if (r < P) {
            const float den = static_cast<float>(min(max(k + r + 1, 0), m) - min(max(k + r + 1 - P, 0), m));
            dv -= Nlow[r] * __frcp_rn(den);
        }
        N[r] = Nq[r];
        dN[r] = static_cast<float>(P) * dv;
    }
}

// Basis on span k of an axis with m spans: uniform pieces when the span's
// knots are unclamped (p-1 <= k <= m-p), the general triangle otherwise.
template <int P>
__device__ __forceinline__ void basis(float x, int k, int m, float N[P + 1], float dN[P + 1])
{
    if (k >= P - 1 && k <= m - P) basis_uniform<P>(x, N, dN);
    else basis_general<P>(x, k, m, N, dN);
}

// Exact k = floor(u*m) for FP32 u in [0, 1], clamped to [0, m-1].  The FP32
// product may round across an integer; a fused multiply-add gives the sign
// of the exact residual u*m - k (one rounding never changes a sign), which
// corrects it.
__device__ __forceinline__ int span_exact(float u, int m, float mf)
{
    int k = static_cast<int>(u * mf);
    if (fmaf(u, mf, -static_cast<float>(k)) < 0.0f) k -= 1;
    else if (fmaf(u, mf, -static_cast<float>(k + 1)) >= 0.0f) k += 1;
    return min(max(k, 0), m - 1);
}

// Storage-type loads through the read-only path.
template <typename T>
__device__ __forceinline__ float load_cp(const T *p);
template <>
__device__ __forceinline__ float load_cp<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load_cp<__half>(const __half *p) { return __half2float(__ldg(p)); }
template <>
__device__ __forceinline__ float load_cp<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}

// Sum-factorised contraction of the (P+1)^3 control points with the basis:
//   f  = sum N_i N_j N_k P_ijk,   f_u = sum N'_i N_j N_k P_ijk, ...
// u first (2 sums per row), then v (3 sums), then w (4 sums):
// 2(P+1)^3 + 3(P+1)^2 + 4(P+1) fused multiply-adds.  `cp(i, j, k)` yields the
// control point; r = {f, df/dx_u, df/dx_v, df/dx_w} in local units.
template <int P, typename CP>
__device__ __forceinline__ void contract(const float Nu[P + 1], const float dNu[P + 1], const float Nv[P + 1],
                                         const float dNv[P + 1], const float Nw[P + 1], const float dNw[P + 1],
                                         CP cp, float r[4])
{
    float f = 0.f, fu = 0.f, fv = 0.f, fw = 0.f;
#pragma unroll
    for (int k = 0; k <= P; ++k) {
        float c = 0.f, dv = 0.f, e = 0.f;
#pragma unroll
        for (int j = 0; j <= P; ++j) {
            float a = 0.f, b = 0.f;
#pragma unroll
            for (int i = 0; i <= P; ++i) {
                const float pv = cp(i, j, k);
                a = fmaf(Nu[i], pv, a);
                b = fmaf(dNu[i], pv, b);
            }
            c = fmaf(Nv[j], a, c);
            dv = fmaf(dNv[j], a, dv);
            e = fmaf(Nv[j], b, e);
        }
        f = fmaf(Nw[k], c, f);
        fw = fmaf(dNw[k], c, fw);
        fv = fmaf(Nw[k], dv, fv);
        fu = fmaf(Nw[k], e, fu);
    }
    r[0] = f;
    r[1] = fu;
    r[2] = fv;
    r[3] = fw;
}

}  // namespace mfadvr
