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

#include "mfa_internal.h"

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

// Scale of the basis values returned by basis_uniform_scaled<P>: the cubic
// closed form below returns 6 N and 6 N' (its coefficients are integers);
// other degrees return N and N' unscaled.  Contractions carry the factor
// kBasisScale<P>^3 until the end.
template <int P>
struct BasisScale {
    static constexpr float value = 1.0f;
};
template <>
struct BasisScale<3> {
    static constexpr float value = 6.0f;
};
static_assert(BasisScale<3>::value == basis_scale_host(3) && BasisScale<2>::value == basis_scale_host(2),
              "host and device basis scales differ");

// Uniform pieces times BasisScale<P>.  Degree 3 uses the closed form of the
// cubic B-spline in t = x and s = 1 - x:
//   6N0 = s^3, 6N1 = 4 + t^2 (3t - 6), 6N2 = 4 + s^2 (3s - 6), 6N3 = t^3,
//   6N0' = -3s^2, 6N1' = t (9t - 12), 6N2' = -s (9s - 12), 6N3' = 3t^2.
template <int P>
__device__ __forceinline__ void basis_uniform_scaled(float x, float N[P + 1], float dN[P + 1])
{
    if constexpr (P == 3) {
        const float t = x, s = 1.0f - x;
        const float t2 = t * t, s2 = s * s;
        N[0] = s2 * s;
        N[1] = fmaf(t2, fmaf(3.0f, t, -6.0f), 4.0f);
        N[2] = fmaf(s2, fmaf(3.0f, s, -6.0f), 4.0f);
        N[3] = t2 * t;
        dN[0] = -3.0f * s2;
        dN[1] = t * fmaf(9.0f, t, -12.0f);
        dN[2] = -s * fmaf(9.0f, s, -12.0f);
        dN[3] = 3.0f * t2;
    } else {
        basis_uniform<P>(x, N, dN);
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

// True when span k of an axis with m spans has unclamped knots
// (p-1 <= k <= m-p), i.e. the uniform pieces apply.
template <int P>
__device__ __forceinline__ bool span_interior(int k, int m)
{
    return k >= P - 1 && k <= m - P;
}

// Basis on span k of an axis with m spans, times BasisScale<P>: uniform
// pieces on unclamped spans, the general triangle otherwise.
template <int P>
__device__ __forceinline__ void basis(float x, int k, int m, float N[P + 1], float dN[P + 1])
{
    if (span_interior<P>(k, m)) {
        basis_uniform_scaled<P>(x, N, dN);
    } else {
        basis_general<P>(x, k, m, N, dN);
        if constexpr (BasisScale<P>::value != 1.0f) {
#pragma unroll
            for (int r = 0; r <= P; ++r) {
                N[r] *= BasisScale<P>::value;
                dN[r] *= BasisScale<P>::value;
            }
        }
    }
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

// ---------------------------------------------------------------------------
// Quad layout of the control points.  Entry (i, j, k) of the quad array holds
//   {P(i,j,k), P(i,j+1,k), P(i+1,j,k), P(i+1,j+1,k)}
// (zero where i+1 or j+1 runs past the lattice), so the (p+1) x (p+1) block
// of a k-slice under any span is ceil((p+1)/2)^2 aligned vector loads, and
// each load yields two (P(i,j), P(i,j+1)) pairs ready for packed FMAs.
// FP32 entries are 16 bytes, FP16/BF16 entries 8 bytes.
// ---------------------------------------------------------------------------
template <typename T>
struct QuadLoad;
template <>
struct QuadLoad<float> {
    static __device__ __forceinline__ float4 at(const void *q, int idx)
    {
        return __ldg(static_cast<const float4 *>(q) + idx);
    }
};
template <>
struct QuadLoad<__half> {
    static __device__ __forceinline__ float4 at(const void *q, int idx)
    {
        const uint2 raw = __ldg(static_cast<const uint2 *>(q) + idx);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&raw.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&raw.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};
template <>
struct QuadLoad<__nv_bfloat16> {
    static __device__ __forceinline__ float4 at(const void *q, int idx)
    {
        const uint2 raw = __ldg(static_cast<const uint2 *>(q) + idx);
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};

// Pairs per j-column and quads per i-row of a span block.
template <int P>
struct Block {
    static constexpr int JP = (P + 2) / 2;  // j pairs (the last one padded when P is even)
    static constexpr int IQ = (P + 2) / 2;  // quads along i
};

// Sum-factorised contraction of the (P+1)^3 control points under a span
// with the tensor-product basis:
//   f = sum N_i N_j N_k P_ijk,  f_u = sum N'_i N_j N_k P_ijk, f_v, f_w alike.
// pair(k, jp, i) yields (P(i, 2jp, k), P(i, 2jp+1, k)).  The u sums run on
// packed FP32 FMAs over j pairs (two rows per instruction), the v and w sums
// on scalar FMAs: 2(P+1)^3 + 3(P+1)^2 + 4(P+1) multiply-adds (the u sums
// carry a padded row when P is even).  r = {f, df/dx_u, df/dx_v, df/dx_w} in
// span-local units, times the product of the three basis scales.
template <int P, typename PairAt>
__device__ __forceinline__ void contract_pairs(const float Nu[P + 1], const float dNu[P + 1], const float Nv[P + 1],
                                               const float dNv[P + 1], const float Nw[P + 1], const float dNw[P + 1],
                                               PairAt pair, float r[4])
{
    constexpr int JP = Block<P>::JP;
    float f = 0.f, fu = 0.f, fv = 0.f, fw = 0.f;
#pragma unroll
    for (int k = 0; k <= P; ++k) {
        float c = 0.f, dv = 0.f, e = 0.f;
#pragma unroll
        for (int jp = 0; jp < JP; ++jp) {
            float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i <= P; ++i) {
                const float2 pv = pair(k, jp, i);
                a = __ffma2_rn(make_float2(Nu[i], Nu[i]), pv, a);
                b = __ffma2_rn(make_float2(dNu[i], dNu[i]), pv, b);
            }
            // v sums on scalar FMAs: no pair halves to add afterwards
            c = fmaf(Nv[2 * jp], a.x, c);
            dv = fmaf(dNv[2 * jp], a.x, dv);
            e = fmaf(Nv[2 * jp], b.x, e);
            if (2 * jp + 1 <= P) {
                c = fmaf(Nv[2 * jp + 1], a.y, c);
                dv = fmaf(dNv[2 * jp + 1], a.y, dv);
                e = fmaf(Nv[2 * jp + 1], b.y, e);
            }
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

// Loads the quads of the span block whose first control point is quad index
// `base` (= i0 + n0*(j0 + n1*k0)) into q[k][jp][iq].
template <int P, typename T>
__device__ __forceinline__ void load_block(const void *quads, int base, int n0, int n01,
                                           float4 (&q)[P + 1][Block<P>::JP][Block<P>::IQ])
{
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
        for (int jp = 0; jp < Block<P>::JP; ++jp)
#pragma unroll
            for (int iq = 0; iq < Block<P>::IQ; ++iq)
                q[k][jp][iq] = QuadLoad<T>::at(quads, base + 2 * iq + 2 * jp * n0 + k * n01);
}

template <int P>
__device__ __forceinline__ float2 quad_pair(const float4 (&q)[P + 1][Block<P>::JP][Block<P>::IQ], int k, int jp,
                                            int i)
{
    const float4 v = q[k][jp][i >> 1];
    return (i & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
}

}  // namespace mfadvr
