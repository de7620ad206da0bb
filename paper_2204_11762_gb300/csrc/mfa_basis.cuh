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

#include <type_traits>

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

// The cubic closed form (times 6) on a pair of local coordinates, two axes
// per packed instruction.
__device__ __forceinline__ void basis_cubic_pair(float2 x, float2 N[4], float2 dN[4])
{
    const float2 t = x, s = __fadd2_rn(make_float2(1.f, 1.f), make_float2(-x.x, -x.y));
    const float2 t2 = __fmul2_rn(t, t), s2 = __fmul2_rn(s, s);
    N[0] = __fmul2_rn(s2, s);
    N[1] = __ffma2_rn(t2, __ffma2_rn(make_float2(3.f, 3.f), t, make_float2(-6.f, -6.f)), make_float2(4.f, 4.f));
    N[2] = __ffma2_rn(s2, __ffma2_rn(make_float2(3.f, 3.f), s, make_float2(-6.f, -6.f)), make_float2(4.f, 4.f));
    N[3] = __fmul2_rn(t2, t);
    dN[0] = __fmul2_rn(make_float2(-3.f, -3.f), s2);
    dN[1] = __fmul2_rn(t, __ffma2_rn(make_float2(9.f, 9.f), t, make_float2(-12.f, -12.f)));
    dN[2] = __fmul2_rn(make_float2(-s.x, -s.y), __ffma2_rn(make_float2(9.f, 9.f), s, make_float2(-12.f, -12.f)));
    dN[3] = __fmul2_rn(make_float2(3.f, 3.f), t2);
}

// ---------------------------------------------------------------------------
// Pieces on every span.  The span-local knots kappa(j), j = 1-P..P, depend on
// the span only through how close it is to the two clamped ends:
//   a = max(0, P-1-k) knots cut off on the left  (kappa(j) >= -(P-1-a)),
//   b = max(0, k+P-m) knots cut off on the right (kappa(j) <= P-b),
// so P x P knot patterns cover all spans of all lattices, pattern (0, 0)
// being the uniform one.  Each pattern's P+1 basis functions are fixed
// polynomials of the local coordinate; their monomial coefficients come from
// the Cox-de Boor recurrence run on polynomials at compile time, with the
// convention 0/0 = 0 for the empty supports of the clamped ends.
// ---------------------------------------------------------------------------
template <int P>
struct SpanPieces {
    float c[P * P][P + 1][P + 1];  // pattern a*P + b: BasisScale<P> N_r(x) = sum_e c[.][r][e] x^e
};

// Monomial coefficients of the P+1 basis functions on one span, from the
// Cox-de Boor recurrence run on polynomials of the local coordinate x in
// [0, 1].  kap[j + P - 1] is the span-local position of knot t_{s+j},
// j = 1-P..P, in units of the span width (so kap(0) = 0, kap(1) = 1); the
// convention 0/0 = 0 covers repeated end knots.  out[r][e] = scale * coefficient
// of x^e in N_{s-P+r}.  Runs at compile time (the pattern tables below) and
// on the host at model load (per-span tables of general knots).
template <int P>
constexpr void pieces_from_knots(const double (&kap)[2 * P], double scale, double (&out)[P + 1][P + 1])
{
    double B[P + 1][P + 1][P + 1] = {};  // [q][r][e]: N_{s-q+r, q}
    B[0][0][0] = 1.0;
    for (int q = 1; q <= P; ++q) {
        for (int r = 0; r <= q; ++r) {
            const int i = r - q;
            if (r > 0) {  // (x - kappa(i)) / (kappa(i+q) - kappa(i)) N_{s+i, q-1}
                const double k0 = kap[i + P - 1], den = kap[i + q + P - 1] - k0;
                if (den != 0.0)
                    for (int e = 0; e < q; ++e) {
                        B[q][r][e + 1] += B[q - 1][r - 1][e] / den;
                        B[q][r][e] -= k0 * B[q - 1][r - 1][e] / den;
                    }
            }
            if (r < q) {  // (kappa(i+q+1) - x) / (kappa(i+q+1) - kappa(i+1)) N_{s+i+1, q-1}
                const double k1 = kap[i + q + P], den = k1 - kap[i + P];
                if (den != 0.0)
                    for (int e = 0; e < q; ++e) {
                        B[q][r][e] += k1 * B[q - 1][r][e] / den;
                        B[q][r][e + 1] -= B[q - 1][r][e] / den;
                    }
            }
        }
    }
    for (int r = 0; r <= P; ++r)
        for (int e = 0; e <= P; ++e) out[r][e] = scale * B[P][r][e];
}

template <int P>
constexpr SpanPieces<P> make_span_pieces(double scale)
{
    SpanPieces<P> out{};
    for (int a = 0; a < P; ++a) {
        for (int b = 0; b < P; ++b) {
            double kap[2 * P] = {};  // kap[j + P - 1] = kappa(j)
            for (int j = 1 - P; j <= P; ++j) {
                int v = j < -(P - 1 - a) ? -(P - 1 - a) : j;
                kap[j + P - 1] = v > P - b ? P - b : v;
            }
            double c[P + 1][P + 1] = {};
            pieces_from_knots<P>(kap, scale, c);
            for (int r = 0; r <= P; ++r)
                for (int e = 0; e <= P; ++e) out.c[a * P + b][r][e] = static_cast<float>(c[r][e]);
        }
    }
    return out;
}

// Compile-time pins of the tables: pattern (0, 0) is the uniform pieces, and
// every pattern sums to BasisScale<P> (partition of unity: the constant term
// sums to the scale, higher terms cancel).
template <int P>
constexpr bool span_pieces_consistent(double scale)
{
    constexpr UniformPieces<P> U = make_uniform_pieces<P>();
    const SpanPieces<P> S = make_span_pieces<P>(scale);
    for (int r = 0; r <= P; ++r)
        for (int e = 0; e <= P; ++e) {
            const double d = S.c[0][r][e] - scale * U.c[r][e];
            if (d > 1e-6 || d < -1e-6) return false;
        }
    for (int pat = 0; pat < P * P; ++pat)
        for (int e = 0; e <= P; ++e) {
            double sum = 0.0;
            for (int r = 0; r <= P; ++r) sum += S.c[pat][r][e];
            const double want = e == 0 ? scale : 0.0;
            if (sum - want > 1e-5 || sum - want < -1e-5) return false;
        }
    return true;
}

struct AllSpanPieces {
    SpanPieces<1> p1;
    SpanPieces<2> p2;
    SpanPieces<3> p3;
    SpanPieces<4> p4;
    SpanPieces<5> p5;
};
static_assert(span_pieces_consistent<1>(1.0) && span_pieces_consistent<2>(1.0) && span_pieces_consistent<3>(6.0) &&
                  span_pieces_consistent<4>(1.0) && span_pieces_consistent<5>(1.0),
              "span piece tables disagree with the uniform pieces or the partition of unity");

static __constant__ AllSpanPieces kSpanPieces = {
    make_span_pieces<1>(BasisScale<1>::value), make_span_pieces<2>(BasisScale<2>::value),
    make_span_pieces<3>(BasisScale<3>::value), make_span_pieces<4>(BasisScale<4>::value),
    make_span_pieces<5>(BasisScale<5>::value)};

template <int P>
__device__ __forceinline__ const SpanPieces<P> &span_pieces()
{
    if constexpr (P == 1) return kSpanPieces.p1;
    else if constexpr (P == 2) return kSpanPieces.p2;
    else if constexpr (P == 3) return kSpanPieces.p3;
    else if constexpr (P == 4) return kSpanPieces.p4;
    else return kSpanPieces.p5;
}

// Basis (times BasisScale<P>) and local derivative on span k of an axis
// with m spans, from the piece table of the span's knot pattern: Horner's
// rule for the value and its derivative together.
template <int P>
__device__ __forceinline__ void basis_table(float x, int k, int m, float N[P + 1], float dN[P + 1])
{
    const int a = max(0, P - 1 - k), b = max(0, k + P - m);
    const float(&c)[P + 1][P + 1] = span_pieces<P>().c[a * P + b];
#pragma unroll
    for (int r = 0; r <= P; ++r) {
        float v = c[r][P], d = 0.0f;
#pragma unroll
        for (int e = P - 1; e >= 0; --e) {
            d = fmaf(d, x, v);
            v = fmaf(v, x, c[r][e]);
        }
        N[r] = v;
        dN[r] = d;
    }
}

// True when span k of an axis with m spans has unclamped knots
// (p-1 <= k <= m-p), i.e. the uniform pieces apply.
template <int P>
__device__ __forceinline__ bool span_interior(int k, int m)
{
    return k >= P - 1 && k <= m - P;
}

// Basis on span k of an axis with m spans, times BasisScale<P>: the uniform
// closed form on unclamped spans, the piece table otherwise.
template <int P>
__device__ __forceinline__ void basis(float x, int k, int m, float N[P + 1], float dN[P + 1])
{
    if (span_interior<P>(k, m)) basis_uniform_scaled<P>(x, N, dN);
    else basis_table<P>(x, k, m, N, dN);
}

// ---------------------------------------------------------------------------
// General (non-uniform) clamped knots.  Per axis the model holds the m+1
// span breakpoints b_k = t_{p+k}, the inverse widths 1/(b_{k+1} - b_k), a
// lookup grid of G+1 cells (G = 2m; cell c holds the span containing c/G)
// and, per span, the monomial coefficients of its P+1 basis functions in the
// local coordinate x = (u - b_k) / (b_{k+1} - b_k), times BasisScale<P>,
// each span's block padded to a multiple of 8 floats (one 32-byte sector per
// 8 coefficients).
// ---------------------------------------------------------------------------
template <int P>
struct GeneralPieces {
    static constexpr int kStride = ((P + 1) * (P + 1) + 7) / 8 * 8;  // floats per span
};

// Span k in [lo, hi] with b_k <= u < b_{k+1}, given b_lo <= u: binary search,
// exact FP32 compares, at most ceil(log2(hi - lo + 1)) steps.
__device__ __forceinline__ int span_bisect(const float *__restrict__ brk, int lo, int hi, float u)
{
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(brk + mid) <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Span of FP32 u in [0, 1] (u = 1 in the last span) through the lookup grid.
// With c* = floor(u G) the span lies in [cell[c*], cell[c*+1]]; the FP32
// product u G can round across one integer, so [cell[c-1], cell[c+2]] is
// searched, which holds that range whichever way it rounded.
__device__ __forceinline__ int span_search(const float *__restrict__ brk, const int *__restrict__ cell, int G,
                                           float u)
{
    const int c = min(static_cast<int>(u * static_cast<float>(G)), G);
    const int lo = __ldg(cell + max(c - 1, 0)), hi = __ldg(cell + min(c + 2, G));
    return span_bisect(brk, lo, hi, u);
}

// Basis (times BasisScale<P>) and derivative with respect to the local
// coordinate on span k, from the span's pieces: Horner's rule for the value
// and its derivative together.
template <int P>
__device__ __forceinline__ void basis_pieces(float x, const float *__restrict__ pieces, int k, float N[P + 1],
                                             float dN[P + 1])
{
    constexpr int S = GeneralPieces<P>::kStride;
    float c[S];
    const float *src = pieces + static_cast<int64_t>(k) * S;
#pragma unroll
    for (int q = 0; q < S / 8; ++q)
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(c[8 * q]), "=f"(c[8 * q + 1]), "=f"(c[8 * q + 2]), "=f"(c[8 * q + 3]), "=f"(c[8 * q + 4]),
              "=f"(c[8 * q + 5]), "=f"(c[8 * q + 6]), "=f"(c[8 * q + 7])
            : "l"(src + 8 * q));
#pragma unroll
    for (int r = 0; r <= P; ++r) {
        float v = c[r * (P + 1) + P], d = 0.0f;
#pragma unroll
        for (int e = P - 1; e >= 0; --e) {
            d = fmaf(d, x, v);
            v = fmaf(v, x, c[r * (P + 1) + e]);
        }
        N[r] = v;
        dN[r] = d;
    }
}

// ---------------------------------------------------------------------------
// Second derivatives (the Hessian query): basis values, first and second
// derivatives with respect to the local coordinate, times BasisScale<P>.
// ---------------------------------------------------------------------------

// Horner's rule for a polynomial sum_e c(e) x^e and its first two derivatives.
template <int P, typename Coef>
__device__ __forceinline__ void horner_d2(float x, Coef c, float &v, float &d1, float &d2)
{
    v = c(P);
    d1 = 0.0f;
    d2 = 0.0f;
#pragma unroll
    for (int e = P - 1; e >= 0; --e) {
        d2 = fmaf(d2, x, 2.0f * d1);
        d1 = fmaf(d1, x, v);
        v = fmaf(v, x, c(e));
    }
}

// Uniform pieces: the cubic closed form differentiated once more
// (6N0'' = 6s, 6N1'' = 18t - 12, 6N2'' = 18s - 12, 6N3'' = 6t), Horner on
// the compile-time pieces for the other degrees.
template <int P>
__device__ __forceinline__ void basis_uniform_d2(float x, float N[P + 1], float dN[P + 1], float d2N[P + 1])
{
    if constexpr (P == 3) {
        basis_uniform_scaled<3>(x, N, dN);
        const float t = x, s = 1.0f - x;
        d2N[0] = 6.0f * s;
        d2N[1] = fmaf(18.0f, t, -12.0f);
        d2N[2] = fmaf(18.0f, s, -12.0f);
        d2N[3] = 6.0f * t;
    } else {
        constexpr UniformPieces<P> U = make_uniform_pieces<P>();
#pragma unroll
        for (int r = 0; r <= P; ++r) horner_d2<P>(x, [&](int e) { return U.c[r][e]; }, N[r], dN[r], d2N[r]);
    }
}

// Any span of uniform knots: the closed form inside, the clamped-pattern
// table near the ends.
template <int P>
__device__ __forceinline__ void basis_d2(float x, int k, int m, float N[P + 1], float dN[P + 1], float d2N[P + 1])
{
    if (span_interior<P>(k, m)) {
        basis_uniform_d2<P>(x, N, dN, d2N);
    } else {
        const int a = max(0, P - 1 - k), b = max(0, k + P - m);
        const float(&c)[P + 1][P + 1] = span_pieces<P>().c[a * P + b];
#pragma unroll
        for (int r = 0; r <= P; ++r) horner_d2<P>(x, [&](int e) { return c[r][e]; }, N[r], dN[r], d2N[r]);
    }
}

// General knots: from the span's pieces.
template <int P>
__device__ __forceinline__ void basis_pieces_d2(float x, const float *__restrict__ pieces, int k, float N[P + 1],
                                                float dN[P + 1], float d2N[P + 1])
{
    constexpr int S = GeneralPieces<P>::kStride;
    const float *src = pieces + static_cast<int64_t>(k) * S;
#pragma unroll
    for (int r = 0; r <= P; ++r)
        horner_d2<P>(x, [&](int e) { return __ldg(src + r * (P + 1) + e); }, N[r], dN[r], d2N[r]);
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
// Row layout of the control points.  Every entry is 32 bytes (one L2 sector,
// one 256-bit load) and holds the pairs (P(i+d, j+2h, k), P(i+d, j+2h+1, k)),
// zero where i+d or j+2h+1 runs past the lattice:
//  - FP32: entry (i, j, k) holds d = 0..3, h = 0 (4 x 2 points);
//  - FP16/BF16: entry (i, j, k) holds d = 0..3, h = 0..1 (4 x 4 points),
//    word (d + 4h) the 16-bit pair.
// A k-slice of the block under a span is ceil((p+1)/4) entries along i by
// ceil((p+1)/2) (FP32) or ceil((p+1)/4) (16-bit) along j, and every entry
// yields pairs ready for packed FMAs: 8 loads per degree-3 block in FP32, 4
// in 16 bits.
// ---------------------------------------------------------------------------
struct Row {
    float2 p[4];
};
struct Row16 {
    unsigned w[8];
};

// The 256-bit row and span-cell loads do not allocate in L1: a lane keeps
// what it loads in registers, and only a fraction of the loads would hit L1
// again (the power-form render: 1.856 -> 1.794 ms per default frame; the point
// query: 0.508 -> 0.499 ms for 2^24 points).  row32c_at is the cached load,
// for the degree-4 cells (608 bytes, about 2.4 samples each on the 512^3
// frame), which neighbouring lanes do re-read from L1 (28.7 -> 30.2 ms per
// frame without it).
__device__ __forceinline__ Row row32_at(const void *rows, int idx)
{
    const float *a = static_cast<const float *>(rows) + 8 * static_cast<int64_t>(idx);
    Row r;
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(r.p[0].x), "=f"(r.p[0].y), "=f"(r.p[1].x), "=f"(r.p[1].y), "=f"(r.p[2].x), "=f"(r.p[2].y),
          "=f"(r.p[3].x), "=f"(r.p[3].y)
        : "l"(a));
    return r;
}

__device__ __forceinline__ Row row32c_at(const void *rows, int idx)
{
    const float *a = static_cast<const float *>(rows) + 8 * static_cast<int64_t>(idx);
    Row r;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(r.p[0].x), "=f"(r.p[0].y), "=f"(r.p[1].x), "=f"(r.p[1].y), "=f"(r.p[2].x), "=f"(r.p[2].y),
          "=f"(r.p[3].x), "=f"(r.p[3].y)
        : "l"(a));
    return r;
}

__device__ __forceinline__ Row16 row16_at(const void *rows, int idx)
{
    const unsigned *a = static_cast<const unsigned *>(rows) + 8 * static_cast<int64_t>(idx);
    Row16 r;
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]), "=r"(r.w[4]), "=r"(r.w[5]), "=r"(r.w[6]),
          "=r"(r.w[7])
        : "l"(a));
    return r;
}

// The FP32 pair of a stored 16-bit pair.
template <typename T>
__device__ __forceinline__ float2 pair16_to_float2(unsigned w);
template <>
__device__ __forceinline__ float2 pair16_to_float2<__half>(unsigned w)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}
template <>
__device__ __forceinline__ float2 pair16_to_float2<__nv_bfloat16>(unsigned w)
{
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
}

// Pairs per j-column and row entries per i-run of a span block.
template <int P>
struct Block {
    static constexpr int JP = (P + 2) / 2;  // j pairs (the last one padded when P is even)
    static constexpr int IR = (P + 4) / 4;  // row entries along i
};

// Entry geometry of the storage type: j pairs per entry and entries along j.
template <int P, typename T>
struct Entries {
    static constexpr bool k16 = sizeof(T) == 2;
    static constexpr int JPE = k16 ? 2 : 1;                          // j pairs per entry
    static constexpr int JE = (Block<P>::JP + JPE - 1) / JPE;        // entries along j
    using E = typename std::conditional<k16, Row16, Row>::type;
};

// Index of the entry holding pair (k, jp, i) of the block at entry `base`,
// and the pair's place in it.
template <typename T>
__device__ __forceinline__ int entry_of(int base, int n0, int n01, int k, int jp, int i)
{
    return sizeof(T) == 2 ? base + (i & ~3) + 4 * (jp >> 1) * n0 + k * n01 : base + (i & ~3) + 2 * jp * n0 + k * n01;
}

// What a query computes: bit 0 the value f, bit 1 the gradient (mfadvr_query).
constexpr int kQueryValue = 1, kQueryGradient = 2, kQueryBoth = 3;
// The Hessian query: value, gradient and the six second partial derivatives.
constexpr int kQueryHessian = 4;

// Multiply-adds of contract<P, Q>: value only (p+1)^3 + (p+1)^2 + (p+1);
// gradient only 2(p+1)^3 + 3(p+1)^2 + 3(p+1); both 2(p+1)^3 + 3(p+1)^2 + 4(p+1).
constexpr int contract_fma(int p, int q)
{
    const int a = p + 1;
    return q == kQueryValue ? a * a * a + a * a + a
                            : (q == kQueryGradient ? 2 * a * a * a + 3 * a * a + 3 * a : 2 * a * a * a + 3 * a * a + 4 * a);
}

static_assert(contract_fma(3, kQueryBoth) == 192 && contract_fma(4, kQueryBoth) == 345 &&
                  contract_fma(3, kQueryValue) == 84 && contract_fma(3, kQueryGradient) == 188,
              "multiply-add counts of the contraction");

// Sum-factorised contraction of the (P+1)^3 control points under a span
// with the tensor-product basis:
//   f = sum N_i N_j N_k P_ijk,  f_u = sum N'_i N_j N_k P_ijk, f_v, f_w alike.
// pair(k, jp, i) yields (P(i, 2jp, k), P(i, 2jp+1, k)).  The u sums run on
// packed FP32 FMAs over j pairs (two rows per instruction), the v and w sums
// on scalar FMAs; Q selects the value, the gradient or both, and only the
// sums those need are formed (contract_fma counts them; the u sums carry a
// padded row when P is even).  r = {f, df/dx_u, df/dx_v, df/dx_w} in
// span-local units, times the product of the three basis scales; entries Q
// does not ask for are left unset.
template <int P, int Q, typename PairAt>
__device__ __forceinline__ void contract(const float Nu[P + 1], const float dNu[P + 1], const float Nv[P + 1],
                                         const float dNv[P + 1], const float Nw[P + 1], const float dNw[P + 1],
                                         PairAt pair, float r[4])
{
    constexpr int JP = Block<P>::JP;
    constexpr bool kV = (Q & kQueryValue) != 0, kG = (Q & kQueryGradient) != 0;
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
                if constexpr (kG) b = __ffma2_rn(make_float2(dNu[i], dNu[i]), pv, b);
            }
            // v sums on scalar FMAs: no pair halves to add afterwards
            c = fmaf(Nv[2 * jp], a.x, c);
            if constexpr (kG) {
                dv = fmaf(dNv[2 * jp], a.x, dv);
                e = fmaf(Nv[2 * jp], b.x, e);
            }
            if (2 * jp + 1 <= P) {
                c = fmaf(Nv[2 * jp + 1], a.y, c);
                if constexpr (kG) {
                    dv = fmaf(dNv[2 * jp + 1], a.y, dv);
                    e = fmaf(Nv[2 * jp + 1], b.y, e);
                }
            }
        }
        if constexpr (kV) f = fmaf(Nw[k], c, f);
        if constexpr (kG) {
            fw = fmaf(dNw[k], c, fw);
            fv = fmaf(Nw[k], dv, fv);
            fu = fmaf(Nw[k], e, fu);
        }
    }
    if constexpr (kV) r[0] = f;
    if constexpr (kG) {
        r[1] = fu;
        r[2] = fv;
        r[3] = fw;
    }
}

// ---------------------------------------------------------------------------
// Span polynomials (the POWER render form).  On span cell (i, j, k) the model
// is a polynomial of the cell's local coordinates; with t = x - 1/2 per axis
// (the offset from the cell centre),
//   BasisScale^3 f = sum_{a,b,c} A[a][b][c] tu^a tv^b tw^c,
//   A[a][b][c] = sum_{r,s,q} Cu[r][a] Cv[s][b] Cw[q][c] P(i+r, j+s, k+q),
// where C[r][e] is the coefficient of t^e in BasisScale N_r on the span: the
// span's pieces (pieces_from_knots on its knots, uniform or general), shifted
// to the centre.  A cell stores the pairs (A[a][b][2g], A[a][b][2g+1]) (two
// tw powers) in the order [g][b][a], the last g padded with 0 when P is even,
// in whole 32-byte sectors: the order of the render kernel's span cache,
// whose flat pair index is (g (P+1) + b) (P+1) + a.  Pairing along tw lets
// both the tu and the tv Horner levels run on packed FMAs.
// ---------------------------------------------------------------------------
template <int P>
struct PolyCell {
    static constexpr int JP = Block<P>::JP;
    static constexpr int kPairs = (P + 1) * JP * (P + 1);
    static constexpr int kSectors = (kPairs + 3) / 4;
};
static_assert(PolyCell<1>::kSectors * 32 == poly_cell_bytes(1) && PolyCell<2>::kSectors * 32 == poly_cell_bytes(2) &&
                  PolyCell<3>::kSectors * 32 == poly_cell_bytes(3) && PolyCell<4>::kSectors * 32 == poly_cell_bytes(4),
              "span-polynomial cell sizes of host and device differ");

// Loads span cell `cell` of the polynomial array into the lane's cache, pair
// f of the cell to flat element f of v (PolyCell).
template <int P>
__device__ __forceinline__ void load_poly(const float *poly, int64_t cell, float2 (&v)[P + 1][Block<P>::JP][P + 1])
{
    constexpr int S = PolyCell<P>::kSectors, JP = Block<P>::JP;
    const float *base = poly + cell * (8 * S);
    Row q[S];
#pragma unroll
    for (int k = 0; k < S; ++k) q[k] = P >= 4 ? row32c_at(base, k) : row32_at(base, k);
#pragma unroll
    for (int f = 0; f < PolyCell<P>::kPairs; ++f) v[f / (JP * (P + 1))][(f / (P + 1)) % JP][f % (P + 1)] = q[f / 4].p[f % 4];
}

// Value and local gradient (times BasisScale^3, like contract<P, kQueryBoth>)
// of a span cell's polynomial at centred coordinates (tu, tv, tw) in
// [-1/2, 1/2]: per pair of tw powers, Horner's rule in tu on the coefficient
// pairs, then in tv, both on packed FMAs; then, per tw power, in tw.  Each
// level carries the derivative sums the gradient needs (for p(t) = sum A_e
// t^e, the recurrences p <- p t + A_e and d <- d t + p give p and p').
// pair(f) is the cache's flat pair f = (g (P+1) + b) (P+1) + a.  At degree 3:
// 56 packed and 11 scalar multiply-adds.
template <int P, typename PairAt>
__device__ __forceinline__ void contract_poly(PairAt pair, float tu, float tv, float tw, float r[4])
{
    constexpr int K = P + 1, CP = Block<P>::JP;
    const float2 uu = make_float2(tu, tu), vv = make_float2(tv, tv);
    float Fv[2 * CP], Fu[2 * CP], Fvv[2 * CP];  // per tw power: value, d/du and d/dv of the (u, v) polynomial
#pragma unroll
    for (int g = 0; g < CP; ++g) {
        float2 pv[K], pu[K];
#pragma unroll
        for (int b = 0; b < K; ++b) {
            float2 p = pair((g * K + b) * K + P), d = p;
#pragma unroll
            for (int a = P - 1; a >= 0; --a) {
                if (a < P - 1) d = __ffma2_rn(d, uu, p);
                p = __ffma2_rn(p, uu, pair((g * K + b) * K + a));
            }
            pv[b] = p;
            pu[b] = d;
        }
        float2 q = pv[P], qv = q, qu = pu[P];
#pragma unroll
        for (int b = P - 1; b >= 0; --b) {
            if (b < P - 1) qv = __ffma2_rn(qv, vv, q);
            qu = __ffma2_rn(qu, vv, pu[b]);
            q = __ffma2_rn(q, vv, pv[b]);
        }
        Fv[2 * g] = q.x;
        Fv[2 * g + 1] = q.y;
        Fvv[2 * g] = qv.x;
        Fvv[2 * g + 1] = qv.y;
        Fu[2 * g] = qu.x;
        Fu[2 * g + 1] = qu.y;
    }
    float f = Fv[P], fw = f, fv = Fvv[P], fu = Fu[P];
#pragma unroll
    for (int c = P - 1; c >= 0; --c) {
        if (c < P - 1) fw = fmaf(fw, tw, f);
        fv = fmaf(fv, tw, Fvv[c]);
        fu = fmaf(fu, tw, Fu[c]);
        f = fmaf(f, tw, Fv[c]);
    }
    r[0] = f;
    r[1] = fu;
    r[2] = fv;
    r[3] = fw;
}

// Derivative orders (u, v, w) of the ten outputs of the Hessian query:
// f, f_u, f_v, f_w, f_uu, f_vv, f_ww, f_uv, f_uw, f_vw.
__device__ __forceinline__ constexpr int hessian_order(int o, int axis)
{
    constexpr int ord[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                                {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
    return ord[o][axis];
}

// Sum-factorised contraction for the Hessian query: the u sums for orders
// 0..2 on packed FMAs, the v sums for the six order pairs of total <= 2, the
// w sums for the ten outputs.  N*[order][r]; r[o] in span-local units times
// the product of the basis scales.  Multiply-adds: 3(P+1)^3 + 6(P+1)^2 +
// 10(P+1) (u sums over padded j pairs when P is even).
template <int P, typename PairAt>
__device__ __forceinline__ void contract_hessian(const float (&Nu)[3][P + 1], const float (&Nv)[3][P + 1],
                                                 const float (&Nw)[3][P + 1], PairAt pair, float r[10])
{
    constexpr int JP = Block<P>::JP;
    float acc[10];
#pragma unroll
    for (int o = 0; o < 10; ++o) acc[o] = 0.0f;
#pragma unroll
    for (int k = 0; k <= P; ++k) {
        float c[3][3];  // c[ou][ov], ou + ov <= 2
#pragma unroll
        for (int ou = 0; ou < 3; ++ou)
#pragma unroll
            for (int ov = 0; ov < 3; ++ov) c[ou][ov] = 0.0f;
#pragma unroll
        for (int jp = 0; jp < JP; ++jp) {
            float2 a[3];
#pragma unroll
            for (int ou = 0; ou < 3; ++ou) a[ou] = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i <= P; ++i) {
                const float2 pv = pair(k, jp, i);
#pragma unroll
                for (int ou = 0; ou < 3; ++ou) a[ou] = __ffma2_rn(make_float2(Nu[ou][i], Nu[ou][i]), pv, a[ou]);
            }
#pragma unroll
            for (int ou = 0; ou < 3; ++ou)
#pragma unroll
                for (int ov = 0; ov + ou < 3; ++ov) {
                    c[ou][ov] = fmaf(Nv[ov][2 * jp], a[ou].x, c[ou][ov]);
                    if (2 * jp + 1 <= P) c[ou][ov] = fmaf(Nv[ov][2 * jp + 1], a[ou].y, c[ou][ov]);
                }
        }
#pragma unroll
        for (int o = 0; o < 10; ++o)
            acc[o] = fmaf(Nw[hessian_order(o, 2)][k], c[hessian_order(o, 0)][hessian_order(o, 1)], acc[o]);
    }
#pragma unroll
    for (int o = 0; o < 10; ++o) r[o] = acc[o];
}

// Loads the entries of the span block whose first control point is entry
// index `base` (= i0 + n0*(j0 + n1*k0)) into q[k][je][ir].
template <int P, typename T>
__device__ __forceinline__ void load_block(const void *rows, int base, int n0, int n01,
                                           typename Entries<P, T>::E (&q)[P + 1][Entries<P, T>::JE][Block<P>::IR])
{
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
        for (int je = 0; je < Entries<P, T>::JE; ++je)
#pragma unroll
            for (int ir = 0; ir < Block<P>::IR; ++ir) {
                const int idx = base + 4 * ir + 2 * Entries<P, T>::JPE * je * n0 + k * n01;
                if constexpr (Entries<P, T>::k16) q[k][je][ir] = row16_at(rows, idx);
                else q[k][je][ir] = row32_at(rows, idx);
            }
}

// The stored word of pair (k, jp, i) in a loaded 16-bit block.
template <int P, typename T>
__device__ __forceinline__ unsigned block_word(const Row16 (&q)[P + 1][Entries<P, T>::JE][Block<P>::IR], int k,
                                               int jp, int i)
{
    return q[k][jp >> 1][i >> 2].w[(i & 3) + 4 * (jp & 1)];
}

// Pair (P(i0+i, j0+2jp, k0+k), P(i0+i, j0+2jp+1, k0+k)) of a loaded block, in FP32.
template <int P, typename T>
__device__ __forceinline__ float2 block_pair(
    const typename Entries<P, T>::E (&q)[P + 1][Entries<P, T>::JE][Block<P>::IR], int k, int jp, int i)
{
    if constexpr (Entries<P, T>::k16) return pair16_to_float2<T>(block_word<P, T>(q, k, jp, i));
    else return q[k][jp][i >> 2].p[i & 3];
}

// The same pair read from the row array directly (no block in registers).
template <typename T>
__device__ __forceinline__ float2 row_pair(const void *rows, int base, int n0, int n01, int k, int jp, int i)
{
    const int idx = entry_of<T>(base, n0, n01, k, jp, i);
    if constexpr (sizeof(T) == 2) return pair16_to_float2<T>(row16_at(rows, idx).w[(i & 3) + 4 * (jp & 1)]);
    else return row32_at(rows, idx).p[i & 3];
}

}  // namespace mfadvr
