// mfadvr_render: the ray caster of Algorithm 1 as one fused kernel, and its
// batched form over many images and models.  The kernel templates live here;
// render_p1.cu .. render_p5.cu instantiate one degree each (compiled in
// parallel) and render_kernels.cu picks the degree.
//
// Per pixel: ray definition (Sec. 3.1), slab test against the world box
// (Sample_First..Sample_Last), constant-distance samples, value and gradient
// query of the MFA model, transfer-function lookup (applyTFs), optional
// gradient shading (getLightingCoefficient / addShading), front-to-back
// compositing (doColorCompositing) and early ray termination once the
// cumulative opacity exceeds O_max.
//
// GPU mapping.  A persistent grid of warps takes 32-ray tiles (tile_w x
// 32/tile_w pixels) from a global counter; every lane owns one ray of the
// tile, and the warp takes its next tile once all 32 rays have ended (exit or
// early termination).  Neighbouring rays that start together cross span
// cells together, which keeps a warp's reloads few and shared; a lane whose
// ray ended early idles until the tile is done (about 3% of lane slots on
// the 128^3 frame, against 21% of the frame time saved).  Each
// lane walks its ray in lattice units (one FMA per axis per sample; parameter
// units on general knots), keeps the control points of its current span
// block in registers (FP32 pairs, or the stored 16-bit pairs) and reloads
// them (8 256-bit loads at degree 3 in FP32, 4 in 16 bits) only when a
// sample leaves the span.  One iteration contracts sample s while it
// composites sample s-1.  The contraction runs on packed FP32 FMAs.  Template
// flags: G (gradient queried: shading on), NU (general knots), R (rational).
//
// The batched kernel runs the same per-ray code over the concatenated tiles
// of many render jobs (one image of one model each).  A warp keeps its
// current job's model and settings in a shared-memory slot and moves to the
// next job's tiles only when all its lanes are idle.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mfa_basis.cuh"
#include "mfa_internal.h"

namespace mfadvr {
namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float clamp01f(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

// The span block is cached in registers up to degree 4; degree 5 (216
// values) and rational models (two blocks: w P and w) read it from the row
// arrays at every sample.
template <int P, bool R>
struct CacheCP {
    static constexpr bool value = R ? P <= 3 : P <= 4;
};

// Storage tag of the POWER render form: the lane caches its span cell's
// polynomial coefficients (FP32 pairs, PolyCell in mfa_basis.cuh) and
// evaluates them by Horner's rule; no basis per sample.
struct PolyF32 {};

// Resident CTAs per SM the compiler is asked to fit: four (16 warps, at
// most 128 registers a thread) up to degree 3, where the 64-value cache
// fits beside the ray state; three for an FP32 B-spline block on general
// knots, whose span bounds and widths take nine more registers (the power
// form, with no basis, fits four there: 4.82 -> 4.21 ms on graded knots, and
// so does the 16-bit block, 32 registers: 5.95 -> 5.42 ms in BF16); at
// degree 4 three for the 16-bit cache (75 registers; measured 41.6 against
// 49.1 ms per 512^3 frame at one) and one for the FP32 cache, which needs the
// whole register file of a thread; at degree 5 (no cache) three (about 4%
// faster than one); rational models keep two contractions in flight.
template <int P, typename T, bool NU, bool R>
struct MinBlocks {
    static constexpr bool kPoly = std::is_same<T, PolyF32>::value;
    static constexpr int value =
        R ? 2 : (P <= 3 ? (NU && !kPoly && sizeof(T) == 4 ? 3 : 4) : (!NU && (P == 5 || sizeof(T) == 2) ? 3 : 1));
};

// State of the ray a lane is marching.
struct LaneRay {
    int pix;
    float X0[3], dX[3], dir[3];  // sample s sits at lattice coordinates X0 + s dX
    float kf[3];                 // current span (local index) per axis, as float (power form on uniform
                                 // knots: the span's centre, index + 1/2)
    int kk[3];                   // the same as int
    float lo[3], hi[3], ih[3];   // general knots: span bounds and inverse width per axis
    int base;                    // row-entry index of the span block's first control point
    bool interior;               // all three spans unclamped: uniform pieces apply
    float sf, nsf;               // samples contracted / samples on the ray
    float Cr, Cg, Cb, A;         // premultiplied colour and opacity so far
    float r[4];                  // query of sample sf - 1, not yet composited
};

// Cached span block: FP32 pairs for FP32 storage; for 16-bit storage the
// stored pairs themselves (one 32-bit register each, half the registers),
// converted to FP32 as the contraction uses them.
template <typename T>
struct CacheElem {
    using type = float2;
    static constexpr bool kPacked = false;
};
template <>
struct CacheElem<__half> {
    using type = unsigned;
    static constexpr bool kPacked = true;
};
template <>
struct CacheElem<__nv_bfloat16> {
    using type = unsigned;
    static constexpr bool kPacked = true;
};

template <int P, typename T, bool R>
struct SpanCache {
    static constexpr bool kOn = CacheCP<P, R>::value;
    static constexpr int K = kOn ? P + 1 : 1, J = kOn ? Block<P>::JP : 1, KW = kOn && R ? P + 1 : 1;
    typename CacheElem<T>::type v[K][J][K];    // the block (rational models: w P)
    typename CacheElem<T>::type w[KW][J][KW];  // rational models: the weights' block
    template <typename E>
    static __device__ __forceinline__ float2 to_pair(E e)
    {
        if constexpr (CacheElem<T>::kPacked) return pair16_to_float2<T>(e);
        else return e;
    }
    __device__ __forceinline__ float2 pair(int k, int jp, int i) const { return to_pair(v[k][jp][i]); }
    __device__ __forceinline__ float2 wpair(int k, int jp, int i) const { return to_pair(w[k][jp][i]); }
};

// Pixel of ray slot `slot` (tile = slot / 32, lane-in-tile = slot % 32) for
// tiles of 2^tw_log2 x 32/2^tw_log2 pixels, tiles_x tiles per image row.
__device__ __forceinline__ void slot_pixel(int slot, int tiles_x, int tw_log2, int &px, int &py)
{
    const int tile = slot >> 5, l = slot & 31;
    const int th_log2 = 5 - tw_log2;
    px = ((tile % tiles_x) << tw_log2) + (l & ((1 << tw_log2) - 1));
    py = ((tile / tiles_x) << th_log2) + (l >> tw_log2);
}

// Ray of pixel (px, py): origin o, direction dir (unit length for a
// perspective camera) and the distance t0 at which it enters the world box;
// returns its sample count, floor((t1 - t0) / step) for the chord [t0, t1]
// inside the box, or 0 when it misses the box.
__device__ __forceinline__ float ray_chord(const RenderSetup &rs, int px, int py, float o[3], float dir[3],
                                           float &t0)
{
    const float sx = fmaf(rs.sx_scale, static_cast<float>(px) + 0.5f, rs.sx_off);
    const float sy = fmaf(rs.sy_scale, static_cast<float>(py) + 0.5f, rs.sy_off);
    if (rs.kind == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = fmaf(sy, rs.up[a], fmaf(sx, rs.right[a], rs.eye[a]));
            dir[a] = rs.fwd[a];
        }
    } else {
        float dd = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = rs.eye[a];
            dir[a] = fmaf(sy, rs.up[a], fmaf(sx, rs.right[a], rs.fwd[a]));
            dd = fmaf(dir[a], dir[a], dd);
        }
        const float inv = 1.0f / sqrtf(dd);
#pragma unroll
        for (int a = 0; a < 3; ++a) dir[a] *= inv;
    }
    // slab test: [t0, t1] inside the box, t0 >= 0
    t0 = 0.0f;
    float t1 = INFINITY;
    bool hit = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dir[a] == 0.0f) {
            if (o[a] < rs.box_min[a] || o[a] > rs.box_max[a]) hit = false;
        } else {
            float ta = (rs.box_min[a] - o[a]) / dir[a];
            float tb = (rs.box_max[a] - o[a]) / dir[a];
            if (ta > tb) { const float s = ta; ta = tb; tb = s; }
            t0 = fmaxf(t0, ta);
            t1 = fminf(t1, tb);
        }
    }
    return (hit && t1 > t0) ? floorf((t1 - t0) / rs.step) : 0.0f;
}

// Ray definition and slab test for pixel (px, py).  Returns true when the
// ray has samples; otherwise writes the empty pixel and returns false.
__device__ __forceinline__ bool start_ray(const RenderSetup &rs, int px, int py, LaneRay &ray)
{
    ray.pix = py * rs.width + px;
    float o[3], t0;
    ray.nsf = ray_chord(rs, px, py, o, ray.dir, t0);
    if (ray.nsf < 1.0f) {
        rs.out[ray.pix] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (rs.nsamples) rs.nsamples[ray.pix] = 0;
        return false;
    }
    const float tm = fmaf(0.5f, rs.step, t0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ray.X0[a] = (fmaf(tm, ray.dir[a], o[a]) - rs.box_min[a]) * rs.lat_scale[a];
        ray.dX[a] = rs.step * ray.dir[a] * rs.lat_scale[a];
        ray.kf[a] = -2.0f;  // forces a span lookup at the first sample
        ray.lo[a] = 2.0f;   // (general knots: an empty span)
        ray.hi[a] = -1.0f;
        ray.kk[a] = 0;
    }
    ray.sf = 0.f;
    ray.Cr = ray.Cg = ray.Cb = ray.A = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) ray.r[c] = 0.f;
    return true;
}

// Transfer-function lookups: `TfShared` reads (entry, next - entry) pairs the
// kernel staged in shared memory; `TfGlobal` reads two entries of the
// caller's table through the read-only cache.
struct TfShared {
    const float4 *t;
    __device__ __forceinline__ void at(int i, float4 &a, float4 &d) const
    {
        a = t[2 * i];
        d = t[2 * i + 1];
    }
};
struct TfGlobal {
    const float4 *t;
    __device__ __forceinline__ void at(int i, float4 &a, float4 &d) const
    {
        a = __ldg(t + i);
        const float4 b = __ldg(t + i + 1);
        d = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, b.w - a.w);
    }
};

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Loads the span block whose first row entry is `base` into the lane's cache
// (and, for a rational model, the weights' block).
template <int P, typename T, bool R>
__device__ __forceinline__ void reload_block(const ModelView &mv, int base, SpanCache<P, T, R> &cache)
{
    constexpr int JP = Block<P>::JP;
    typename Entries<P, T>::E q[P + 1][Entries<P, T>::JE][Block<P>::IR];
    load_block<P, T>(mv.rows, base, mv.n[0], mv.n01, q);
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
        for (int jp = 0; jp < JP; ++jp)
#pragma unroll
            for (int i = 0; i <= P; ++i) {
                if constexpr (CacheElem<T>::kPacked) cache.v[k][jp][i] = block_word<P, T>(q, k, jp, i);
                else cache.v[k][jp][i] = block_pair<P, T>(q, k, jp, i);
            }
    if constexpr (R) {
        load_block<P, T>(mv.wrows, base, mv.n[0], mv.n01, q);
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int jp = 0; jp < JP; ++jp)
#pragma unroll
                for (int i = 0; i <= P; ++i) {
                    if constexpr (CacheElem<T>::kPacked) cache.w[k][jp][i] = block_word<P, T>(q, k, jp, i);
                    else cache.w[k][jp][i] = block_pair<P, T>(q, k, jp, i);
                }
    }
}

// One iteration of the lane's ray, software-pipelined over two samples:
// the span bookkeeping (with a cache reload when the span changed), basis
// and contraction of sample sf, and the applyTFs, shading and compositing
// of sample sf - 1, whose query the previous iteration left in ray.r.  The
// two halves are independent, so the compiler interleaves the contraction's
// FMAs with the serial TF / shading / compositing chain.  Early termination
// is decided on the composited sample; the query of sample sf is then
// dropped, as is the one past the last sample.  G: the gradient is queried
// (shading on); without it the value-only contraction runs.  NU: general
// knots, the ray walked in parameter units; on a span change the axes that
// left their span take the neighbouring span when two compares confirm it,
// else a search of the span grid; the basis comes from the span's pieces.
// R: rational model, the value f = A / W and its gradient
// (grad A - f grad W) / W from the contractions of w P and of w.  Returns
// true when the ray is finished (pixel written).
// Render-path trace (a test facility): for each ray's first max_samples
// samples, the FP32 position the kernel walks (lattice units on uniform
// knots, parameter units on general knots) and the knot spans it contracts
// with, as written by TraceOn; TraceOff compiles to nothing.
struct TraceOff {};  // TraceOn: mfa_internal.h

// Which sample of its ray an iteration is at: the first (contract only: it
// has no predecessor to composite) or a later one.
enum StepMode { kStepFirst = 1, kStepLater = 2 };

template <int P, typename T, bool G, bool NU, bool R, int MODE, typename Tf, typename Tr = TraceOff>
__device__ __forceinline__ bool sample_step(const ModelView &mv, const RenderSetup &rs, const Tf &tf, LaneRay &ray,
                                            SpanCache<P, T, R> &cache, const Tr &tr = Tr{})
{
    constexpr bool kCache = SpanCache<P, T, R>::kOn;
    constexpr bool kPoly = std::is_same<T, PolyF32>::value;
    static_assert(!kPoly || (P <= 4 && G && kCache), "span polynomials: shaded renders, degree <= 4");
    const float s = ray.sf;

    // ---- span of sample s; positions are clamped to the lattice only when
    // the span changes (a sample outside [0, m] always leaves its span) ------
    float x[3];
    bool moved = false;
    // Power form on uniform knots: x is the offset from the span's centre
    // (index + 1/2), exact while the sample is in the span (|x| < 1/2: the
    // subtraction of the centre is exact there by Sterbenz's lemma), and the
    // Horner sums take it as it is.  A sample on the span's lower face
    // (x = -1/2) also counts as moved: the lookup below finds the same span.
    constexpr bool kCentred = kPoly && !NU;
    if constexpr (kCentred) {
        float amax = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            x[a] = fmaf(s, ray.dX[a], ray.X0[a]) - ray.kf[a];
            amax = fmaxf(amax, fabsf(x[a]));
        }
        moved = amax >= 0.5f;
    } else if constexpr (NU) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            x[a] = fmaf(s, ray.dX[a], ray.X0[a]);  // parameter u, turned local below
            moved |= (x[a] < ray.lo[a]) | (x[a] >= ray.hi[a]);
        }
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            x[a] = fmaf(s, ray.dX[a], ray.X0[a]) - ray.kf[a];
            moved |= (x[a] < 0.0f) | (x[a] >= 1.0f);
        }
    }
    if (moved) {
        if constexpr (NU) {
            // Only the axes whose span no longer holds x are resolved.  A
            // march leaves a span into its neighbour on that side, which two
            // exact compares confirm (breakpoints strictly increase, so the
            // span holding x is unique); anything else (a new ray, a skipped
            // narrow span) takes the grid search.
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                x[a] = clamp01f(x[a]);
                if (x[a] >= ray.lo[a] && x[a] < ray.hi[a]) continue;
                const int last = mv.m[a] - 1;
                int k = ray.kk[a] + (x[a] >= ray.hi[a] ? 1 : -1);
                k = min(max(k, 0), last);
                float lo = __ldg(mv.brk[a] + k), hi = __ldg(mv.brk[a] + k + 1);
                if (!(ray.lo[a] <= ray.hi[a] && lo <= x[a] && (x[a] < hi || k == last))) {
                    k = span_search(mv.brk[a], mv.cell[a], mv.grid[a], x[a]);
                    lo = __ldg(mv.brk[a] + k);
                    hi = __ldg(mv.brk[a] + k + 1);
                }
                ray.kk[a] = k;
                ray.lo[a] = lo;
                ray.hi[a] = hi;
                ray.ih[a] = __ldg(mv.ih[a] + k);
            }
        } else if constexpr (kCentred) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float mfa = static_cast<float>(mv.m[a]);
                const float X = fminf(fmaxf(fmaf(s, ray.dX[a], ray.X0[a]), 0.0f), mfa);
                // span floor(X) (the last one at X = m): an add rounded toward
                // -infinity gives 2^23 + floor(X) exactly for 0 <= X < 2^23;
                // the centre k + 1/2 = k23 - (2^23 - 1/2) is exact too (the
                // operands are within a factor 2: Sterbenz's lemma)
                const float k23 = fminf(__fadd_rd(X, 8388608.0f), 8388607.0f + mfa);
                ray.kk[a] = __float_as_int(k23) - 0x4B000000;
                ray.kf[a] = k23 - 8388607.5f;
                x[a] = X - ray.kf[a];
            }
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float mfa = static_cast<float>(mv.m[a]);
                const float X = fminf(fmaxf(fmaf(s, ray.dX[a], ray.X0[a]), 0.0f), mfa);
                ray.kf[a] = fminf(floorf(X), mfa - 1.0f);
                x[a] = X - ray.kf[a];
                ray.kk[a] = static_cast<int>(ray.kf[a]);
            }
        }
        if constexpr (kPoly) {
            // cells < 2^31: the lattice has fewer than 2^31 control points
            const int cell = ray.kk[0] + mv.m[0] * (ray.kk[1] + mv.m[1] * ray.kk[2]);
            load_poly<P>(mv.poly, cell, cache.v);
            if constexpr (R) load_poly<P>(mv.wpoly, cell, cache.w);
        } else {
            ray.base = ray.kk[0] + mv.n[0] * ray.kk[1] + mv.n01 * ray.kk[2];
            ray.interior = span_interior<P>(ray.kk[0], mv.m[0]) && span_interior<P>(ray.kk[1], mv.m[1]) &&
                           span_interior<P>(ray.kk[2], mv.m[2]);
            if constexpr (kCache) reload_block<P, T, R>(mv, ray.base, cache);
        }
    }
    if constexpr (std::is_same<Tr, TraceOn>::value) {
        const int k = static_cast<int>(s);
        if (k < tr.max_samples) {
            const int64_t at = (static_cast<int64_t>(ray.pix) * tr.max_samples + k) * 3;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                tr.pos[at + a] = fmaf(s, ray.dX[a], ray.X0[a]);
                tr.span[at + a] = ray.kk[a] + P;
            }
        }
    }
    float Nu[P + 1], dNu[P + 1], Nv[P + 1], dNv[P + 1], Nw[P + 1], dNw[P + 1];
    if constexpr (kPoly) {
        // no basis: the cell's polynomial is evaluated directly below, in the
        // span's local coordinates (general knots: from the span bounds; a
        // rounded multiply, so that no kernel fuses it with the centring and
        // batched and single renders agree bit for bit)
        if constexpr (NU) {
#pragma unroll
            for (int a = 0; a < 3; ++a) x[a] = __fmul_rn(x[a] - ray.lo[a], ray.ih[a]);
        }
    } else if constexpr (NU) {
        // local coordinate on the span, basis from the span's pieces
#pragma unroll
        for (int a = 0; a < 3; ++a) x[a] = (x[a] - ray.lo[a]) * ray.ih[a];
        basis_pieces<P>(x[0], mv.pieces[0], ray.kk[0], Nu, dNu);
        basis_pieces<P>(x[1], mv.pieces[1], ray.kk[1], Nv, dNv);
        basis_pieces<P>(x[2], mv.pieces[2], ray.kk[2], Nw, dNw);
    } else {
        // uniform pieces, replaced from the piece table on clamped spans;
        // the cubic's v and w bases share packed instructions
        basis_uniform_scaled<P>(x[0], Nu, dNu);
        if constexpr (P == 3) {
            float2 Nvw[4], dNvw[4];
            basis_cubic_pair(make_float2(x[1], x[2]), Nvw, dNvw);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                Nv[r] = Nvw[r].x;
                dNv[r] = dNvw[r].x;
                Nw[r] = Nvw[r].y;
                dNw[r] = dNvw[r].y;
            }
        } else {
            basis_uniform_scaled<P>(x[1], Nv, dNv);
            basis_uniform_scaled<P>(x[2], Nw, dNw);
        }
        if (!ray.interior) {
            if (!span_interior<P>(ray.kk[0], mv.m[0])) basis_table<P>(x[0], ray.kk[0], mv.m[0], Nu, dNu);
            if (!span_interior<P>(ray.kk[1], mv.m[1])) basis_table<P>(x[1], ray.kk[1], mv.m[1], Nv, dNv);
            if (!span_interior<P>(ray.kk[2], mv.m[2])) basis_table<P>(x[2], ray.kk[2], mv.m[2], Nw, dNw);
        }
    }

    // ---- applyTFs on sample s - 1: linear interpolation in the table -------
    if constexpr (MODE != kStepFirst) {
        const float r[4] = {ray.r[0], ray.r[1], ray.r[2], ray.r[3]};
        // Table coordinate xt in [0, N-1]; entry floor(xt), capped at N-2, and
        // the fraction past it.  The floor comes from one add rounded toward
        // -infinity (2^23 + floor(xt) exactly, for 0 <= xt < 2^23), whose bits
        // hold the integer; the subtraction of 2^23 is exact.  No conversion
        // instructions on the serial TF chain.
        const float xt = __saturatef(fmaf(r[0], rs.tf_a, rs.tf_b)) * static_cast<float>(rs.tf_size - 1);
        const float it23 = fminf(__fadd_rd(xt, 8388608.0f), 8388608.0f + static_cast<float>(rs.tf_size - 2));
        const int it = __float_as_int(it23) - 0x4B000000;
        const float fr = xt - (it23 - 8388608.0f);
        float4 ta, td;
        tf.at(it, ta, td);
        float cr = fmaf(fr, td.x, ta.x);
        float cg = fmaf(fr, td.y, ta.y);
        float cb = fmaf(fr, td.z, ta.z);
        float alpha = __saturatef(fmaf(fr, td.w, ta.w));
        const float corrected = 1.0f - ex2_approx(lg2_approx(1.0f - alpha) * rs.opacity_ratio);
        alpha = rs.correct_opacity ? corrected : alpha;

        // ---- shading: Blinn-Phong, headlight L = V = -d, two-sided -------------
        {
            const float gx = r[1] * rs.grad_scale[0];
            const float gy = r[2] * rs.grad_scale[1];
            const float gz = r[3] * rs.grad_scale[2];
            const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
            const float ndl = __saturatef(fabsf(fmaf(gx, ray.dir[0], fmaf(gy, ray.dir[1], gz * ray.dir[2]))) * rsqrtf(g2));
            // a flat gradient (|g| at or below the threshold) shades ambient-only,
            // unclamped: c ka; otherwise c (ka + kd ndl) + ks ndl^shininess,
            // clamped to [0, 1]
            const bool flat = g2 <= rs.gthresh2;
            const float spec = rs.ks * __powf(ndl, rs.shininess);
            const float diff = fmaf(rs.kd, ndl, rs.ka);
            if constexpr (G) {  // the gradient is queried exactly when shading is on
                cr = flat ? cr * rs.ka : __saturatef(fmaf(cr, diff, spec));
                cg = flat ? cg * rs.ka : __saturatef(fmaf(cg, diff, spec));
                cb = flat ? cb * rs.ka : __saturatef(fmaf(cb, diff, spec));
            }
        }

        // ---- front-to-back compositing of sample s - 1 -------------------------
        const float wgt = (1.0f - ray.A) * alpha;
        ray.Cr = fmaf(wgt, cr, ray.Cr);
        ray.Cg = fmaf(wgt, cg, ray.Cg);
        ray.Cb = fmaf(wgt, cb, ray.Cb);
        ray.A += wgt;
    }

    // ---- query of sample s (composited by the next iteration) -------------
    constexpr int Q = G ? kQueryBoth : kQueryValue;
    if constexpr (kCentred) {
        contract_poly<P>([&](int f) { return (&cache.v[0][0][0])[f]; }, x[0], x[1], x[2], ray.r);
    } else if constexpr (kPoly) {
        contract_poly<P>([&](int f) { return (&cache.v[0][0][0])[f]; }, x[0] - 0.5f, x[1] - 0.5f,
                         x[2] - 0.5f, ray.r);
    } else if constexpr (kCache) {
        contract<P, Q>(Nu, dNu, Nv, dNv, Nw, dNw, [&](int k, int jp, int i) { return cache.pair(k, jp, i); }, ray.r);
    } else {
        const int n0 = mv.n[0], n01 = mv.n01, base = ray.base;
        contract<P, Q>(Nu, dNu, Nv, dNv, Nw, dNw,
                       [&](int k, int jp, int i) { return row_pair<T>(mv.rows, base, n0, n01, k, jp, i); }, ray.r);
    }
    if constexpr (R) {
        {
            float rw[4];
            if constexpr (kCentred) {
                contract_poly<P>([&](int f) { return (&cache.w[0][0][0])[f]; }, x[0], x[1], x[2], rw);
            } else if constexpr (kPoly) {
                contract_poly<P>([&](int f) { return (&cache.w[0][0][0])[f]; }, x[0] - 0.5f, x[1] - 0.5f,
                                 x[2] - 0.5f, rw);
            } else if constexpr (kCache) {
                contract<P, Q>(Nu, dNu, Nv, dNv, Nw, dNw, [&](int k, int jp, int i) { return cache.wpair(k, jp, i); },
                               rw);
            } else {
                const int n0 = mv.n[0], n01 = mv.n01, base = ray.base;
                contract<P, Q>(Nu, dNu, Nv, dNv, Nw, dNw,
                               [&](int k, int jp, int i) { return row_pair<T>(mv.wrows, base, n0, n01, k, jp, i); },
                               rw);
            }
            // the basis scale cancels in A / W; the storage scales do not
            const float W = rw[0] * mv.wscale, f = (ray.r[0] * mv.scale) / W;
            if constexpr (G) {
#pragma unroll
                for (int d = 1; d < 4; ++d) ray.r[d] = (ray.r[d] * mv.scale - f * (rw[d] * mv.wscale)) / W;
            }
            ray.r[0] = f;
        }
    }
    if constexpr (NU && G) {
        // d/du = (1 / span width) d/dx, applied now: the next iteration may
        // change span before it shades this query
#pragma unroll
        for (int a = 0; a < 3; ++a) ray.r[a + 1] *= ray.ih[a];
    }
    ray.sf = s + 1.0f;

    // ---- early ray termination / end of the ray: s samples composited ------
    if constexpr (MODE == kStepFirst) return false;  // a ray has at least one sample
    if (ray.A > rs.max_opacity || s >= ray.nsf) {
        rs.out[ray.pix] = make_float4(ray.Cr, ray.Cg, ray.Cb, ray.A);
        if (rs.nsamples) rs.nsamples[ray.pix] = static_cast<int>(s);
        return true;
    }
    return false;
}

// ---------------------------------------------------------------------------
// One image
// ---------------------------------------------------------------------------
template <int P, typename T, bool G, bool NU, bool R, typename Tr = TraceOff>
__global__ void __launch_bounds__(kThreads, MinBlocks<P, T, NU, R>::value)
    render_kernel(ModelView mv, RenderSetup rs, int *__restrict__ counter, Tr tr)
{
    // transfer function as (entry, next entry - entry) pairs: one FMA per
    // channel interpolates
    extern __shared__ float4 s_tf[];
    for (int i = threadIdx.x; i < rs.tf_size; i += blockDim.x) {
        const float4 a = rs.tf[i];
        const float4 b = (i + 1 < rs.tf_size) ? rs.tf[i + 1] : a;
        s_tf[2 * i] = a;
        s_tf[2 * i + 1] = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, b.w - a.w);
    }
    __syncthreads();
    const TfShared tf{s_tf};

    const int lane = threadIdx.x & 31;
    const int tw_log2 = rs.tile_w_log2;
    const int tiles_x = (rs.width + (1 << tw_log2) - 1) >> tw_log2;
    const int tiles_y = (rs.height + (32 >> tw_log2) - 1) >> (5 - tw_log2);
    const int total = tiles_x * tiles_y * 32;  // ray slots, some outside the image

    LaneRay ray;
    SpanCache<P, T, R> cache;

    for (;;) {
        // ---- a wholly idle warp takes its next tile ------------------------
        // Lanes that march neighbouring rays from the same start change cells
        // together, so a warp's iteration touches half as many distinct cells
        // and a quarter of its iterations change none.  The first sample of
        // every ray is then contracted in one step of its own, and later
        // iterations carry no test for a missing predecessor.
        // Tiles are taken in the order rs.tile_order lists them (costliest
        // first, so that the last tiles of the frame are short ones), else
        // in row order.
        int b = 0;
        if (lane == 0) b = atomicAdd(counter, 32);
        b = __shfl_sync(kFull, b, 0);
        if (b >= total) break;
        if (rs.tile_order) b = __ldg(rs.tile_order + (b >> 5)) << 5;
        int px, py;
        slot_pixel(b + lane, tiles_x, tw_log2, px, py);
        bool active = px < rs.width && py < rs.height && start_ray(rs, px, py, ray);
        if (active) sample_step<P, T, G, NU, R, kStepFirst>(mv, rs, tf, ray, cache, tr);
        while (__any_sync(kFull, active)) {
            if (active && sample_step<P, T, G, NU, R, kStepLater>(mv, rs, tf, ray, cache, tr)) active = false;
        }
    }
}

// ---------------------------------------------------------------------------
// Many images (render jobs) of one degree and storage type
// ---------------------------------------------------------------------------
template <int P, typename T, bool G, bool NU, bool R>
__global__ void __launch_bounds__(kThreads, MinBlocks<P, T, NU, R>::value)
    render_batch_kernel(const RenderJob *__restrict__ jobs, int njobs, int total_tiles, int *__restrict__ counter,
                        const int *__restrict__ order)
{
    __shared__ RenderJob s_job[kWarps];  // the current job of each warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lane_lt = (1u << lane) - 1u;
    RenderJob &J = s_job[warp];

    int cur = -1;   // current job
    int held = -1;  // a fetched tile not yet handed out
    int pool_next = 0, pool_end = 0;
    bool exhausted = false;
    bool idle = true;
    LaneRay ray;
    SpanCache<P, T, R> cache;

    for (;;) {
        // as in render_kernel: rays are handed out only to a wholly idle warp
        const unsigned need = __ballot_sync(kFull, idle);
        if (need == kFull) {
            if (pool_next >= pool_end && held < 0 && !exhausted) {
                int t = 0;
                if (lane == 0) t = atomicAdd(counter, 1);
                t = __shfl_sync(kFull, t, 0);
                // tiles costliest first when `order` lists them, else in job order
                if (t >= total_tiles) exhausted = true;
                else held = order ? __ldg(order + t) : t;
            }
            if (held >= 0 && pool_next >= pool_end) {
                // the job owning the tile: jobs are sorted by tile_begin
                int j = 0;
                while (j + 1 < njobs && __ldg(&jobs[j + 1].tile_begin) <= held) ++j;
                if (j != cur && need == kFull) {
                    // all lanes idle: take the new job's model and settings
                    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(jobs + j);
                    unsigned long long *dst = reinterpret_cast<unsigned long long *>(&J);
                    for (int w = lane; w < static_cast<int>(sizeof(RenderJob) / 8); w += 32) dst[w] = src[w];
                    __syncwarp();
                    cur = j;
                }
                if (j == cur) {
                    pool_next = (held - J.tile_begin) * 32;
                    pool_end = pool_next + 32;
                    held = -1;
                }
            }
            const int avail = pool_end - pool_next;
            const int rank = __popc(need & lane_lt);
            if (idle && rank < avail) {
                int px, py;
                slot_pixel(pool_next + rank, J.tiles_x, J.rs.tile_w_log2, px, py);
                if (px < J.rs.width && py < J.rs.height) idle = !start_ray(J.rs, px, py, ray);
            }
            pool_next += min(avail, __popc(need));
            if (exhausted && held < 0 && __all_sync(kFull, idle)) break;
            // the rays just started contract their first sample in a step of
            // their own, as in render_kernel (multi16 FP32: 68.5 -> 66.8 ms)
            if (!idle) {
                const TfGlobal tf{J.rs.tf};
                sample_step<P, T, G, NU, R, kStepFirst>(J.mv, J.rs, tf, ray, cache);
            }
        }
        if (idle) continue;
        const TfGlobal tf{J.rs.tf};
        if (sample_step<P, T, G, NU, R, kStepLater>(J.mv, J.rs, tf, ray, cache)) idle = true;
    }
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

template <int P, typename T, bool G, bool NU, bool R, typename Tr = TraceOff>
cudaError_t launch_render_t(const ModelView &mv, const RenderSetup &rs, int *counter, cudaStream_t stream,
                            Tr tr = Tr{})
{
    const size_t smem = 2 * sizeof(float4) * static_cast<size_t>(rs.tf_size);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(render_kernel<P, T, G, NU, R, Tr>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_kernel<P, T, G, NU, R, Tr>, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (rs.ctas_per_sm > 0 && rs.ctas_per_sm < per_sm) per_sm = rs.ctas_per_sm;
    // no more warps than ray tiles
    const int tw = 1 << rs.tile_w_log2, th = 32 / tw;
    const int64_t tiles = static_cast<int64_t>((rs.width + tw - 1) / tw) * ((rs.height + th - 1) / th);
    int64_t blocks = static_cast<int64_t>(sm_count()) * per_sm;
    const int64_t need = (tiles + kWarps - 1) / kWarps;
    if (blocks > need) blocks = need;
    e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    if (rs.tile_order) {
        e = launch_tile_order(rs, (rs.width + tw - 1) / tw, static_cast<int>(tiles), stream);
        if (e != cudaSuccess) return e;
    }
    render_kernel<P, T, G, NU, R, Tr><<<static_cast<int>(blocks), kThreads, smem, stream>>>(mv, rs, counter, tr);
    return cudaGetLastError();
}

template <int P, typename T, bool G, bool NU, bool R>
cudaError_t launch_batch_t(const RenderJob *jobs, int njobs, int total_tiles, int ctas_per_sm, int *counter,
                           const int *order, cudaStream_t stream)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_batch_kernel<P, T, G, NU, R>, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    int64_t blocks = static_cast<int64_t>(sm_count()) * per_sm;
    const int64_t need = (static_cast<int64_t>(total_tiles) + kWarps - 1) / kWarps;
    if (blocks > need) blocks = need;
    if (blocks < 1) return cudaSuccess;
    e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    render_batch_kernel<P, T, G, NU, R><<<static_cast<int>(blocks), kThreads, 0, stream>>>(jobs, njobs, total_tiles, counter, order);
    return cudaGetLastError();
}

template <int P, typename T, bool G, bool NU, bool R>
struct RenderOne {
    static cudaError_t run(const ModelView *mv, const RenderSetup *rs, int *counter, cudaStream_t s)
    {
        return launch_render_t<P, T, G, NU, R>(*mv, *rs, counter, s);
    }
};
// The traced render: FP32 models (either render form, uniform or general
// knots, plain), shading on; other kinds are not compiled for it.
template <int P, typename T, bool G, bool NU, bool R>
struct RenderTrace {
    static cudaError_t run(const ModelView *mv, const RenderSetup *rs, int *counter, TraceOn tr, cudaStream_t s)
    {
        if constexpr (G && !R && (std::is_same<T, PolyF32>::value || std::is_same<T, float>::value))
            return launch_render_t<P, T, G, NU, R, TraceOn>(*mv, *rs, counter, s, tr);
        else
            return cudaErrorNotSupported;
    }
};
template <int P, typename T, bool G, bool NU, bool R>
struct RenderBatch {
    static cudaError_t run(const RenderJob *jobs, int njobs, int total_tiles, int ctas_per_sm, int *counter,
                           const int *order, cudaStream_t s)
    {
        return launch_batch_t<P, T, G, NU, R>(jobs, njobs, total_tiles, ctas_per_sm, counter, order, s);
    }
};

// Calls F<P, T, G, NU, R>::run for a fixed degree P and the model's storage
// type, whether the gradient is queried, whether the knots are general and
// whether the model is rational.
template <int P, typename TT, template <int, typename, bool, bool, bool> class F, typename... A>
cudaError_t dispatch_flags(bool grad, bool nu, bool rat, A... args)
{
    const int k = (grad ? 4 : 0) | (nu ? 2 : 0) | (rat ? 1 : 0);
    switch (k) {
    case 0: return F<P, TT, false, false, false>::run(args...);
    case 1: return F<P, TT, false, false, true>::run(args...);
    case 2: return F<P, TT, false, true, false>::run(args...);
    case 3: return F<P, TT, false, true, true>::run(args...);
    case 4: return F<P, TT, true, false, false>::run(args...);
    case 5: return F<P, TT, true, false, true>::run(args...);
    case 6: return F<P, TT, true, true, false>::run(args...);
    default: return F<P, TT, true, true, true>::run(args...);
    }
}

template <int P, template <int, typename, bool, bool, bool> class F, typename... A>
cudaError_t dispatch_degree(int dtype, bool grad, bool nu, bool rat, A... args)
{
    switch (dtype) {
    case kPolyForm:
        // span polynomials exist only for FP32 models of degree <= 3, and for
        // plain ones of degree 4
        if constexpr (P == 4) {
            if (!grad || rat) return cudaErrorInvalidValue;
            return nu ? F<P, PolyF32, true, true, false>::run(args...) : F<P, PolyF32, true, false, false>::run(args...);
        } else if constexpr (P <= 3) {
            if (!grad) return cudaErrorInvalidValue;
            const int k = (nu ? 2 : 0) | (rat ? 1 : 0);
            switch (k) {
            case 0: return F<P, PolyF32, true, false, false>::run(args...);
            case 1: return F<P, PolyF32, true, false, true>::run(args...);
            case 2: return F<P, PolyF32, true, true, false>::run(args...);
            default: return F<P, PolyF32, true, true, true>::run(args...);
            }
        } else {
            return cudaErrorInvalidValue;
        }
    case MFADVR_F32: return dispatch_flags<P, float, F>(grad, nu, rat, args...);
    case MFADVR_F16: return dispatch_flags<P, __half, F>(grad, nu, rat, args...);
    case MFADVR_BF16: return dispatch_flags<P, __nv_bfloat16, F>(grad, nu, rat, args...);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// The per-degree launchers one render_pN.cu defines.
#define MFADVR_RENDER_DEGREE(PP)                                                                             \
    cudaError_t launch_render_p##PP(const ModelView &mv, const RenderSetup &rs, int *counter,                 \
                                    cudaStream_t stream)                                                     \
    {                                                                                                        \
        return dispatch_degree<PP, RenderOne>(render_form_key(mv, rs.shading), rs.shading != 0, mv.nu != 0,  \
                                               mv.rational != 0, &mv, &rs, counter, stream);                 \
    }                                                                                                        \
    cudaError_t launch_render_trace_p##PP(const ModelView &mv, const RenderSetup &rs, int *counter,           \
                                          const TraceOn &tr, cudaStream_t stream)                             \
    {                                                                                                        \
        return dispatch_degree<PP, RenderTrace>(render_form_key(mv, rs.shading), rs.shading != 0, mv.nu != 0, \
                                                 mv.rational != 0, &mv, &rs, counter, tr, stream);           \
    }                                                                                                        \
    cudaError_t launch_render_batch_p##PP(int dtype, int grad, int nu, int rat, const RenderJob *jobs_dev,     \
                                          int njobs, int total_tiles, int ctas_per_sm, int *counter,           \
                                          const int *order, cudaStream_t stream)                             \
    {                                                                                                        \
        return dispatch_degree<PP, RenderBatch>(dtype, grad != 0, nu != 0, rat != 0, jobs_dev, njobs,         \
                                                 total_tiles, ctas_per_sm, counter, order, stream);          \
    }

cudaError_t launch_render_p1(const ModelView &, const RenderSetup &, int *, cudaStream_t);
cudaError_t launch_render_p2(const ModelView &, const RenderSetup &, int *, cudaStream_t);
cudaError_t launch_render_p3(const ModelView &, const RenderSetup &, int *, cudaStream_t);
cudaError_t launch_render_p4(const ModelView &, const RenderSetup &, int *, cudaStream_t);
cudaError_t launch_render_p5(const ModelView &, const RenderSetup &, int *, cudaStream_t);
cudaError_t launch_render_trace_p1(const ModelView &, const RenderSetup &, int *, const TraceOn &, cudaStream_t);
cudaError_t launch_render_trace_p2(const ModelView &, const RenderSetup &, int *, const TraceOn &, cudaStream_t);
cudaError_t launch_render_trace_p3(const ModelView &, const RenderSetup &, int *, const TraceOn &, cudaStream_t);
cudaError_t launch_render_trace_p4(const ModelView &, const RenderSetup &, int *, const TraceOn &, cudaStream_t);
cudaError_t launch_render_trace_p5(const ModelView &, const RenderSetup &, int *, const TraceOn &, cudaStream_t);
cudaError_t launch_render_batch_p1(int, int, int, int, const RenderJob *, int, int, int, int *, const int *,
                                   cudaStream_t);
cudaError_t launch_render_batch_p2(int, int, int, int, const RenderJob *, int, int, int, int *, const int *,
                                   cudaStream_t);
cudaError_t launch_render_batch_p3(int, int, int, int, const RenderJob *, int, int, int, int *, const int *,
                                   cudaStream_t);
cudaError_t launch_render_batch_p4(int, int, int, int, const RenderJob *, int, int, int, int *, const int *,
                                   cudaStream_t);
cudaError_t launch_render_batch_p5(int, int, int, int, const RenderJob *, int, int, int, int *, const int *,
                                   cudaStream_t);

}  // namespace mfadvr
