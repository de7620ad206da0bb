// mfadvr_render: the ray caster of Algorithm 1 as one fused kernel.
//
// Per pixel: ray definition (Sec. 3.1), slab test against the world box
// (Sample_First..Sample_Last), constant-distance samples, value and gradient
// query of the MFA model, transfer-function lookup (applyTFs), optional
// gradient shading (getLightingCoefficient / addShading), front-to-back
// compositing (doColorCompositing) and early ray termination once the
// cumulative opacity exceeds O_max.
//
// GPU mapping.  A persistent grid of warps takes 8x4-pixel ray tiles from a
// global counter; every lane owns one ray and, when its ray ends (exit or
// early termination), takes the next ray of the warp's tile pool, so lanes
// stay busy however unequal the ray lengths are.  Each lane walks its ray in
// lattice units (one FMA per axis per sample), keeps the control points of
// its current span block in registers and reloads them (ceil((p+1)/2)^2 x
// (p+1) vector loads from the quad array) only when a sample leaves the
// span.  The contraction runs on packed FP32 FMAs; the transfer function
// sits in shared memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mfa_basis.cuh"
#include "mfa_internal.h"

namespace mfadvr {
namespace {

constexpr int kThreads = 128;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float clamp01f(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

// The span block is cached in registers up to degree 4; degree 5 (216
// values) reads it from the quad array at every sample.
template <int P>
struct CacheCP {
    static constexpr bool value = P <= 4;
};

// Resident CTAs per SM the compiler is asked to fit: four (16 warps, at
// most 128 registers a thread) up to degree 3, where the 64-value cache
// fits beside the ray state; the degree-4 cache needs the whole register
// file of a thread.
template <int P>
struct MinBlocks {
    static constexpr int value = P <= 3 ? 4 : 1;
};

template <int P, typename T>
__global__ void __launch_bounds__(kThreads, MinBlocks<P>::value)
    render_kernel(ModelView mv, RenderSetup rs, int *__restrict__ counter)
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

    constexpr int JP = Block<P>::JP;
    constexpr bool kCache = CacheCP<P>::value;
    const int lane = threadIdx.x & 31;
    const unsigned lane_lt = (1u << lane) - 1u;
    const int tiles_x = (rs.width + 7) >> 3;
    const int total = tiles_x * ((rs.height + 3) >> 2) * 32;  // ray slots, some outside the image
    const float mf[3] = {static_cast<float>(mv.m[0]), static_cast<float>(mv.m[1]), static_cast<float>(mv.m[2])};
    const float tf_last = static_cast<float>(rs.tf_size - 1);

    int pool_next = 0, pool_end = 0;
    bool exhausted = false;
    bool idle = true;

    // state of the lane's ray
    int pix = 0;
    float X0[3], dX[3], dir[3];
    float kf[3];
    int kk[3];
    int base = 0;
    bool interior = false;  // all three spans unclamped: uniform pieces apply
    float sf = 0.f, nsf = 0.f;
    float Cr = 0.f, Cg = 0.f, Cb = 0.f, A = 0.f;
    float2 cache[kCache ? (P + 1) : 1][kCache ? JP : 1][kCache ? (P + 1) : 1];

    for (;;) {
        // ---- hand rays to idle lanes ------------------------------------
        const unsigned need = __ballot_sync(kFull, idle);
        if (need) {
            if (pool_next >= pool_end && !exhausted) {
                int b = 0;
                if (lane == 0) b = atomicAdd(counter, 32);
                b = __shfl_sync(kFull, b, 0);
                if (b >= total) exhausted = true;
                else { pool_next = b; pool_end = b + 32; }
            }
            const int avail = pool_end - pool_next;
            const int rank = __popc(need & lane_lt);
            if (idle && rank < avail) {
                const int slot = pool_next + rank;
                const int tile = slot >> 5, l = slot & 31;
                const int px = (tile % tiles_x) * 8 + (l & 7);
                const int py = (tile / tiles_x) * 4 + (l >> 3);
                if (px < rs.width && py < rs.height) {
                    pix = py * rs.width + px;
                    // ray definition
                    const float sx = fmaf(rs.sx_scale, static_cast<float>(px) + 0.5f, rs.sx_off);
                    const float sy = fmaf(rs.sy_scale, static_cast<float>(py) + 0.5f, rs.sy_off);
                    float o[3];
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
                    float t0 = 0.0f, t1 = INFINITY;
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
                    nsf = (hit && t1 > t0) ? floorf((t1 - t0) / rs.step) : 0.0f;
                    if (nsf >= 1.0f) {
                        // sample s sits at lattice coordinates X0 + s * dX
                        const float tm = fmaf(0.5f, rs.step, t0);
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            X0[a] = (fmaf(tm, dir[a], o[a]) - rs.box_min[a]) * rs.lat_scale[a];
                            dX[a] = rs.step * dir[a] * rs.lat_scale[a];
                            kf[a] = -2.0f;  // forces a span lookup at the first sample
                        }
                        sf = 0.f;
                        Cr = Cg = Cb = A = 0.f;
                        idle = false;
                    } else {
                        rs.out[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (rs.nsamples) rs.nsamples[pix] = 0;
                    }
                }
            }
            pool_next += min(avail, __popc(need));
            if (exhausted && __all_sync(kFull, idle)) break;
        }
        if (idle) continue;

        // ---- one sample -------------------------------------------------
        float X[3], x[3];
        bool moved = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            X[a] = fminf(fmaxf(fmaf(sf, dX[a], X0[a]), 0.0f), mf[a]);
            x[a] = X[a] - kf[a];
            moved |= (x[a] < 0.0f) | (x[a] >= 1.0f);
        }
        if (moved) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                kf[a] = fminf(floorf(X[a]), mf[a] - 1.0f);
                x[a] = X[a] - kf[a];
                kk[a] = static_cast<int>(kf[a]);
            }
            base = kk[0] + mv.n[0] * kk[1] + mv.n01 * kk[2];
            interior = span_interior<P>(kk[0], mv.m[0]) && span_interior<P>(kk[1], mv.m[1]) &&
                       span_interior<P>(kk[2], mv.m[2]);
            if constexpr (kCache) {
                float4 q[P + 1][JP][Block<P>::IQ];
                load_block<P, T>(mv.quads, base, mv.n[0], mv.n01, q);
#pragma unroll
                for (int k = 0; k <= P; ++k)
#pragma unroll
                    for (int jp = 0; jp < JP; ++jp)
#pragma unroll
                        for (int i = 0; i <= P; ++i) cache[k][jp][i] = quad_pair<P>(q, k, jp, i);
            }
        }
        float Nu[P + 1], dNu[P + 1], Nv[P + 1], dNv[P + 1], Nw[P + 1], dNw[P + 1];
        if (interior) {
            basis_uniform_scaled<P>(x[0], Nu, dNu);
            basis_uniform_scaled<P>(x[1], Nv, dNv);
            basis_uniform_scaled<P>(x[2], Nw, dNw);
        } else {
            basis<P>(x[0], kk[0], mv.m[0], Nu, dNu);
            basis<P>(x[1], kk[1], mv.m[1], Nv, dNv);
            basis<P>(x[2], kk[2], mv.m[2], Nw, dNw);
        }
        float r[4];
        if constexpr (kCache) {
            contract_pairs<P>(Nu, dNu, Nv, dNv, Nw, dNw, [&](int k, int jp, int i) { return cache[k][jp][i]; }, r);
        } else {
            const int n0 = mv.n[0], n01 = mv.n01;
            contract_pairs<P>(Nu, dNu, Nv, dNv, Nw, dNw,
                              [&](int k, int jp, int i) {
                                  const float4 qv = QuadLoad<T>::at(mv.quads, base + (i & ~1) + 2 * jp * n0 + k * n01);
                                  return (i & 1) ? make_float2(qv.z, qv.w) : make_float2(qv.x, qv.y);
                              },
                              r);
        }

        // ---- applyTFs: linear interpolation in the table ---------------
        const float xt = fminf(fmaxf(fmaf(r[0], rs.tf_a, rs.tf_b), 0.0f), tf_last);
        const int it = min(static_cast<int>(xt), rs.tf_size - 2);
        const float fr = xt - static_cast<float>(it);
        const float4 ta = s_tf[2 * it], td = s_tf[2 * it + 1];
        float cr = fmaf(fr, td.x, ta.x);
        float cg = fmaf(fr, td.y, ta.y);
        float cb = fmaf(fr, td.z, ta.z);
        float alpha = clamp01f(fmaf(fr, td.w, ta.w));
        if (rs.correct_opacity) alpha = 1.0f - exp2f(log2f(1.0f - alpha) * rs.opacity_ratio);

        // ---- shading: Blinn-Phong, headlight L = V = -d, two-sided -----
        if (rs.shading) {
            const float gx = r[1] * rs.grad_scale[0];
            const float gy = r[2] * rs.grad_scale[1];
            const float gz = r[3] * rs.grad_scale[2];
            const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
            if (g2 <= rs.gthresh2) {
                cr *= rs.ka; cg *= rs.ka; cb *= rs.ka;
            } else {
                const float ndl =
                    fminf(fabsf(fmaf(gx, dir[0], fmaf(gy, dir[1], gz * dir[2]))) * rsqrtf(g2), 1.0f);
                const float spec = rs.ks * __powf(ndl, rs.shininess);
                const float diff = fmaf(rs.kd, ndl, rs.ka);
                cr = clamp01f(fmaf(cr, diff, spec));
                cg = clamp01f(fmaf(cg, diff, spec));
                cb = clamp01f(fmaf(cb, diff, spec));
            }
        }

        // ---- front-to-back compositing + early ray termination ----------
        const float wgt = (1.0f - A) * alpha;
        Cr = fmaf(wgt, cr, Cr);
        Cg = fmaf(wgt, cg, Cg);
        Cb = fmaf(wgt, cb, Cb);
        A += wgt;
        sf += 1.0f;
        if (A > rs.max_opacity || sf >= nsf) {
            rs.out[pix] = make_float4(Cr, Cg, Cb, A);
            if (rs.nsamples) rs.nsamples[pix] = static_cast<int>(sf);
            idle = true;
        }
    }
}

template <int P, typename T>
cudaError_t launch_render_t(const ModelView &mv, const RenderSetup &rs, int *counter, cudaStream_t stream)
{
    const size_t smem = 2 * sizeof(float4) * static_cast<size_t>(rs.tf_size);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(render_kernel<P, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_kernel<P, T>, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    // no more warps than ray tiles
    const int64_t tiles = static_cast<int64_t>((rs.width + 7) / 8) * ((rs.height + 3) / 4);
    int64_t blocks = static_cast<int64_t>(sms) * per_sm;
    const int64_t need = (tiles + (kThreads / 32) - 1) / (kThreads / 32);
    if (blocks > need) blocks = need;
    e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    render_kernel<P, T><<<static_cast<int>(blocks), kThreads, smem, stream>>>(mv, rs, counter);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_render_dtype(const ModelView &mv, const RenderSetup &rs, int *counter, cudaStream_t stream)
{
    switch (mv.p) {
    case 1: return launch_render_t<1, T>(mv, rs, counter, stream);
    case 2: return launch_render_t<2, T>(mv, rs, counter, stream);
    case 3: return launch_render_t<3, T>(mv, rs, counter, stream);
    case 4: return launch_render_t<4, T>(mv, rs, counter, stream);
    case 5: return launch_render_t<5, T>(mv, rs, counter, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_render(const ModelView &mv, const RenderSetup &rs, int *counter, cudaStream_t stream)
{
    switch (mv.dtype) {
    case MFADVR_F32: return launch_render_dtype<float>(mv, rs, counter, stream);
    case MFADVR_F16: return launch_render_dtype<__half>(mv, rs, counter, stream);
    case MFADVR_BF16: return launch_render_dtype<__nv_bfloat16>(mv, rs, counter, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mfadvr
