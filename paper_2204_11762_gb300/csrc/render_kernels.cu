// mfadvr_render: the ray caster of Algorithm 1 as one fused kernel.
//
// Per pixel: ray definition (Sec. 3.1), slab test against the world box
// (Sample_First..Sample_Last), constant-distance samples, value and gradient
// query of the MFA model, transfer-function lookup (applyTFs), optional
// gradient shading (getLightingCoefficient / addShading), front-to-back
// compositing (doColorCompositing) and early ray termination once the
// cumulative opacity exceeds O_max.
//
// GPU mapping: one thread per ray, a warp per 8x4 pixel tile, a CTA per
// 16x8 tile.  The control points of the current span triple are held in
// registers and reloaded only when a sample leaves that span, so the
// per-sample work is the basis evaluation and the (P+1)^3 contraction on
// the FP32 FMA pipe.  The transfer function sits in shared memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mfa_basis.cuh"
#include "mfa_internal.h"

namespace mfadvr {
namespace {

constexpr int kTileW = 16, kTileH = 8, kThreads = 128;

__device__ __forceinline__ float clamp01f(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

// Control points cached in registers for degrees up to 4; degree 5 reads
// them per sample (216 values do not fit the register file of one thread).
template <int P>
struct CacheCP {
    static constexpr bool value = P <= 4;
};

template <int P, typename T>
__global__ void __launch_bounds__(kThreads) render_kernel(ModelView mv, RenderSetup rs)
{
    extern __shared__ float4 s_tf[];
    for (int i = threadIdx.x; i < rs.tf_size; i += blockDim.x) s_tf[i] = rs.tf[i];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px = blockIdx.x * kTileW + (warp & 1) * 8 + (lane & 7);
    const int py = blockIdx.y * kTileH + (warp >> 1) * 4 + (lane >> 3);
    if (px >= rs.width || py >= rs.height) return;

    // ---- ray definition -------------------------------------------------
    const float sx = fmaf(rs.sx_scale, static_cast<float>(px) + 0.5f, rs.sx_off);
    const float sy = fmaf(rs.sy_scale, static_cast<float>(py) + 0.5f, rs.sy_off);
    float o[3], d[3];
    if (rs.kind == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = fmaf(sy, rs.up[a], fmaf(sx, rs.right[a], rs.eye[a]));
            d[a] = rs.fwd[a];
        }
    } else {
        float dd = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = rs.eye[a];
            d[a] = fmaf(sy, rs.up[a], fmaf(sx, rs.right[a], rs.fwd[a]));
            dd = fmaf(d[a], d[a], dd);
        }
        const float inv = 1.0f / sqrtf(dd);
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] *= inv;
    }

    // ---- slab test: [t0, t1] inside the box, t0 >= 0 --------------------
    float t0 = 0.0f, t1 = INFINITY;
    bool hit = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0f) {
            if (o[a] < rs.box_min[a] || o[a] > rs.box_max[a]) hit = false;
        } else {
            float ta = (rs.box_min[a] - o[a]) / d[a];
            float tb = (rs.box_max[a] - o[a]) / d[a];
            if (ta > tb) { const float s = ta; ta = tb; tb = s; }
            t0 = fmaxf(t0, ta);
            t1 = fminf(t1, tb);
        }
    }
    int nsteps = 0;
    if (hit && t1 > t0) {
        const float nf = floorf((t1 - t0) / rs.step);
        nsteps = nf >= 2.0e9f ? 2000000000 : static_cast<int>(nf);
    }

    // ---- march ----------------------------------------------------------
    const T *__restrict__ cp = static_cast<const T *>(mv.cp);
    const int64_t sj = mv.n[0];
    const int64_t sk = static_cast<int64_t>(mv.n[0]) * mv.n[1];
    const float mf[3] = {static_cast<float>(mv.m[0]), static_cast<float>(mv.m[1]), static_cast<float>(mv.m[2])};
    constexpr int NC = (P + 1) * (P + 1) * (P + 1);
    constexpr bool kCache = CacheCP<P>::value;
    float cache[kCache ? NC : 1];
    int cur0 = -1, cur1 = -1, cur2 = -1;

    float Cr = 0.f, Cg = 0.f, Cb = 0.f, A = 0.f;
    const float tf_last = static_cast<float>(rs.tf_size - 1);
    int s = 0;
    for (; s < nsteps; ++s) {
        const float t = fmaf(static_cast<float>(s) + 0.5f, rs.step, t0);
        float x[3];
        int k[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float q = clamp01f((fmaf(t, d[a], o[a]) - rs.box_min[a]) * rs.inv_ext[a]);
            const float xm = q * mf[a];
            k[a] = min(static_cast<int>(xm), mv.m[a] - 1);
            x[a] = xm - static_cast<float>(k[a]);
        }
        const T *base = cp + (k[0] + sj * k[1] + sk * k[2]);
        if constexpr (kCache) {
            if (k[0] != cur0 || k[1] != cur1 || k[2] != cur2) {
                cur0 = k[0]; cur1 = k[1]; cur2 = k[2];
#pragma unroll
                for (int kk = 0; kk <= P; ++kk)
#pragma unroll
                    for (int jj = 0; jj <= P; ++jj)
#pragma unroll
                        for (int ii = 0; ii <= P; ++ii)
                            cache[(kk * (P + 1) + jj) * (P + 1) + ii] = load_cp<T>(base + ii + sj * jj + sk * kk);
            }
        }
        float Nu[P + 1], dNu[P + 1], Nv[P + 1], dNv[P + 1], Nw[P + 1], dNw[P + 1];
        basis<P>(x[0], k[0], mv.m[0], Nu, dNu);
        basis<P>(x[1], k[1], mv.m[1], Nv, dNv);
        basis<P>(x[2], k[2], mv.m[2], Nw, dNw);
        float r[4];
        if constexpr (kCache)
            contract<P>(Nu, dNu, Nv, dNv, Nw, dNw,
                        [&](int i, int j, int kk) { return cache[(kk * (P + 1) + j) * (P + 1) + i]; }, r);
        else
            contract<P>(Nu, dNu, Nv, dNv, Nw, dNw,
                        [&](int i, int j, int kk) { return load_cp<T>(base + i + sj * j + sk * kk); }, r);

        // ---- applyTFs: linear interpolation in the table ---------------
        const float v = r[0] * mv.scale;
        const float xt = clamp01f((v - rs.tf_lo) * rs.tf_inv_range) * tf_last;
        const int it = min(static_cast<int>(xt), rs.tf_size - 2);
        const float fr = xt - static_cast<float>(it);
        const float4 ta = s_tf[it], tb = s_tf[it + 1];
        float cr = fmaf(fr, tb.x - ta.x, ta.x);
        float cg = fmaf(fr, tb.y - ta.y, ta.y);
        float cb = fmaf(fr, tb.z - ta.z, ta.z);
        float alpha = clamp01f(fmaf(fr, tb.w - ta.w, ta.w));
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
                const float ndl = fminf(fabsf(fmaf(gx, d[0], fmaf(gy, d[1], gz * d[2]))) * rsqrtf(g2), 1.0f);
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
        if (A > rs.max_opacity) { ++s; break; }
    }
    const size_t pix = static_cast<size_t>(py) * rs.width + px;
    rs.out[pix] = make_float4(Cr, Cg, Cb, A);
    if (rs.nsamples) rs.nsamples[pix] = s;
}

template <int P, typename T>
cudaError_t launch_render_t(const ModelView &mv, const RenderSetup &rs, cudaStream_t stream)
{
    const size_t smem = sizeof(float4) * static_cast<size_t>(rs.tf_size);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(render_kernel<P, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    dim3 grid((rs.width + kTileW - 1) / kTileW, (rs.height + kTileH - 1) / kTileH);
    render_kernel<P, T><<<grid, kThreads, smem, stream>>>(mv, rs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_render_dtype(const ModelView &mv, const RenderSetup &rs, cudaStream_t stream)
{
    switch (mv.p) {
    case 1: return launch_render_t<1, T>(mv, rs, stream);
    case 2: return launch_render_t<2, T>(mv, rs, stream);
    case 3: return launch_render_t<3, T>(mv, rs, stream);
    case 4: return launch_render_t<4, T>(mv, rs, stream);
    case 5: return launch_render_t<5, T>(mv, rs, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_render(const ModelView &mv, const RenderSetup &rs, cudaStream_t stream)
{
    switch (mv.dtype) {
    case MFADVR_F32: return launch_render_dtype<float>(mv, rs, stream);
    case MFADVR_F16: return launch_render_dtype<__half>(mv, rs, stream);
    case MFADVR_BF16: return launch_render_dtype<__nv_bfloat16>(mv, rs, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mfadvr
