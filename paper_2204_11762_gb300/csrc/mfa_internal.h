// Internal declarations shared by the translation units of libmfadvr.so.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mfadvr.h"

namespace mfadvr {

// A resident model as the kernels see it.  Control points are one array in
// the storage type, u fastest: (i, j, k) at i + n[0]*(j + n[1]*k).
struct ModelView {
    const void *cp;
    int n[3];       // control points per axis
    int m[3];       // knot spans per axis, m = n - p
    int p;          // degree (equal on all axes)
    int dtype;      // mfadvr_dtype
    float scale;    // storage scale s (1 for FP32)
};

// Everything the render kernel needs besides the model, in FP32, derived on
// the host from mfadvr_camera / mfadvr_render_params.
struct RenderSetup {
    int width, height;
    int kind;                           // 0 orthographic, 1 perspective
    float eye[3], fwd[3], right[3], up[3];
    float sx_scale, sx_off, sy_scale, sy_off;  // sx = sx_scale*(x+1/2) + sx_off
    float box_min[3], box_max[3], inv_ext[3];
    float grad_scale[3];                // local-derivative -> world gradient
    float step, max_opacity, opacity_ratio;
    int correct_opacity;                // 1 when step != ref_step
    const float4 *tf;                   // device table, tf_size >= 2 entries
    int tf_size;
    float tf_lo, tf_inv_range;          // x = clamp((v - lo) * inv_range, 0, 1)
    int shading;
    float ka, kd, ks, shininess;
    float gthresh2;                     // |g|^2 <= gthresh2: ambient only
    float4 *out;                        // H x W
    int32_t *nsamples;                  // H x W or nullptr
};

// Kernel launchers (asynchronous on `stream`).
cudaError_t launch_eval_points(const ModelView &mv, const float *params, int64_t n, float4 *out,
                               int32_t *spans, cudaStream_t stream);
cudaError_t launch_render(const ModelView &mv, const RenderSetup &rs, cudaStream_t stream);
cudaError_t launch_quantize(const float *src, void *dst, int64_t count, int dtype, float inv_scale,
                            cudaStream_t stream);

}  // namespace mfadvr
