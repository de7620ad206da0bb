// Internal declarations shared by the translation units of libmfadvr.so.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mfadvr.h"

namespace mfadvr {

// Factor by which the device-side uniform basis of degree p is scaled
// (BasisScale in mfa_basis.cuh): contractions come out multiplied by its cube.
constexpr float basis_scale_host(int p) { return p == 3 ? 6.0f : 1.0f; }

// A resident model as the kernels see it.  The control points live in the
// row layout (see mfa_basis.cuh): entry (i, j, k) at i + n[0]*(j + n[1]*k)
// holds the pairs (P(i+d,j+2h,k), P(i+d,j+2h+1,k)), d = 0..3, h = 0 (FP32) or
// h = 0..1 (FP16/BF16), in the storage type.
struct ModelView {
    const void *rows;
    int n[3];       // control points per axis
    int n01;        // n[0] * n[1]
    int m[3];       // knot spans per axis, m = n - p
    int p;          // degree (equal on all axes)
    int dtype;      // mfadvr_dtype
    float scale;    // storage scale s (1 for FP32)
    // General (non-uniform) clamped knots when nu != 0; per axis: m+1 span
    // breakpoints, m inverse span widths and per-span basis pieces (layout in
    // mfa_basis.cuh, GeneralPieces).  Null with uniform knots (nu = 0).
    int rational;        // 1: rows hold w P, wrows the weights w (NURBS)
    const void *wrows;
    float wscale;        // storage scale of wrows (1 for FP32)
    // POWER render form: per span cell the monomial coefficients of the
    // model about the cell centre (PolyCell in mfa_basis.cuh); null otherwise.
    // A rational model's poly holds those of w P, wpoly those of w.
    const float *poly;
    const float *wpoly;
    int nu;
    int grid[3];  // lookup cells per axis (G = 2m)
    const float *brk[3];
    const float *ih[3];
    const int *cell[3];
    const float *pieces[3];
};

// Everything the render kernel needs besides the model, in FP32, derived on
// the host from mfadvr_camera / mfadvr_render_params.
struct RenderSetup {
    int width, height;
    int kind;                           // 0 orthographic, 1 perspective
    float eye[3], fwd[3], right[3], up[3];
    float sx_scale, sx_off, sy_scale, sy_off;  // sx = sx_scale*(x+1/2) + sx_off
    float box_min[3], box_max[3], inv_ext[3];
    float lat_scale[3];                 // world -> lattice units: m / extent (general knots: 1 / extent)
    float grad_scale[3];                // contraction derivative -> world gradient
    float step, max_opacity, opacity_ratio;
    int correct_opacity;                // 1 when step != ref_step
    const float4 *tf;                   // device table, tf_size >= 2 entries
    int tf_size;
    // table coordinate of a contraction result r: clamp(r*tf_a + tf_b, 0, 1) (tf_size-1)
    // (folds the storage scale, the basis scale and [lo, hi] into one FMA)
    float tf_a, tf_b;
    int shading;
    float ka, kd, ks, shininess;
    float gthresh2;                     // |g|^2 <= gthresh2: ambient only
    float4 *out;                        // H x W
    int32_t *nsamples;                  // H x W or nullptr
    int tile_w_log2;                    // ray tiles of 2^k x 32/2^k pixels (k = 0..5)
    int ctas_per_sm;                    // resident CTAs per SM to launch (0: as many as fit)
    // Longest-first tile order (mfadvr_render): scratch of one launch, or
    // nullptr for row order.  tile_order: one tile index per tile;
    // tile_level: one byte per tile; tile_hist: 64 ints (per-level counts,
    // then per-level cursors), zeroed by the launcher.
    int *tile_order = nullptr;
    unsigned char *tile_level = nullptr;
    int *tile_hist = nullptr;
};

// One image of a batched render: its model, settings and place in the
// concatenated tile sequence of the launch (sorted by tile_begin).
struct RenderJob {
    ModelView mv;
    RenderSetup rs;
    int tile_begin;  // first tile of this job in the launch
    int tiles_x;     // tiles per image row
    int tiles;       // tiles of this job
    int pad;
};
static_assert(sizeof(RenderJob) % 8 == 0, "RenderJob is copied in 8-byte words");

// Dispatch key of the render kernels: the storage type, or kPolyForm when
// the model's span polynomials are evaluated (the POWER render form, for
// shaded renders: without the gradient the B-spline value-only kernel on the
// row array is the faster one, the polynomial cells being 8x the rows' bytes).
constexpr int kPolyForm = 16;
inline int render_form_key(const ModelView &v, int shading) { return v.poly && shading ? kPolyForm : v.dtype; }

// Bytes of one span cell's coefficients in the POWER form (degree p <= 4):
// (p+1) x ceil((p+1)/2) x (p+1) coefficient pairs, in whole 32-byte sectors.
constexpr int poly_cell_bytes(int p) { return ((p + 1) * ((p + 2) / 2) * (p + 1) * 8 + 31) / 32 * 32; }

// Kernel launchers (asynchronous on `stream`).
// query is an mfadvr_query: out holds n floats (value), 3n (gradient), n
// float4 (both) or 10n (Hessian).  The point-query grid is the SM count
// times the resident CTAs per SM, capped at max_blocks CTAs when that is > 0.
cudaError_t launch_eval_points(const ModelView &mv, const float *params, int64_t n, float *out, int query,
                               int32_t *spans, cudaStream_t stream, int max_blocks = 0);
// `counter` is one device int the render kernel's warps take ray tiles from;
// the launcher zeroes it on `stream` first.  The value-only kernel runs when
// rs.shading is 0 (no gradient is needed).
cudaError_t launch_render(const ModelView &mv, const RenderSetup &rs, int *counter, cudaStream_t stream);
// Fills rs.tile_order (when not null) with the ray tiles of this launch's
// shape, costliest first, on `stream`: launched by the render launcher
// before the render kernel.
cudaError_t launch_tile_order(const RenderSetup &rs, int tiles_x, int tiles, cudaStream_t stream);
// The same render recording, for each ray's first max_samples samples, the
// FP32 position the kernel walks and the knot spans it contracts with
// (mfadvr_render_trace).  FP32 models, shading on, plain (not rational).
struct TraceOn {
    float *pos;      // H x W x max_samples x 3: lattice units (uniform knots) or parameter units
    int32_t *span;   // H x W x max_samples x 3: knot-span index, p..n-1
    int max_samples;
};
cudaError_t launch_render_trace(const ModelView &mv, const RenderSetup &rs, int *counter, const TraceOn &tr,
                                cudaStream_t stream);
// Batched render of njobs jobs of degree p and storage dtype, all with
// shading on (grad = 1) or all off (grad = 0), all on general knots (nu = 1)
// or all on uniform ones, all rational (rat = 1) or none (jobs_dev in device
// memory, sorted by tile_begin, total_tiles tiles in all); `counter` is
// zeroed on `stream` first.  `order`: the tiles in the order the warps take
// them (launch_tile_order_batch), or nullptr for job order.
cudaError_t launch_render_batch(int p, int dtype, int grad, int nu, int rat, const RenderJob *jobs_dev, int njobs,
                                int total_tiles, int ctas_per_sm, int *counter, const int *order, cudaStream_t stream);
// Fills order[0 .. tiles) with the tiles of a batched launch (jobs_dev, as
// for launch_render_batch), costliest first; max_count is the largest sample
// count along a job's box diagonal (the scale of the cost levels); level
// (tiles bytes) and hist (64 ints) are scratch.
cudaError_t launch_tile_order_batch(const RenderJob *jobs_dev, int njobs, int tiles, float max_count, int *order,
                                    unsigned char *level, int *hist, cudaStream_t stream);
// Bytes of one row-layout entry (4 x 2 FP32 or 4 x 4 16-bit control points).
constexpr size_t row_entry_bytes(int) { return 32; }
// Builds the row array of an n0 x n1 x n2 FP32 lattice (device memory),
// scaling by inv_scale and rounding to the storage type.
cudaError_t launch_build_rows(const float *src, void *rows, int n0, int n1, int n2, int dtype, float inv_scale,
                              cudaStream_t stream);
// Span polynomials of an FP32 model of degree p <= 4 from its control points
// (src, as for launch_build_rows) into poly (m0 m1 m2 cells of
// poly_cell_bytes(p)); pieces[a] (device, FP64) holds axis a's span pieces
// about the span centres, m_a x (p+1) x (p+1).
cudaError_t launch_build_poly(const float *src, void *poly, int p, int n0, int n1, int n2,
                              const double *const pieces[3], cudaStream_t stream);

// Render setup for a caller-owned FP32 lattice outside any context, and the
// context-free error sink (mfadvr_last_error(NULL)); both in mfadvr_api.cu.
mfadvr_status setup_for_lattice(int p, const int n[3], const float box_min[3], const float box_max[3],
                                const mfadvr_camera *cam, const mfadvr_render_params *rp, RenderSetup *rs);
mfadvr_status fail_noctx(mfadvr_status st, const char *msg);

}  // namespace mfadvr
