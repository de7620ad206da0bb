/*
 * mfadvr.h -- C ABI of the GB300 MFA-DVR library (libmfadvr.so).
 *
 * MFA-DVR ("MFA-DVR: direct volume rendering of MFA models", Sun, Lenz, Yu,
 * Peterka) renders a multivariate functional approximation (MFA) directly:
 * every sample of every ray queries a tensor-product B-spline model for its
 * value and gradient (Sec. 3.1, Algorithm 1).  The model (Sec. 2.3) is a
 * lattice of control points with a clamped knot vector and a degree p_d per
 * axis over the parameter box [0,1]^3.  Knots are uniform by default:
 *   t_0..t_p = 0,  t_{p+j} = j/m (j = 1..m-1),  t_n..t_{n+p} = 1,  m = n - p;
 * a model may instead give its own clamped knots per axis (the adaptive,
 * non-uniform knots an MFA fit places, Sec. 2.3).
 *
 * Conventions shared by every call:
 *  - Status: every entry point returns an mfadvr_status, 0 on success.  No
 *    C++ exception crosses this boundary.  All argument checks run before any
 *    device work, so a call that returns MFADVR_EINVAL has touched nothing.
 *    A failing call stores a message readable with mfadvr_last_error().
 *  - Lattice layout: control point (i, j, k) sits at i + n0*(j + n1*k), i.e. u
 *    varies fastest.
 *  - Device pointers ("_dev") are owned by the caller, must stay valid until
 *    the work queued on the given stream has finished, and are never freed by
 *    the library.  Host pointers are read (or written) before the call
 *    returns.
 *  - Streams: "stream" is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  mfadvr_eval_points and mfadvr_render only enqueue work
 *    on it and return, as does mfadvr_query_points_host_async (page-locked
 *    host buffers); the other *_host variants and mfadvr_load_model
 *    synchronise.
 *  - Threads: a context is used by one host thread at a time (or under an
 *    external lock).
 *  - Degrees: 1..MFADVR_MAX_DEGREE and equal on the three axes (the kernels
 *    are compiled per degree); other degrees return MFADVR_EUNSUPPORTED.
 *  - Knots: clamped, uniform unless mfadvr_model_desc.knots gives them (see
 *    there).
 */
#ifndef MFADVR_H
#define MFADVR_H

#include <stdint.h>

#if defined(__GNUC__)
#define MFADVR_API __attribute__((visibility("default")))
#else
#define MFADVR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mfadvr_ctx mfadvr_ctx; /* opaque, one per device */
typedef int32_t mfadvr_status;

#define MFADVR_OK 0
#define MFADVR_EINVAL (-1)       /* bad argument: NULL, size, non-finite value  */
#define MFADVR_ENOMEM (-2)       /* HBM budget exceeded or allocation failed     */
#define MFADVR_ECUDA (-3)        /* a CUDA runtime call failed                   */
#define MFADVR_ENOTFOUND (-4)    /* no model with that id                        */
#define MFADVR_ETIMEOUT (-5)     /* a wait ran out of time                       */
#define MFADVR_EBUSY (-6)        /* resource in use                              */
#define MFADVR_EUNSUPPORTED (-7) /* valid but not built (degree, knots, dtype)   */

#define MFADVR_MAX_DEGREE 5
#define MFADVR_MAX_TF_SIZE 4096

/* Storage type of the control points.  F16 and BF16 store P / s with a
 * per-model scale s (s = 1 when all P are 0): for BF16 s = max|P|; for F16
 * the power of two that puts max|P| / s in [2^14, 2^15), so that values down
 * to about 2^-29 max|P| are normal FP16 numbers.  Evaluation converts to
 * FP32, accumulates in FP32 and multiplies the result by s. */
typedef enum { MFADVR_F32 = 0, MFADVR_F16 = 1, MFADVR_BF16 = 2 } mfadvr_dtype;

/* How the render kernels evaluate a model (the point queries always use the
 * B-spline form).  Within one knot-span cell the model is a polynomial of the
 * cell's local coordinates; the POWER form stores, per cell, its monomial
 * coefficients about the cell centre (FP32, computed in FP64 from the basis
 * pieces at load) and evaluates value and gradient by nested Horner sums: no
 * basis per sample, and at degree 3 123 multiply-adds on 83 instructions
 * instead of 192 on 128 plus the basis.  The price is (p+1)^3 floats per
 * cell: at degree 3 and 128^3 control points 500 MB beside the 67 MB row
 * array (twice that for a rational model: the polynomials of w P and of
 * w).  It applies to FP32 models of degree <= 3 (uniform or general knots,
 * plain or rational) and to plain ones of degree 4, with fewer than 2^22
 * spans per axis (a sample is placed by its FP32 offset from the span's
 * centre, index + 1/2, exact below that), and serves shaded
 * renders; unshaded ones
 * (value only) run the B-spline kernel on the row array, which is faster
 * there.  Results agree with the B-spline form to FP32 rounding. */
typedef enum {
    MFADVR_FORM_AUTO = 0,    /* POWER where it applies, fits the HBM budget and
                                takes at most 4 GiB; the B-spline form else   */
    MFADVR_FORM_BSPLINE = 1, /* the basis and the sum-factorised contraction    */
    MFADVR_FORM_POWER = 2    /* required: EUNSUPPORTED where it does not apply,
                                ENOMEM where it does not fit                    */
} mfadvr_render_form;

/* An MFA model (Sec. 2.3): degree, control-point lattice, knots, and the
 * world box that maps onto the parameter box [0,1]^3. */
typedef struct {
    int32_t degree[3];     /* p_d, 1..MFADVR_MAX_DEGREE, equal on all axes     */
    int32_t ncp[3];        /* n_d >= p_d + 1, n_d <= 2^24, n0 n1 n2 < 2^31    */
    float box_min[3];      /* world box; box_max > box_min on every axis       */
    float box_max[3];
    const float *ctrl;     /* HOST, n0*n1*n2 finite FP32 values (u fastest)    */
    const float *knots[3]; /* per axis: NULL (uniform knots) or HOST, n_d+p+1
                              FP32 knots: p+1 zeros, interior knots strictly
                              increasing inside (0,1), p+1 ones.  With any
                              axis given, queries find spans by binary search
                              and take the basis from per-span tables built
                              at load (NULL axes then use j/m rounded to FP32) */
    mfadvr_dtype storage;  /* storage type in HBM                              */
    const float *weights;  /* NULL (non-rational) or HOST n0*n1*n2 positive
                              finite weights indexed like ctrl: a rational
                              model (NURBS, Sec. 2.3), f = sum w P N N N /
                              sum w N N N.  The library stores w P and w in
                              the storage type (16-bit: each with its own
                              scale, as for P); two contractions per query
                              make it about half the plain model's speed */
    int32_t render_form;   /* mfadvr_render_form; 0 (AUTO) when zeroed      */
} mfadvr_model_desc;

/* Camera in world space (the "Ray Definition" step of Sec. 3.1).  Frame:
 * forward f = normalize(center - eye), right r = normalize(up x f),
 * true up u = f x r.  Pixel (x, y), row 0 at the top, has screen offsets
 * sx = (2(x+1/2)/W - 1) * a and sy = (1 - 2(y+1/2)/H) * b:
 *  kind 0 (orthographic): a = ortho_height*W/(2H), b = ortho_height/2;
 *         ray origin eye + sx r + sy u, direction f;
 *  kind 1 (perspective):  a = tan(fovy/2)*W/H, b = tan(fovy/2);
 *         ray origin eye, direction normalize(f + sx r + sy u). */
typedef struct {
    int32_t kind;
    float eye[3], center[3], up[3];
    float fovy_deg;     /* perspective: vertical field of view, (0, 180) */
    float ortho_height; /* orthographic: world height of the image, > 0  */
} mfadvr_camera;

/* Render settings (Algorithm 1).  Samples: t_k = t_enter + (k + 1/2) step,
 * k = 0..N-1, N = floor((t_exit - t_enter)/step), [t_enter, t_exit] the part
 * of the ray inside the world box (t_enter >= 0). */
typedef struct {
    int32_t width, height;  /* 1..65536 each, width * height <= 2^30          */
    float step;             /* constant sample distance, world units, > 0, and
                               at most 2^24 samples along the world box's
                               diagonal (diagonal / step <= 2^24)              */
    float max_opacity;      /* O_max: stop after a sample makes A > O_max      */
    float ref_step;         /* opacity correction 1-(1-a)^(step/ref); <=0: off */
    const float *tf_rgba;   /* tf_size RGBA entries (DEVICE for mfadvr_render,
                               HOST for mfadvr_render_host)                     */
    int32_t tf_size;        /* 1..MFADVR_MAX_TF_SIZE                           */
    float tf_lo, tf_hi;     /* value range of the table; NaN: [min P, max P]   */
    int32_t shading;        /* 0: value only, 1: gradient shading              */
    float ka, kd, ks, shininess; /* Blinn-Phong, one headlight: rgb_tf (ka +
                               kd |n.L|) + ks |n.L|^shininess, clamped to [0,1] */
} mfadvr_render_params;

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the bytes
 * of resident models (0 = no cap).  *out receives the handle.
 * EINVAL: out NULL or device < 0.  ECUDA: no such device. */
MFADVR_API mfadvr_status mfadvr_create(mfadvr_ctx **out, int device, uint64_t hbm_budget_bytes);

/* Free every model and the context.  NULL is accepted (no-op). */
MFADVR_API mfadvr_status mfadvr_destroy(mfadvr_ctx *ctx);

/* Copy a model into library-owned HBM (Sec. 3: the encoded model is the
 * renderer's input).  Synchronous: the caller may free desc->ctrl on return.
 * *model_id receives a handle >= 0.  EINVAL: bad sizes, box, non-finite
 * control points, a knot vector that is not clamped and strictly increasing
 * inside, a weight that is not positive and finite.  EUNSUPPORTED: degree outside
 * 1..MFADVR_MAX_DEGREE or unequal per axis.  ENOMEM: over budget. */
MFADVR_API mfadvr_status mfadvr_load_model(mfadvr_ctx *ctx, const mfadvr_model_desc *desc, int32_t *model_id);

/* Free a model's HBM.  ENOTFOUND: unknown id.  Work already queued that reads
 * the model must have finished (the call synchronises the device). */
MFADVR_API mfadvr_status mfadvr_unload_model(mfadvr_ctx *ctx, int32_t model_id);

/* Value range [min P, max P] of the loaded control points (the default TF
 * domain), the storage scale s and the model's resident bytes (row arrays,
 * knot tables and, in the POWER render form, the span polynomials).  Any
 * output pointer may be NULL. */
MFADVR_API mfadvr_status mfadvr_model_info(mfadvr_ctx *ctx, int32_t model_id, float *pmin, float *pmax,
                                float *scale, uint64_t *bytes);

/* Value and first derivatives at n parameter points (queryValueMFA and
 * queryGradientMFA of Algorithm 1, computed together as Sec. 3.1 asks).
 *  params_dev: n x 3 FP32 (u, v, w); values outside [0,1] (and NaN, read as
 *              0) are clamped to the box.
 *  out_dev:    n x 4 FP32 (f, df/du, df/dv, df/dw), parameter space; 16-byte
 *              aligned.
 *  spans_dev:  n x 3 int32 knot-span indices s_d in [p, n_d - 1] (t_s <= u <
 *              t_{s+1}; u = 1 in the last span), or NULL.
 * n = 0 is a no-op.  EINVAL: NULL buffers with n > 0, n < 0, misalignment. */
MFADVR_API mfadvr_status mfadvr_eval_points(mfadvr_ctx *ctx, int32_t model_id, const float *params_dev, int64_t n,
                                 float *out_dev, int32_t *spans_dev, void *stream);

/* As mfadvr_eval_points with HOST buffers: copies params in, evaluates and
 * copies the results back through library-owned staging memory, then
 * synchronises.  Page-locked (pinned) host buffers are read and written by
 * the kernel directly, with no staging copies.  Other buffers go through
 * staging: from 2^20 points up in 16 chunks on three streams of the context,
 * ordered after the work already queued on `stream`, so that copies in,
 * kernels and copies out of neighbouring chunks overlap. */
MFADVR_API mfadvr_status mfadvr_eval_points_host(mfadvr_ctx *ctx, int32_t model_id, const float *params_host,
                                      int64_t n, float *out_host, int32_t *spans_host, void *stream);

/* What a point query returns: the value alone (queryValueMFA), the gradient
 * alone (queryGradientMFA), or both (Algorithm 1; the parameter study of
 * Sec. 4.3.3 times each of the three).  Only the sums a query needs are
 * formed: per point (p+1)^3 + (p+1)^2 + (p+1) multiply-adds for the value,
 * 2(p+1)^3 + 3(p+1)^2 + 3(p+1) for the gradient, 2(p+1)^3 + 3(p+1)^2 + 4(p+1)
 * for both. */
typedef enum {
    MFADVR_QUERY_VALUE = 1,    /* out: n FP32 f, 4-byte aligned */
    MFADVR_QUERY_GRADIENT = 2, /* out: n x 3 FP32 (df/du, df/dv, df/dw), 4-byte aligned */
    MFADVR_QUERY_BOTH = 3,     /* out: n x 4 FP32 (f, df/du, df/dv, df/dw), 16-byte aligned */
    MFADVR_QUERY_HESSIAN = 4   /* out: n x 10 FP32 (f, f_u, f_v, f_w, f_uu, f_vv, f_ww, f_uv,
                                  f_uw, f_vw), 4-byte aligned: the higher-order query of
                                  Sec. 3.1 (curvature-based transfer functions), analytic
                                  up to the degree (Sec. 2); 3(p+1)^3 + 6(p+1)^2 + 10(p+1)
                                  multiply-adds per point */
} mfadvr_query;

/* mfadvr_eval_points for one mfadvr_query (an int32 here); with
 * MFADVR_QUERY_BOTH it is mfadvr_eval_points.  params_dev and spans_dev as
 * there; out_dev laid out as the query says.  Each output equals the same
 * component of MFADVR_QUERY_BOTH bit for bit (the Hessian query's first
 * four outputs agree with it to rounding).  EINVAL: an unknown query, plus
 * mfadvr_eval_points' cases. */
MFADVR_API mfadvr_status mfadvr_query_points(mfadvr_ctx *ctx, int32_t model_id, const float *params_dev, int64_t n,
                                  int32_t query, float *out_dev, int32_t *spans_dev, void *stream);

/* mfadvr_query_points with HOST buffers, as mfadvr_eval_points_host. */
MFADVR_API mfadvr_status mfadvr_query_points_host(mfadvr_ctx *ctx, int32_t model_id, const float *params_host,
                                       int64_t n, int32_t query, float *out_host, int32_t *spans_host,
                                       void *stream);

/* Stream-ordered mfadvr_query_points_host for page-locked host buffers
 * (cudaHostAlloc, cudaHostRegister, pinned tensors): the query is queued on
 * `stream` and the call returns without waiting.  The kernel reads params_host
 * and writes out_host (and spans_host) over the host link; the results are in
 * place once the stream's work up to this call has completed, and the buffers
 * must stay allocated until then.  Results equal mfadvr_query_points' bit for
 * bit.
 *  max_ctas: at most this many 256-thread blocks serve the query, 0 = as many
 *            as fill the GPU.  A query on host buffers waits on the host link
 *            and on its gathers more than on the SMs, so a few blocks keep most
 *            of its rate and leave the other SMs to work queued on other
 *            streams after it, e.g. a render: that is how the point query of a
 *            step overlaps the step's frame.
 * EINVAL: a buffer that is not page-locked, out not aligned as
 * mfadvr_query_points requires, max_ctas < 0, plus mfadvr_query_points' cases.
 * n = 0 is a no-op. */
MFADVR_API mfadvr_status mfadvr_query_points_host_async(mfadvr_ctx *ctx, int32_t model_id, const float *params_host,
                                             int64_t n, int32_t query, float *out_host, int32_t *spans_host,
                                             int32_t max_ctas, void *stream);

/* Ray-cast one image (Algorithm 1): per pixel, march the ray through the
 * model's world box, query value (+ gradient when shading), map through the
 * transfer function, shade, composite front to back and stop early once the
 * cumulative opacity exceeds max_opacity.
 *  rgba_dev:     height x width x 4 FP32, premultiplied RGBA, row 0 at the
 *                top, 16-byte aligned; pixels whose ray misses the box are 0.
 *  nsamples_dev: height x width int32 samples composited per pixel, or NULL.
 * Scheduling (no pixel depends on it): the persistent kernel's warps take
 * 32-ray tiles costliest first, so that the frame ends on short tiles; two
 * small kernels before it bin the tiles by the largest sample count of their
 * rays (the chord through the box over the step) and sort them.  That order
 * needs a scratch area from a ring of 8 (about 2.5 MiB each, allocated at
 * the first render of the context); a render waits on its stream for the
 * render that used the same area 8 calls earlier.  Images of fewer than 32
 * or more than 1024 tiles per SM (or more than 2^19 tiles) take their tiles
 * in row order: too few tiles leave no tail to shorten, and with many the
 * tail is small and row order keeps the tiles that run together close.
 * The call is not meant for CUDA stream capture: its first call on a context
 * allocates, and later ones wait on an event of an earlier render.
 * EINVAL: bad camera/params/buffers. */
MFADVR_API mfadvr_status mfadvr_render(mfadvr_ctx *ctx, int32_t model_id, const mfadvr_camera *camera,
                            const mfadvr_render_params *params, float *rgba_dev, int32_t *nsamples_dev,
                            void *stream);

/* mfadvr_render with a record of the knot spans (a test and inspection
 * facility): the same kernel, instantiated with a trace, also writes for each
 * ray's first max_samples samples the FP32 position the kernel walks and the
 * knot-span index it evaluates the model on (queryValueMFA / queryGradientMFA
 * inside Algorithm 1, Sec. 3.1), so that the spans can be checked exactly
 * against a span search on those positions.
 *  rgba_dev, nsamples_dev: as for mfadvr_render.
 *  max_samples:  samples recorded per ray, >= 1; width*height*max_samples
 *                at most 2^24.
 *  pos_dev:      DEVICE, height x width x max_samples x 3 FP32: sample k of
 *                the ray of pixel (x, y) at [(y width + x) max_samples + k]:
 *                its position in lattice units on uniform knots (the
 *                parameter u times the span count m, unclamped), in parameter
 *                units on general knots.  Entries past the ray's last
 *                contracted sample are not written.
 *  span_dev:     DEVICE, same layout, int32: the knot-span index s in
 *                [p, n-1] per axis (the span of the position clamped to the
 *                parameter box).
 * Only shaded renders of plain FP32 models (either render form, uniform or
 * general knots) are traced: EUNSUPPORTED otherwise.  Asynchronous on
 * stream. */
MFADVR_API mfadvr_status mfadvr_render_trace(mfadvr_ctx *ctx, int32_t model_id, const mfadvr_camera *camera,
                                             const mfadvr_render_params *params, float *rgba_dev,
                                             int32_t *nsamples_dev, int32_t max_samples, float *pos_dev,
                                             int32_t *span_dev, void *stream);

/* As mfadvr_render with HOST buffers (params->tf_rgba is then a host
 * pointer): copies the table in, renders, copies the image (and sample
 * counts, if requested) back and synchronises the stream.  Page-locked
 * output buffers (16-byte aligned for rgba) are written by the kernel
 * directly instead. */
MFADVR_API mfadvr_status mfadvr_render_host(mfadvr_ctx *ctx, int32_t model_id, const mfadvr_camera *camera,
                                 const mfadvr_render_params *params, float *rgba_host,
                                 int32_t *nsamples_host, void *stream);

/* One image of a batched render: a loaded model seen by a camera. */
typedef struct {
    int32_t model_id;
    mfadvr_camera camera;
    mfadvr_render_params params; /* tf_rgba: 16-byte aligned DEVICE table, tf_size >= 2 */
    float *rgba_dev;             /* height x width x 4 FP32, 16-byte aligned           */
    int32_t *nsamples_dev;       /* height x width int32, or NULL                      */
} mfadvr_render_job;

#define MFADVR_MAX_BATCH 256

/* Render njobs images (Algorithm 1 for each), of any loaded models, in one
 * call.  Jobs are grouped by degree and storage type; each group is ONE
 * launch of a persistent kernel whose warps take 32-ray tiles from a single
 * queue over the concatenated tiles of the group's images (kernels are
 * compiled per degree, so a batch of several degrees launches once per
 * degree).  Each image equals what mfadvr_render gives for its job.  As in
 * mfadvr_render, a group of 32 to 1024 tiles per SM takes them costliest
 * first (two small kernels before it, on the ring of order scratch areas);
 * the serving loop's batches take them in job order.
 * 1 <= njobs <= MFADVR_MAX_BATCH.  Asynchronous on `stream`; the job table
 * is copied before the call returns.  The context keeps a ring of 32 job
 * tables and 1024 tile counters: more than 32 batches (or 1024 render
 * launches) in flight at once on different streams would reuse one.
 * EINVAL / ENOTFOUND as for mfadvr_render, per job. */
MFADVR_API mfadvr_status mfadvr_render_batch(mfadvr_ctx *ctx, int32_t njobs, const mfadvr_render_job *jobs,
                                             void *stream);

/* Launch shape of the render kernels, chosen by the autotuner. */
typedef struct {
    int32_t tile_w;      /* ray tile of tile_w x 32/tile_w pixels: 1, 2, 4, 8, 16 or 32 */
    int32_t ctas_per_sm; /* resident CTAs per SM (0: as many as fit)                  */
    float ms;            /* measured render time of the chosen shape                  */
} mfadvr_tuning;

/* Time mfadvr_render of this job under each candidate launch shape (tile
 * shapes x occupancy), keep the fastest in the context's tuning table under
 * the key (degree, storage type, log2 of the lattice size, log2 of the image
 * size), and return it in *best (may be NULL).  mfadvr_render and
 * mfadvr_render_batch use the table for every matching key.  Synchronous;
 * writes the job's outputs.  A "batching" knob of the paper's design space
 * (Sec. 4.3: performance depends on degree, lattice and image size). */
MFADVR_API mfadvr_status mfadvr_autotune(mfadvr_ctx *ctx, int32_t model_id, const mfadvr_camera *camera,
                                         const mfadvr_render_params *params, float *rgba_dev,
                                         int32_t *nsamples_dev, void *stream, mfadvr_tuning *best);

/* Write / read the tuning table as text, one "p dtype lattice_log2
 * image_log2 tile_w ctas_per_sm ms" line per key.  Loading merges into the
 * table.  EINVAL: unreadable file or malformed line. */
MFADVR_API mfadvr_status mfadvr_tuning_save(mfadvr_ctx *ctx, const char *path);
MFADVR_API mfadvr_status mfadvr_tuning_load(mfadvr_ctx *ctx, const char *path);

/* ---- Serving: continuous batching ---------------------------------------
 * A serving loop (one host thread per context) takes render requests at any
 * time and keeps the GPU busy with them: each scheduling step admits the
 * oldest queued requests while their output images fit the frame-buffer
 * budget (and the batch and in-flight limits), packs them into one batched
 * launch per degree and storage type (as mfadvr_render_batch), replays that
 * launch sequence through a CUDA graph kept per group signature and stream,
 * and marks the requests done when the batch completes.  Requests arriving
 * while batches run join the next step, on another stream, so their work
 * overlaps the batches in flight.  Each image equals mfadvr_render of its
 * job.  While the loop runs, call only mfadvr_submit / mfadvr_wait /
 * mfadvr_serve_stats / mfadvr_serve_stop on the context, from any threads;
 * models must stay loaded until their requests are done. */
typedef struct {
    uint64_t frame_budget_bytes; /* output bytes (rgba + nsamples) in flight; 0: 1 GiB.
                                    An idle loop admits one request even if it is larger. */
    int32_t max_batch;           /* requests per scheduling step, 0..MFADVR_MAX_BATCH (0: 64) */
    int32_t max_in_flight;       /* batches on the GPU at once, 0..8 (0: 2) */
} mfadvr_serve_config;

/* Start the serving loop.  EBUSY if it runs already. */
MFADVR_API mfadvr_status mfadvr_serve_start(mfadvr_ctx *ctx, const mfadvr_serve_config *config);
/* Finish every queued and running request, then stop the loop. */
MFADVR_API mfadvr_status mfadvr_serve_stop(mfadvr_ctx *ctx);
/* Queue one render request (validated now, as mfadvr_render_batch does per
 * job); *ticket identifies it.  The job's buffers must stay valid until the
 * request is done. */
MFADVR_API mfadvr_status mfadvr_submit(mfadvr_ctx *ctx, const mfadvr_render_job *job, uint64_t *ticket);
/* Wait until the request is done: timeout_us < 0 waits without limit, 0
 * polls.  On MFADVR_OK the ticket is released and *latency_us (may be NULL)
 * holds the time from submission to the completion of its batch.
 * ETIMEOUT: not done yet (the ticket stays valid).  ENOTFOUND: unknown or
 * already released ticket.  ECUDA: its batch failed on the GPU. */
MFADVR_API mfadvr_status mfadvr_wait(mfadvr_ctx *ctx, uint64_t ticket, int64_t timeout_us, int64_t *latency_us);
/* Counters of the loop: batched launches, graph updates, graph instantiations. */
MFADVR_API mfadvr_status mfadvr_serve_stats(mfadvr_ctx *ctx, uint64_t *launches, uint64_t *graph_updates,
                                            uint64_t *graph_instantiations);

/* One batch of the serving loop, times in microseconds since
 * mfadvr_serve_start: a trace of the scheduler. */
typedef struct {
    int64_t oldest_submit_us; /* submission of the batch's oldest request     */
    int64_t t_admit_us;       /* admission                                      */
    int64_t t_launched_us;    /* the launch call returned                       */
    int64_t t_done_us;        /* completion seen by the loop                    */
    int32_t jobs;             /* requests in the batch                          */
    int32_t groups;           /* launches (degree x storage groups)             */
    int32_t stream;           /* stream index                                   */
    int32_t queued_after;     /* requests still queued after admission          */
} mfadvr_serve_trace_record;

/* Copy the most recent completed batches (at most `capacity`, oldest first;
 * the loop keeps the last 4096) into records; *count receives how many. */
MFADVR_API mfadvr_status mfadvr_serve_trace(mfadvr_ctx *ctx, mfadvr_serve_trace_record *records, int32_t capacity,
                                            int32_t *count);

/* ---- Allocation-free render -------------------------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory during a render.  Examples are code recording
 * into a CUDA stream capture, plug-in hosts whose device memory belongs to
 * the host application's pool allocator, and real-time loops that cannot
 * afford the device synchronisation an allocation implies.  mfadvr_create,
 * mfadvr_load_model and mfadvr_render all allocate; this call does not.
 *
 * It renders like mfadvr_render from a lattice the caller keeps in its own
 * device memory, with no context and no loaded model:
 *  ctrl_dev:     DEVICE, ncp[0]*ncp[1]*ncp[2] FP32 control points (u fastest),
 *                4-byte aligned; at most MFADVR_NOALLOC_MAX_POINTS of them
 *                (larger lattices return MFADVR_ENOMEM).  Values must be
 *                finite (they are not scanned).
 *  degree, ncp, box_min, box_max: as in mfadvr_model_desc (clamped uniform
 *                knots, FP32 storage).
 *  params:       as for mfadvr_render, with tf_rgba a 16-byte aligned DEVICE
 *                table of at least 2 entries, and tf_lo / tf_hi given (NaN is
 *                refused: the lattice range is not computed).  Shading treats
 *                only an exactly zero gradient as ambient-only.
 *  rgba_dev, nsamples_dev, stream: as for mfadvr_render.
 * Scratch: the row layout of the lattice (8 FP32 values per control point)
 * and the ray-tile counter live in one file-scope device array of
 * 256 + 32 * MFADVR_NOALLOC_MAX_POINTS bytes (16 MiB + 256 B), which every GPU
 * that loads the library holds until the process exits.  Every call rebuilds
 * the rows and zeroes the counter on its
 * stream before reading them, so no call reads what an earlier call left
 * there; but all calls share that one array, so calls whose work overlaps
 * on the GPU (different streams, or different host threads) race and
 * corrupt each other's images.  Serialise them.
 * Set-up: the first call on a device, with that device current, looks up
 * the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture on that device.  A cudaDeviceReset gives the
 * device a new context, and the next call looks the address up again, so
 * make a call outside any capture after a reset too.  The work runs on the
 * current device and is asynchronous on `stream`; every buffer must be
 * memory of that device (or managed memory), else MFADVR_EINVAL.  Errors
 * are read with mfadvr_last_error(NULL). */
#define MFADVR_NOALLOC_MAX_POINTS (1 << 19)
MFADVR_API mfadvr_status mfadvr_render_lattice_noalloc(const float *ctrl_dev, const int32_t degree[3],
                                                       const int32_t ncp[3], const float box_min[3],
                                                       const float box_max[3], const mfadvr_camera *camera,
                                                       const mfadvr_render_params *params, float *rgba_dev,
                                                       int32_t *nsamples_dev, void *stream);

/* FP32 multiply-add throughput probe.  The paper has no counterpart: this is
 * a measurement.  The render and point-query kernels run on the FP32 FMA
 * pipe, and a benchmark divides their multiply-adds per second by this
 * call's, beside the peak derived from unit counts and clocks.
 * Enqueues one kernel on `stream` (asynchronous) on the current device: one
 * block of 256 threads per resident slot on every SM, each thread running
 * eight independent multiply-add chains for `iters` loop iterations of 64
 * chain steps, as scalar FMAs (packed = 0) or packed fma.rn.f32x2 pairs
 * (packed = 1).  Time it with events on the same stream.
 *  packed:    0 or 1.
 *  iters:     1..2^24 loop iterations per thread.
 *  sink_dev:  DEVICE, at least one float of the current device; written only
 *             in a case that does not arise (it keeps the chains live).
 *  fma_count: HOST, set to the multiply-adds the launch executes (2 FLOP
 *             each).
 * Errors (before any launch): EINVAL for NULL pointers, iters or packed out of
 * range, or a sink that is not memory of the current device; ECUDA if the
 * launch fails.  Read the message with mfadvr_last_error(NULL). */
MFADVR_API mfadvr_status mfadvr_probe_fma(int32_t packed, int32_t iters, float *sink_dev, void *stream,
                                          double *fma_count);

/* Static text for a status code. */
MFADVR_API const char *mfadvr_status_string(mfadvr_status status);

/* Message of the last failing call on ctx ("" if none); valid until the next
 * call on ctx.  NULL ctx gives the message of the last failing create. */
MFADVR_API const char *mfadvr_last_error(mfadvr_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MFADVR_H */
