// C ABI of libmfadvr.so: context, resident model store, argument checks and
// kernel dispatch.  See include/mfadvr.h for the contract of each call.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <algorithm>
#include <string>
#include <tuple>
#include <vector>

#include "ctx.h"
#include "mfa_basis.cuh"
#include "mfa_internal.h"
#include "mfadvr.h"

using namespace mfadvr;
using namespace mfadvr::api;

namespace {

std::mutex g_create_mu;
std::string g_create_err;

}  // namespace

namespace mfadvr {
namespace api {

mfadvr_status fail(mfadvr_ctx *ctx, mfadvr_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    else {
        std::lock_guard<std::mutex> g(g_create_mu);
        g_create_err = buf;
    }
    return st;
}

mfadvr_status cuda_fail(mfadvr_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, MFADVR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// True for device or managed memory; host pointers (registered or not) and
// foreign pointers are refused before any launch reads them.
bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

bool finite3(const float v[3]) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

ModelView view_of(const Model &m)
{
    ModelView v;
    v.rows = m.d_rows;
    v.n01 = m.n[0] * m.n[1];
    v.p = m.p;
    v.dtype = m.dtype;
    v.scale = m.scale;
    for (int a = 0; a < 3; ++a) {
        v.n[a] = m.n[a];
        v.m[a] = m.n[a] - m.p;
    }
    v.rational = m.rational;
    v.poly = static_cast<const float *>(m.d_poly);
    v.wpoly = m.d_poly && m.rational ? v.poly + m.poly_bytes / 2 / sizeof(float) : nullptr;
    v.wrows = m.d_wrows;
    v.wscale = m.wscale;
    v.nu = m.nu;
    const float *k = static_cast<const float *>(m.d_knots);
    for (int a = 0; a < 3; ++a) {
        v.grid[a] = 2 * (m.n[a] - m.p);
        v.brk[a] = m.nu ? k + m.brk_off[a] : nullptr;
        v.ih[a] = m.nu ? k + m.ih_off[a] : nullptr;
        v.cell[a] = m.nu ? reinterpret_cast<const int *>(k + m.cell_off[a]) : nullptr;
        v.pieces[a] = m.nu ? k + m.pc_off[a] : nullptr;
    }
    return v;
}


// Bytes of one tile-order scratch area: 64 ints of level counts and cursors,
// the order (an int per tile), the levels (a byte per tile).
constexpr size_t kOrderSlotBytes = 64 * sizeof(int) + mfadvr_ctx::kOrderTiles * (sizeof(int) + 1);

// The next tile-order scratch area for a launch of `tiles` ray tiles, when
// they are between 2 and 64 per resident warp (16 per SM): with fewer, every
// warp takes a tile or two and there is no tail to shorten; with more, the
// tail is a small part of the launch and row order keeps the tiles that run
// together close in the model (measured on a 3840x2160 frame: the order
// gained nothing).  Makes `s` wait for the area's previous launch; *slot = -1
// (no order) otherwise.  record_order marks the area's use once the launch
// that reads it is queued.
mfadvr_status take_order_slot(mfadvr_ctx *ctx, int64_t tiles, cudaStream_t s, int **order, unsigned char **level,
                              int **hist, int *slot)
{
    *slot = -1;
    *order = nullptr;
    *level = nullptr;
    *hist = nullptr;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) sms = 0;
    if (tiles > mfadvr_ctx::kOrderTiles || tiles < int64_t(2) * 16 * sms || tiles > int64_t(64) * 16 * sms)
        return MFADVR_OK;
    if (!ctx->order_pool) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, kOrderSlotBytes * mfadvr_ctx::kOrderSlots);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "tile-order allocation");
        for (unsigned i = 0; i < mfadvr_ctx::kOrderSlots && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&ctx->order_done[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (unsigned i = 0; i < mfadvr_ctx::kOrderSlots; ++i)
                if (ctx->order_done[i]) cudaEventDestroy(ctx->order_done[i]), ctx->order_done[i] = nullptr;
            cudaFree(p);
            return cuda_fail(ctx, e, "tile-order events");
        }
        ctx->order_pool = static_cast<char *>(p);
    }
    const unsigned k = ctx->next_order++ % mfadvr_ctx::kOrderSlots;
    cudaError_t e = cudaStreamWaitEvent(s, ctx->order_done[k], 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tile-order slot wait");
    char *base = ctx->order_pool + kOrderSlotBytes * k;
    *hist = reinterpret_cast<int *>(base);
    *order = reinterpret_cast<int *>(base + 64 * sizeof(int));
    *level = reinterpret_cast<unsigned char *>(base + 64 * sizeof(int) + mfadvr_ctx::kOrderTiles * sizeof(int));
    *slot = static_cast<int>(k);
    return MFADVR_OK;
}

// Points rs->tile_order (and its scratch) at an order area for this render
// (take_order_slot), or at nothing (row order).
mfadvr_status take_order(mfadvr_ctx *ctx, RenderSetup *rs, cudaStream_t s, int *slot)
{
    const int64_t tw = int64_t(1) << rs->tile_w_log2, th = 32 / tw;
    const int64_t tiles = ((rs->width + tw - 1) / tw) * ((rs->height + th - 1) / th);
    return take_order_slot(ctx, tiles, s, &rs->tile_order, &rs->tile_level, &rs->tile_hist, slot);
}

mfadvr_status record_order(mfadvr_ctx *ctx, int slot, cudaStream_t s)
{
    if (slot < 0) return MFADVR_OK;
    cudaError_t e = cudaEventRecord(ctx->order_done[slot], s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tile-order slot event");
    return MFADVR_OK;
}

mfadvr_status next_counter(mfadvr_ctx *ctx, int **out)
{
    if (!ctx->counters) {
        cudaError_t e = cudaMalloc(&ctx->counters, sizeof(int) * mfadvr_ctx::kCounters);
        if (e != cudaSuccess) {
            ctx->counters = nullptr;
            return cuda_fail(ctx, e, "counter allocation");
        }
    }
    *out = ctx->counters + (ctx->next_counter++ % mfadvr_ctx::kCounters);
    return MFADVR_OK;
}

mfadvr_status find_model(mfadvr_ctx *ctx, int32_t id, Model **out)
{
    auto it = ctx->models.find(id);
    if (it == ctx->models.end()) return fail(ctx, MFADVR_ENOTFOUND, "no model with id %d", id);
    *out = &it->second;
    return MFADVR_OK;
}

// Camera frame and per-pixel mapping in double, rounded once to FP32.
mfadvr_status make_setup(mfadvr_ctx *ctx, const Model &m, const mfadvr_camera *cam,
                         const mfadvr_render_params *rp, RenderSetup *rs)
{
    if (!cam || !rp) return fail(ctx, MFADVR_EINVAL, "camera and params must not be NULL");
    if (cam->kind != 0 && cam->kind != 1) return fail(ctx, MFADVR_EINVAL, "camera kind must be 0 or 1");
    if (!finite3(cam->eye) || !finite3(cam->center) || !finite3(cam->up))
        return fail(ctx, MFADVR_EINVAL, "camera vectors must be finite");
    if (cam->kind == 1 && !(cam->fovy_deg > 0.0f && cam->fovy_deg < 180.0f))
        return fail(ctx, MFADVR_EINVAL, "fovy_deg must be in (0, 180)");
    if (cam->kind == 0 && !(cam->ortho_height > 0.0f && std::isfinite(cam->ortho_height)))
        return fail(ctx, MFADVR_EINVAL, "ortho_height must be > 0");
    if (rp->width <= 0 || rp->height <= 0 || rp->width > 65536 || rp->height > 65536 ||
        static_cast<int64_t>(rp->width) * rp->height > (int64_t(1) << 30))
        return fail(ctx, MFADVR_EINVAL, "image sides must be in 1..65536 and width*height <= 2^30");
    if (!(rp->step > 0.0f) || !std::isfinite(rp->step)) return fail(ctx, MFADVR_EINVAL, "step must be > 0");
    {
        // Bound the samples on one ray (the chord of the box is at most its
        // diagonal) so that no launch can run unboundedly long.
        double diag2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double e = static_cast<double>(m.box_max[a]) - m.box_min[a];
            diag2 += e * e;
        }
        if (std::sqrt(diag2) / rp->step > static_cast<double>(1 << 24))
            return fail(ctx, MFADVR_EINVAL, "step gives more than 2^24 samples per ray");
    }
    if (!std::isfinite(rp->max_opacity)) return fail(ctx, MFADVR_EINVAL, "max_opacity must be finite");
    if (!std::isfinite(rp->ref_step)) return fail(ctx, MFADVR_EINVAL, "ref_step must be finite");
    if (!rp->tf_rgba || rp->tf_size < 1 || rp->tf_size > MFADVR_MAX_TF_SIZE)
        return fail(ctx, MFADVR_EINVAL, "tf_rgba must be set and tf_size in 1..%d", MFADVR_MAX_TF_SIZE);
    if (rp->shading != 0 && rp->shading != 1) return fail(ctx, MFADVR_EINVAL, "shading must be 0 or 1");
    if (!std::isfinite(rp->ka) || !std::isfinite(rp->kd) || !std::isfinite(rp->ks) ||
        !std::isfinite(rp->shininess) || rp->shininess < 0.0f)
        return fail(ctx, MFADVR_EINVAL, "ka, kd, ks must be finite and shininess >= 0");
    if (std::isinf(rp->tf_lo) || std::isinf(rp->tf_hi))
        return fail(ctx, MFADVR_EINVAL, "tf_lo/tf_hi must be finite or NaN");

    double f[3], up[3], r[3], u[3];
    for (int a = 0; a < 3; ++a) {
        f[a] = static_cast<double>(cam->center[a]) - cam->eye[a];
        up[a] = cam->up[a];
    }
    double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fl > 0.0)) return fail(ctx, MFADVR_EINVAL, "camera eye and center coincide");
    for (double &x : f) x /= fl;
    r[0] = up[1] * f[2] - up[2] * f[1];
    r[1] = up[2] * f[0] - up[0] * f[2];
    r[2] = up[0] * f[1] - up[1] * f[0];
    double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(rl > 1e-12)) return fail(ctx, MFADVR_EINVAL, "camera up is parallel to the view direction");
    for (double &x : r) x /= rl;
    u[0] = f[1] * r[2] - f[2] * r[1];
    u[1] = f[2] * r[0] - f[0] * r[2];
    u[2] = f[0] * r[1] - f[1] * r[0];

    const double W = rp->width, H = rp->height;
    double a, b;
    if (cam->kind == 0) {
        a = cam->ortho_height * W / (2.0 * H);
        b = cam->ortho_height / 2.0;
    } else {
        const double th = std::tan(cam->fovy_deg * (M_PI / 180.0) * 0.5);
        a = th * W / H;
        b = th;
    }
    std::memset(rs, 0, sizeof *rs);
    const double bs = basis_scale_host(m.p), bs3 = bs * bs * bs;
    rs->width = rp->width;
    rs->height = rp->height;
    rs->kind = cam->kind;
    for (int i = 0; i < 3; ++i) {
        rs->eye[i] = cam->eye[i];
        rs->fwd[i] = static_cast<float>(f[i]);
        rs->right[i] = static_cast<float>(r[i]);
        rs->up[i] = static_cast<float>(u[i]);
        rs->box_min[i] = m.box_min[i];
        rs->box_max[i] = m.box_max[i];
        const double ext = static_cast<double>(m.box_max[i]) - m.box_min[i];
        rs->inv_ext[i] = static_cast<float>(1.0 / ext);
        // uniform knots: lattice units (span k covers [k, k+1)); general
        // knots: parameter units, the span's inverse width applied per sample
        const double units = m.nu ? 1.0 : static_cast<double>(m.n[i] - m.p);
        rs->lat_scale[i] = static_cast<float>(units / ext);
        // rational models: the kernel forms f = A / W from scaled sums, so
        // its value and gradient carry neither the storage nor the basis scale
        rs->grad_scale[i] = static_cast<float>(units * (m.rational ? 1.0 : m.scale / bs3) / ext);
    }
    rs->sx_scale = static_cast<float>(2.0 * a / W);
    rs->sx_off = static_cast<float>(-a);
    rs->sy_scale = static_cast<float>(-2.0 * b / H);
    rs->sy_off = static_cast<float>(b);
    rs->step = rp->step;
    rs->max_opacity = rp->max_opacity;
    rs->correct_opacity = (rp->ref_step > 0.0f && rp->ref_step != rp->step) ? 1 : 0;
    rs->opacity_ratio = rs->correct_opacity ? static_cast<float>(static_cast<double>(rp->step) / rp->ref_step) : 1.0f;
    rs->tf_size = rp->tf_size;
    const double lo = std::isnan(rp->tf_lo) ? m.pmin : rp->tf_lo;
    const double hi = std::isnan(rp->tf_hi) ? m.pmax : rp->tf_hi;
    const double last = rp->tf_size > 1 ? rp->tf_size - 1 : 1;
    const double inv_range = hi > lo ? 1.0 / (hi - lo) : 0.0;
    rs->tf_a = static_cast<float>((m.rational ? 1.0 : static_cast<double>(m.scale) / bs3) * inv_range);
    rs->tf_b = static_cast<float>(-lo * inv_range);
    rs->shading = rp->shading;
    rs->ka = rp->ka;
    rs->kd = rp->kd;
    rs->ks = rp->ks;
    rs->shininess = rp->shininess;
    const double th = 1e-20 * m.pabs;
    rs->gthresh2 = static_cast<float>(th * th);
    rs->tile_w_log2 = 3;  // 8 x 4 pixel tiles unless tuned
    rs->ctas_per_sm = 0;
    return MFADVR_OK;
}

// A one-entry table is widened to two equal entries so the kernel's
// interpolation never reads past the end.
mfadvr_status stage_tf(mfadvr_ctx *ctx, const float *tf, int size, bool tf_on_host, RenderSetup *rs,
                       cudaStream_t stream)
{
    if (size >= 2 && !tf_on_host) {
        if (reinterpret_cast<uintptr_t>(tf) % 16 != 0)
            return fail(ctx, MFADVR_EINVAL, "tf_rgba must be 16-byte aligned");
        rs->tf = reinterpret_cast<const float4 *>(tf);
        return MFADVR_OK;
    }
    const int n = size >= 2 ? size : 2;
    cudaError_t e = ctx->st_aux.reserve(sizeof(float4) * n);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "staging allocation");
    float4 *dst = static_cast<float4 *>(ctx->st_aux.ptr);
    const cudaMemcpyKind kind = tf_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    e = cudaMemcpyAsync(dst, tf, sizeof(float4) * size, kind, stream);
    if (e == cudaSuccess && size == 1) e = cudaMemcpyAsync(dst + 1, tf, sizeof(float4), kind, stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "transfer-function copy");
    rs->tf = dst;
    rs->tf_size = n;
    return MFADVR_OK;
}

int ilog2_u64(uint64_t v)
{
    int r = 0;
    while (v > 1) {
        v >>= 1;
        ++r;
    }
    return r;
}

TuneKey tune_key(const Model &m, int width, int height)
{
    const uint64_t pts = static_cast<uint64_t>(m.n[0]) * m.n[1] * m.n[2];
    return TuneKey(m.p, m.d_poly ? kPolyForm : m.dtype, ilog2_u64(pts),
                   ilog2_u64(static_cast<uint64_t>(width) * height));
}

// Launch shape from the tuning table, if this key has been tuned.
mfadvr_status make_job(mfadvr_ctx *ctx, const mfadvr_render_job &jb, int index, RenderJob *out)
{
    Model *m = nullptr;
    if (mfadvr_status st = find_model(ctx, jb.model_id, &m)) return st;
    RenderSetup &rs = out->rs;
    if (mfadvr_status st = make_setup(ctx, *m, &jb.camera, &jb.params, &rs)) return st;
    apply_tuning(ctx, *m, &rs);
    if (jb.params.tf_size < 2 || reinterpret_cast<uintptr_t>(jb.params.tf_rgba) % 16 != 0)
        return fail(ctx, MFADVR_EINVAL, "job %d: tf_rgba must be 16-byte aligned with tf_size >= 2", index);
    if (!jb.rgba_dev || reinterpret_cast<uintptr_t>(jb.rgba_dev) % 16 != 0 ||
        reinterpret_cast<uintptr_t>(jb.nsamples_dev) % 4 != 0)
        return fail(ctx, MFADVR_EINVAL, "job %d: rgba must be 16-byte and nsamples 4-byte aligned", index);
    if (!is_device_ptr(jb.rgba_dev) || !is_device_ptr(jb.params.tf_rgba) ||
        (jb.nsamples_dev && !is_device_ptr(jb.nsamples_dev)))
        return fail(ctx, MFADVR_EINVAL, "job %d: rgba, tf_rgba and nsamples must be device pointers", index);
    rs.tf = reinterpret_cast<const float4 *>(jb.params.tf_rgba);
    rs.out = reinterpret_cast<float4 *>(jb.rgba_dev);
    rs.nsamples = jb.nsamples_dev;
    out->mv = view_of(*m);
    return MFADVR_OK;
}

std::vector<BatchGroup> pack_jobs(const RenderJob *jobs, int n, RenderJob *dst)
{
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    auto key = [&](int a) {
        const RenderJob &j = jobs[a];
        return std::make_tuple(j.mv.p, render_form_key(j.mv, j.rs.shading), j.rs.shading != 0, j.mv.nu != 0,
                               j.mv.rational != 0);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key(a) < key(b); });
    std::vector<BatchGroup> groups;
    for (int k = 0; k < n; ++k) {
        RenderJob jb = jobs[order[k]];
        const int grad = jb.rs.shading != 0 ? 1 : 0, nu = jb.mv.nu != 0 ? 1 : 0, rat = jb.mv.rational != 0 ? 1 : 0;
        const int form = render_form_key(jb.mv, jb.rs.shading);
        if (groups.empty() || groups.back().p != jb.mv.p || groups.back().dtype != form ||
            groups.back().grad != grad || groups.back().nu != nu || groups.back().rat != rat)
            groups.push_back({jb.mv.p, form, grad, nu, rat, k, 0, 0});
        BatchGroup &gr = groups.back();
        const int tw = 1 << jb.rs.tile_w_log2, th = 32 / tw;
        jb.tiles_x = (jb.rs.width + tw - 1) / tw;
        jb.tiles = jb.tiles_x * ((jb.rs.height + th - 1) / th);
        jb.tile_begin = gr.tiles;
        jb.pad = 0;
        gr.tiles += jb.tiles;
        gr.count += 1;
        dst[k] = jb;
    }
    return groups;
}

void apply_tuning(const mfadvr_ctx *ctx, const Model &m, RenderSetup *rs)
{
    auto it = ctx->tuning.find(tune_key(m, rs->width, rs->height));
    if (it == ctx->tuning.end()) return;
    rs->tile_w_log2 = ilog2_u64(static_cast<uint64_t>(it->second.tile_w));
    rs->ctas_per_sm = it->second.ctas_per_sm;
}

// ---- general (non-uniform) clamped knots --------------------------------

// A clamped knot vector of n+p+1 finite FP32 values: p+1 zeros, strictly
// increasing interior knots in (0, 1), p+1 ones.  Returns an empty string or
// the reason it is not one.
std::string knot_problem(const float *t, int n, int p)
{
    for (int i = 0; i < n + p + 1; ++i)
        if (!std::isfinite(t[i])) return "knots must be finite";
    for (int i = 0; i <= p; ++i)
        if (t[i] != 0.0f || t[n + i] != 1.0f) return "knots must start with p+1 zeros and end with p+1 ones";
    for (int i = p + 1; i <= n; ++i)
        if (!(t[i] > t[i - 1])) return "interior knots must increase strictly inside (0, 1)";
    return std::string();
}

// Per-span pieces of one axis with knot vector t (n+p+1 values, as FP64):
// the span-local positions of the 2P knots around each span, then the
// recurrence of pieces_from_knots, scaled by the device basis scale.
template <int P>
void axis_pieces(const std::vector<double> &t, int n, float *pieces)
{
    constexpr int S = GeneralPieces<P>::kStride;
    const double scale = basis_scale_host(P);
    for (int k = 0; k < n - P; ++k) {
        const int s = P + k;
        const double h = t[s + 1] - t[s];
        double kap[2 * P] = {};
        for (int j = 1 - P; j <= P; ++j) kap[j + P - 1] = (t[s + j] - t[s]) / h;
        double c[P + 1][P + 1] = {};
        pieces_from_knots<P>(kap, scale, c);
        float *dst = pieces + static_cast<size_t>(k) * S;
        for (int q = 0; q < S; ++q) dst[q] = 0.0f;
        for (int r = 0; r <= P; ++r)
            for (int e = 0; e <= P; ++e) dst[r * (P + 1) + e] = static_cast<float>(c[r][e]);
    }
}

void axis_pieces_p(int p, const std::vector<double> &t, int n, float *pieces)
{
    switch (p) {
    case 1: axis_pieces<1>(t, n, pieces); break;
    case 2: axis_pieces<2>(t, n, pieces); break;
    case 3: axis_pieces<3>(t, n, pieces); break;
    case 4: axis_pieces<4>(t, n, pieces); break;
    default: axis_pieces<5>(t, n, pieces); break;
    }
}

int pieces_stride(int p)
{
    switch (p) {
    case 1: return GeneralPieces<1>::kStride;
    case 2: return GeneralPieces<2>::kStride;
    case 3: return GeneralPieces<3>::kStride;
    case 4: return GeneralPieces<4>::kStride;
    default: return GeneralPieces<5>::kStride;
    }
}

// Knot vector t_0..t_{n+p} of axis a as the kernels use it: clamped uniform
// j/m (exact in lattice units) for uniform-knot models; for general-knot
// models the given knots, or j/m rounded to FP32 on axes given none.
std::vector<double> model_knots(const mfadvr_model_desc *desc, const Model &m, int a)
{
    const int p = m.p, n = m.n[a], mm = n - p;
    std::vector<double> t(static_cast<size_t>(n + p + 1));
    for (int i = 0; i < n + p + 1; ++i) {
        const int j = i < p ? 0 : (i > n ? mm : i - p);
        if (m.nu && desc->knots[a]) t[i] = desc->knots[a][i];
        else if (m.nu) t[i] = static_cast<float>(static_cast<double>(j) / mm);
        else t[i] = static_cast<double>(j) / mm;
    }
    return t;
}

// The span pieces of one axis about each span's centre, for the span
// polynomials: c[(k (P+1) + r) (P+1) + f] = coefficient of t^f, t = x - 1/2,
// of BasisScale N_r on span k (x the span's local coordinate), in FP64: the
// pieces of pieces_from_knots, then the Taylor shift
// x^e = sum_f binom(e, f) 2^(f-e) t^f.
template <int P>
std::vector<double> centred_axis_pieces(const std::vector<double> &t, int n)
{
    constexpr int K = P + 1;
    std::vector<double> out(static_cast<size_t>(n - P) * K * K);
    for (int k = 0; k < n - P; ++k) {
        const int s = P + k;
        const double h = t[s + 1] - t[s];
        double kap[2 * P] = {};
        for (int j = 1 - P; j <= P; ++j) kap[j + P - 1] = (t[s + j] - t[s]) / h;
        double c[K][K] = {};
        pieces_from_knots<P>(kap, basis_scale_host(P), c);
        for (int r = 0; r < K; ++r)
            for (int f = 0; f < K; ++f) {
                double sum = 0.0, binom = 1.0, half = 1.0;  // binom(e, f), 2^(f-e) for e = f, f+1, ...
                for (int e = f; e < K; ++e) {
                    sum += c[r][e] * binom * half;
                    binom = binom * (e + 1) / (e + 1 - f);
                    half *= 0.5;
                }
                out[(static_cast<size_t>(k) * K + r) * K + f] = sum;
            }
    }
    return out;
}

std::vector<double> centred_axis_pieces_p(int p, const std::vector<double> &t, int n)
{
    switch (p) {
    case 1: return centred_axis_pieces<1>(t, n);
    case 2: return centred_axis_pieces<2>(t, n);
    case 3: return centred_axis_pieces<3>(t, n);
    default: return centred_axis_pieces<4>(t, n);
    }
}

// Host image of a general-knot model's knot buffer: per axis the m+1
// breakpoints t_p..t_n, the m inverse widths, the 2m+1 lookup cells (int32:
// cell c holds the largest k with t_{p+k} <= c / 2m) and the m x stride
// pieces, each section starting on an 8-float (32-byte) boundary.  Axes
// without knots get the uniform knots j/m rounded to FP32.
std::vector<float> build_knot_buffer(const mfadvr_model_desc *desc, Model *m)
{
    auto up4 = [](size_t v) { return (v + 7) / 8 * 8; };
    const int p = m->p;
    std::vector<float> buf;
    for (int a = 0; a < 3; ++a) {
        const int n = m->n[a], mm = n - p;
        const std::vector<double> t = model_knots(desc, *m, a);
        m->brk_off[a] = buf.size();
        buf.resize(up4(buf.size() + mm + 1), 0.0f);
        for (int k = 0; k <= mm; ++k) buf[m->brk_off[a] + k] = static_cast<float>(t[p + k]);
        m->ih_off[a] = buf.size();
        buf.resize(up4(buf.size() + mm), 0.0f);
        for (int k = 0; k < mm; ++k)
            buf[m->ih_off[a] + k] = static_cast<float>(1.0 / (t[p + k + 1] - t[p + k]));
        const int G = 2 * mm;
        m->cell_off[a] = buf.size();
        buf.resize(up4(buf.size() + G + 1), 0.0f);
        for (int c = 0, k = 0; c <= G; ++c) {
            const double x = static_cast<double>(c) / G;
            while (k + 1 < mm && t[p + k + 1] <= x) ++k;
            const int32_t kc = k;
            std::memcpy(&buf[m->cell_off[a] + c], &kc, sizeof kc);
        }
        m->pc_off[a] = buf.size();
        buf.resize(buf.size() + static_cast<size_t>(mm) * pieces_stride(p), 0.0f);
        axis_pieces_p(p, t, n, buf.data() + m->pc_off[a]);
    }
    return buf;
}

}  // namespace api
}  // namespace mfadvr

// Render setup for a lattice that lives outside any context (the
// allocation-free entry point): FP32 values, scale 1, an explicit TF range,
// and a shading threshold of zero because max|P| is not known.  Errors go to
// the context-free last-error message.
mfadvr_status mfadvr::setup_for_lattice(int p, const int n[3], const float box_min[3], const float box_max[3],
                                         const mfadvr_camera *cam, const mfadvr_render_params *rp, RenderSetup *rs)
{
    Model m;
    m.p = p;
    m.dtype = MFADVR_F32;
    m.scale = 1.0f;
    for (int a = 0; a < 3; ++a) {
        m.n[a] = n[a];
        m.box_min[a] = box_min[a];
        m.box_max[a] = box_max[a];
    }
    return make_setup(nullptr, m, cam, rp, rs);
}

mfadvr_status mfadvr::fail_noctx(mfadvr_status st, const char *msg) { return fail(nullptr, st, "%s", msg); }

namespace {

// The device address of a page-locked (pinned, registered) host buffer, or
// NULL for any other pointer.
void *pinned_alias(const void *h)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Output bytes per point of a query, 0 for an unknown query.
size_t query_out_bytes(int32_t query)
{
    switch (query) {
    case MFADVR_QUERY_VALUE: return 4;
    case MFADVR_QUERY_GRADIENT: return 12;
    case MFADVR_QUERY_BOTH: return 16;
    case MFADVR_QUERY_HESSIAN: return 40;
    default: return 0;
    }
}

mfadvr_status query_device(mfadvr_ctx *ctx, int32_t model_id, const float *params_dev, int64_t n, int32_t query,
                           float *out_dev, int32_t *spans_dev, void *stream)
{
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    Model *m = nullptr;
    if (mfadvr_status st = find_model(ctx, model_id, &m)) return st;
    if (query_out_bytes(query) == 0) return fail(ctx, MFADVR_EINVAL, "query must be 1 (value), 2 (gradient), 3 or 4");
    if (n < 0) return fail(ctx, MFADVR_EINVAL, "n must be >= 0");
    if (n == 0) return MFADVR_OK;
    if (!params_dev || !out_dev) return fail(ctx, MFADVR_EINVAL, "params and out must not be NULL");
    const uintptr_t out_align = query == MFADVR_QUERY_BOTH ? 16 : 4;
    if (reinterpret_cast<uintptr_t>(out_dev) % out_align != 0 || reinterpret_cast<uintptr_t>(params_dev) % 4 != 0 ||
        reinterpret_cast<uintptr_t>(spans_dev) % 4 != 0)
        return fail(ctx, MFADVR_EINVAL, "out must be %u-byte aligned, params and spans 4-byte aligned",
                    static_cast<unsigned>(out_align));
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "cudaSetDevice");
    if (!is_device_ptr(params_dev) || !is_device_ptr(out_dev) || (spans_dev && !is_device_ptr(spans_dev)))
        return fail(ctx, MFADVR_EINVAL, "params, out and spans must be device pointers");
    cudaError_t e = launch_eval_points(view_of(*m), params_dev, n, out_dev, query, spans_dev,
                                       static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "eval_points launch");
    return MFADVR_OK;
}

// Device addresses of a query's page-locked host buffers.
struct HostAliases {
    const float *params = nullptr;
    float *out = nullptr;
    int32_t *spans = nullptr;
};

// True when params, out (and spans, when given) are page-locked host memory
// and out is aligned for the query's output rows.
bool host_aliases(const float *params_host, float *out_host, int32_t *spans_host, int32_t query, HostAliases *a)
{
    a->params = static_cast<const float *>(pinned_alias(params_host));
    a->out = static_cast<float *>(pinned_alias(out_host));
    a->spans = spans_host ? static_cast<int32_t *>(pinned_alias(spans_host)) : nullptr;
    const uintptr_t align = query == MFADVR_QUERY_BOTH ? 16 : 4;
    return a->params && a->out && (!spans_host || a->spans) && reinterpret_cast<uintptr_t>(a->out) % align == 0 &&
           reinterpret_cast<uintptr_t>(a->params) % 4 == 0 && reinterpret_cast<uintptr_t>(a->spans) % 4 == 0;
}

// Argument checks shared by the host-buffer queries; *skip is set for n = 0.
mfadvr_status check_host_query(mfadvr_ctx *ctx, int32_t model_id, const float *params_host, int64_t n,
                               int32_t query, const float *out_host, Model **m, bool *skip)
{
    *skip = false;
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    if (mfadvr_status st = find_model(ctx, model_id, m)) return st;
    if (query_out_bytes(query) == 0) return fail(ctx, MFADVR_EINVAL, "query must be 1 (value), 2 (gradient), 3 or 4");
    if (n < 0) return fail(ctx, MFADVR_EINVAL, "n must be >= 0");
    *skip = n == 0;
    if (n > 0 && (!params_host || !out_host)) return fail(ctx, MFADVR_EINVAL, "params and out must not be NULL");
    return MFADVR_OK;
}

mfadvr_status query_host_async(mfadvr_ctx *ctx, int32_t model_id, const float *params_host, int64_t n,
                               int32_t query, float *out_host, int32_t *spans_host, int32_t max_ctas, void *stream)
{
    Model *m = nullptr;
    bool skip = false;
    if (mfadvr_status st = check_host_query(ctx, model_id, params_host, n, query, out_host, &m, &skip)) return st;
    if (max_ctas < 0) return fail(ctx, MFADVR_EINVAL, "max_ctas must be >= 0");
    if (skip) return MFADVR_OK;
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "cudaSetDevice");
    HostAliases z;
    if (!host_aliases(params_host, out_host, spans_host, query, &z))
        return fail(ctx, MFADVR_EINVAL, "params, out and spans must be page-locked host memory, out aligned to %d bytes",
                    query == MFADVR_QUERY_BOTH ? 16 : 4);
    const cudaError_t e = launch_eval_points(view_of(*m), z.params, n, z.out, query, z.spans,
                                             static_cast<cudaStream_t>(stream), max_ctas);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "query_points_host_async");
    return MFADVR_OK;
}

mfadvr_status query_host(mfadvr_ctx *ctx, int32_t model_id, const float *params_host, int64_t n, int32_t query,
                         float *out_host, int32_t *spans_host, void *stream)
{
    Model *m = nullptr;
    bool skip = false;
    if (mfadvr_status st = check_host_query(ctx, model_id, params_host, n, query, out_host, &m, &skip)) return st;
    if (skip) return MFADVR_OK;
    const size_t per = query_out_bytes(query);
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        // Pinned (page-locked, registered) host buffers: the kernel reads the
        // points from and writes the results to them directly over the
        // host link, with no staging copies.  Other buffers take the chunked
        // copy pipeline below.
        HostAliases z;
        if (host_aliases(params_host, out_host, spans_host, query, &z)) {
            cudaError_t e = launch_eval_points(view_of(*m), z.params, n, z.out, query, z.spans, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "eval_points_host");
            return MFADVR_OK;
        }
    }
    const size_t in_b = static_cast<size_t>(n) * 12;
    const size_t out_b = (static_cast<size_t>(n) * per + 15) / 16 * 16;
    const size_t sp_b = spans_host ? static_cast<size_t>(n) * 12 : 0;
    cudaError_t e = ctx->st_in.reserve(in_b);
    if (e == cudaSuccess) e = ctx->st_out.reserve(out_b + sp_b);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "staging allocation");
    float *d_in = static_cast<float *>(ctx->st_in.ptr);
    float *d_out = static_cast<float *>(ctx->st_out.ptr);
    int32_t *d_sp = spans_host ? reinterpret_cast<int32_t *>(static_cast<char *>(ctx->st_out.ptr) + out_b) : nullptr;
    // The points go through in 16 chunks on the context's pipe streams: chunk c
    // is copied in, evaluated and copied out on pipe[c % kPipes], so the
    // copy-in of one chunk, the kernel of another and the copy-out of a third
    // overlap.  The pipes start after the work already queued on `s`, and the
    // call returns when all of them have finished.
    for (int q = 0; q < mfadvr_ctx::kPipes && e == cudaSuccess; ++q)
        if (!ctx->pipe[q]) e = cudaStreamCreateWithFlags(&ctx->pipe[q], cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->pipe_start) e = cudaEventCreateWithFlags(&ctx->pipe_start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->pipe_start, s);
    for (int q = 0; q < mfadvr_ctx::kPipes && e == cudaSuccess; ++q)
        e = cudaStreamWaitEvent(ctx->pipe[q], ctx->pipe_start, 0);
    const int64_t kChunks = n >= (int64_t(1) << 20) ? 16 : 1;
    const int64_t chunk = (n + kChunks - 1) / kChunks;
    const ModelView mv = view_of(*m);
    for (int64_t c = 0, off = 0; off < n && e == cudaSuccess; ++c, off += chunk) {
        const int64_t cnt = n - off < chunk ? n - off : chunk;
        cudaStream_t ps = ctx->pipe[c % mfadvr_ctx::kPipes];
        const size_t o = static_cast<size_t>(off);
        e = cudaMemcpyAsync(d_in + 3 * o, params_host + 3 * o, static_cast<size_t>(cnt) * 12, cudaMemcpyHostToDevice,
                            ps);
        float *dout = reinterpret_cast<float *>(reinterpret_cast<char *>(d_out) + o * per);
        if (e == cudaSuccess)
            e = launch_eval_points(mv, d_in + 3 * o, cnt, dout, query, d_sp ? d_sp + 3 * o : nullptr, ps);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(reinterpret_cast<char *>(out_host) + o * per, dout, static_cast<size_t>(cnt) * per,
                                cudaMemcpyDeviceToHost, ps);
        if (e == cudaSuccess && d_sp)
            e = cudaMemcpyAsync(spans_host + 3 * o, d_sp + 3 * o, static_cast<size_t>(cnt) * 12, cudaMemcpyDeviceToHost,
                                ps);
    }
    for (int q = 0; q < mfadvr_ctx::kPipes; ++q) {
        const cudaError_t e2 = cudaStreamSynchronize(ctx->pipe[q]);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "eval_points_host");
    return MFADVR_OK;
}

// Uploads each axis's span pieces about the span centres (FP64,
// centred_axis_pieces) into one device buffer *buf; cpd[a] points at axis a's.
cudaError_t upload_centred_pieces(const mfadvr_model_desc *desc, const Model &m, void **buf, const double *cpd[3])
{
    std::vector<double> cp[3];
    size_t total = 0;
    for (int a = 0; a < 3; ++a) {
        cp[a] = centred_axis_pieces_p(m.p, model_knots(desc, m, a), m.n[a]);
        total += cp[a].size();
    }
    cudaError_t e = cudaMalloc(buf, total * sizeof(double));
    for (size_t a = 0, off = 0; a < 3 && e == cudaSuccess; off += cp[a].size(), ++a) {
        double *dst = static_cast<double *>(*buf) + off;
        cpd[a] = dst;
        e = cudaMemcpy(dst, cp[a].data(), cp[a].size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    return e;
}

// The row array of one FP32 source lattice in device memory and, when poly is
// given, its span polynomials.
cudaError_t build_arrays(const Model &m, const float *src, void *rows, void *poly, float inv_scale,
                         const double *const cpd[3])
{
    cudaError_t e = launch_build_rows(src, rows, m.n[0], m.n[1], m.n[2], m.dtype, inv_scale, nullptr);
    if (e == cudaSuccess && poly) e = launch_build_poly(src, poly, m.p, m.n[0], m.n[1], m.n[2], cpd, nullptr);
    return e;
}

}  // namespace

// Largest span-polynomial array the AUTO render form builds (MFADVR_FORM_POWER
// builds any size within the HBM budget).
constexpr uint64_t kAutoPolyBytes = uint64_t(4) << 30;

extern "C" {

mfadvr_status mfadvr_create(mfadvr_ctx **out, int device, uint64_t hbm_budget_bytes)
{
    if (!out) return fail(nullptr, MFADVR_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (device < 0) return fail(nullptr, MFADVR_EINVAL, "device must be >= 0");
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return fail(nullptr, MFADVR_ECUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device >= count) return fail(nullptr, MFADVR_ECUDA, "device %d not present (%d devices)", device, count);
    mfadvr_ctx *ctx = new (std::nothrow) mfadvr_ctx();
    if (!ctx) return fail(nullptr, MFADVR_ENOMEM, "out of host memory");
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    *out = ctx;
    return MFADVR_OK;
}

mfadvr_status mfadvr_destroy(mfadvr_ctx *ctx)
{
    if (!ctx) return MFADVR_OK;
    stop_server(ctx);
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        for (auto &kv : ctx->models) {
            if (kv.second.d_rows) cudaFree(kv.second.d_rows);
            if (kv.second.d_knots) cudaFree(kv.second.d_knots);
            if (kv.second.d_wrows) cudaFree(kv.second.d_wrows);
            if (kv.second.d_poly) cudaFree(kv.second.d_poly);
        }
        if (ctx->counters) cudaFree(ctx->counters);
        if (ctx->order_pool) cudaFree(ctx->order_pool);
        for (unsigned i = 0; i < mfadvr_ctx::kOrderSlots; ++i)
            if (ctx->order_done[i]) cudaEventDestroy(ctx->order_done[i]);
        if (ctx->d_jobs) cudaFree(ctx->d_jobs);
        if (ctx->h_jobs) cudaFreeHost(ctx->h_jobs);
        for (auto &e : ctx->job_done)
            if (e) cudaEventDestroy(e);
        for (auto &q : ctx->pipe)
            if (q) cudaStreamDestroy(q);
        if (ctx->pipe_start) cudaEventDestroy(ctx->pipe_start);
        ctx->st_in.release();
        ctx->st_out.release();
        ctx->st_aux.release();
    }
    delete ctx;
    return MFADVR_OK;
}

// Scale s of a 16-bit array whose largest magnitude is amax; the array holds
// P / s.  BF16 (FP32's exponent range): s = amax.  FP16: a power of two that
// puts amax in [2^14, 2^15), the top binade FP16 holds, so that values down
// to about 2^-29 amax stay normal numbers (with s = amax, everything below
// 6.1e-5 amax was subnormal: the near-flat regions of a field lost their
// precision, and their shading normals with it); multiplying by 1/s is then
// exact.  FP32 storage, or an all-zero array: 1.
static float storage_scale(int storage, float amax)
{
    if (storage == MFADVR_F32 || !(amax > 0.0f)) return 1.0f;
    if (storage == MFADVR_BF16) return amax;
    int e = 0;
    std::frexp(amax, &e);  // amax = f 2^e, f in [0.5, 1)
    return std::ldexp(1.0f, e - 15);
}

mfadvr_status mfadvr_load_model(mfadvr_ctx *ctx, const mfadvr_model_desc *desc, int32_t *model_id)
{
    TraceRange trace("mfadvr_load_model");
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    if (!desc || !model_id) return fail(ctx, MFADVR_EINVAL, "desc and model_id must not be NULL");
    if (!desc->ctrl) return fail(ctx, MFADVR_EINVAL, "desc->ctrl must not be NULL");
    if (desc->storage != MFADVR_F32 && desc->storage != MFADVR_F16 && desc->storage != MFADVR_BF16)
        return fail(ctx, MFADVR_EINVAL, "unknown storage type %d", static_cast<int>(desc->storage));
    for (int a = 0; a < 3; ++a) {
        if (desc->degree[a] < 1) return fail(ctx, MFADVR_EINVAL, "degree must be >= 1");
        if (desc->ncp[a] < desc->degree[a] + 1 || desc->ncp[a] > (1 << 24))
            return fail(ctx, MFADVR_EINVAL, "ncp[%d] = %d must be in degree+1..2^24", a, desc->ncp[a]);
        if (!std::isfinite(desc->box_min[a]) || !std::isfinite(desc->box_max[a]) ||
            !(desc->box_max[a] > desc->box_min[a]))
            return fail(ctx, MFADVR_EINVAL, "box_max must exceed box_min on every axis");
    }
    if (desc->degree[0] > MFADVR_MAX_DEGREE || desc->degree[1] > MFADVR_MAX_DEGREE ||
        desc->degree[2] > MFADVR_MAX_DEGREE)
        return fail(ctx, MFADVR_EUNSUPPORTED, "degree above %d", MFADVR_MAX_DEGREE);
    if (desc->degree[0] != desc->degree[1] || desc->degree[0] != desc->degree[2])
        return fail(ctx, MFADVR_EUNSUPPORTED, "degrees must be equal on the three axes");
    if (desc->render_form < MFADVR_FORM_AUTO || desc->render_form > MFADVR_FORM_POWER)
        return fail(ctx, MFADVR_EINVAL, "unknown render form %d", static_cast<int>(desc->render_form));
    for (int a = 0; a < 3; ++a) {
        if (!desc->knots[a]) continue;
        const std::string why = knot_problem(desc->knots[a], desc->ncp[a], desc->degree[a]);
        if (!why.empty()) return fail(ctx, MFADVR_EINVAL, "knots[%d]: %s", a, why.c_str());
    }

    // n0 n1 <= 2^48 cannot wrap; the third side is checked by division so
    // that no wrapped product of three sides passes the limit.
    const uint64_t ncp01 = static_cast<uint64_t>(desc->ncp[0]) * static_cast<uint64_t>(desc->ncp[1]);
    if (ncp01 > ((uint64_t(1) << 31) - 1) / static_cast<uint64_t>(desc->ncp[2]))
        return fail(ctx, MFADVR_EUNSUPPORTED, "lattices of 2^31 or more control points are not supported");
    const uint64_t count = ncp01 * static_cast<uint64_t>(desc->ncp[2]);
    float pmin = INFINITY, pmax = -INFINITY, pabs = 0.0f;
    for (uint64_t i = 0; i < count; ++i) {
        const float v = desc->ctrl[i];
        if (!std::isfinite(v)) return fail(ctx, MFADVR_EINVAL, "control point %llu is not finite",
                                           static_cast<unsigned long long>(i));
        pmin = v < pmin ? v : pmin;
        pmax = v > pmax ? v : pmax;
        pabs = std::fabs(v) > pabs ? std::fabs(v) : pabs;
    }
    // Rational model: the weighted points w P go to the row array in place
    // of P, the weights to a second one.  Convex weights keep f inside
    // [min P, max P], so the TF domain stays that of P.
    std::vector<float> wctrl;
    float qabs = pabs, wmax = 1.0f;
    if (desc->weights) {
        wctrl.resize(count);
        qabs = 0.0f;
        wmax = 0.0f;
        for (uint64_t i = 0; i < count; ++i) {
            const float w = desc->weights[i];
            if (!(w > 0.0f) || !std::isfinite(w))
                return fail(ctx, MFADVR_EINVAL, "weight %llu is not positive and finite",
                            static_cast<unsigned long long>(i));
            wctrl[i] = static_cast<float>(static_cast<double>(w) * desc->ctrl[i]);
            if (!std::isfinite(wctrl[i])) return fail(ctx, MFADVR_EINVAL, "weight x control point overflows");
            qabs = std::fabs(wctrl[i]) > qabs ? std::fabs(wctrl[i]) : qabs;
            wmax = w > wmax ? w : wmax;
        }
    }
    Model m;
    m.p = desc->degree[0];
    m.dtype = desc->storage;
    m.rational = desc->weights ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        m.n[a] = desc->ncp[a];
        m.box_min[a] = desc->box_min[a];
        m.box_max[a] = desc->box_max[a];
    }
    m.pmin = pmin;
    m.pmax = pmax;
    m.pabs = pabs;
    m.scale = storage_scale(desc->storage, qabs);
    m.wscale = m.rational ? storage_scale(desc->storage, wmax) : 1.0f;
    const uint64_t rows_b = count * row_entry_bytes(m.dtype);
    m.bytes = rows_b * (m.rational ? 2 : 1);
    std::vector<float> knot_buf;
    if (desc->knots[0] || desc->knots[1] || desc->knots[2]) {
        m.nu = 1;
        knot_buf = build_knot_buffer(desc, &m);
        m.knot_bytes = knot_buf.size() * sizeof(float);
        m.bytes += m.knot_bytes;
    }
    if (ctx->budget && ctx->used + m.bytes > ctx->budget)
        return fail(ctx, MFADVR_ENOMEM, "model of %llu bytes exceeds the HBM budget (%llu of %llu used)",
                    static_cast<unsigned long long>(m.bytes), static_cast<unsigned long long>(ctx->used),
                    static_cast<unsigned long long>(ctx->budget));
    // POWER render form: span polynomials beside the row array, where the
    // model allows them (AUTO: and where they fit the budget).
    // degree 4: plain models only (a rational one keeps no register cache there)
    // The kernels place a sample by its offset from the span's centre, index
    // + 1/2, exact in FP32 below 2^22 spans per axis.
    const bool poly_ok = m.dtype == MFADVR_F32 && (m.p <= 3 || (m.p == 4 && !m.rational)) &&
                         m.n[0] - m.p < (1 << 22) && m.n[1] - m.p < (1 << 22) && m.n[2] - m.p < (1 << 22);
    const uint64_t poly_b = poly_ok ? static_cast<uint64_t>(m.n[0] - m.p) * (m.n[1] - m.p) * (m.n[2] - m.p) *
                                          static_cast<uint64_t>(poly_cell_bytes(m.p)) * (m.rational ? 2 : 1)
                                    : 0;
    if (desc->render_form == MFADVR_FORM_POWER && !poly_ok)
        return fail(ctx, MFADVR_EUNSUPPORTED,
                    "the power render form needs FP32 storage, degree <= 3 (degree 4: without weights) and "
                    "fewer than 2^22 spans per axis");
    const bool poly_fits = !ctx->budget || ctx->used + m.bytes + poly_b <= ctx->budget;
    if (desc->render_form == MFADVR_FORM_POWER && !poly_fits)
        return fail(ctx, MFADVR_ENOMEM, "span polynomials of %llu bytes exceed the HBM budget",
                    static_cast<unsigned long long>(poly_b));
    const bool want_poly = poly_ok && poly_fits &&
                           (desc->render_form == MFADVR_FORM_POWER ||
                            (desc->render_form == MFADVR_FORM_AUTO && poly_b <= kAutoPolyBytes));

    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "cudaSetDevice");
    cudaError_t e = cudaMalloc(&m.d_rows, rows_b);
    if (e != cudaSuccess) {
        cudaGetLastError();
        m.d_rows = nullptr;
        return fail(ctx, MFADVR_ENOMEM, "cudaMalloc(%llu): %s", static_cast<unsigned long long>(m.bytes),
                    cudaGetErrorString(e));
    }
    if (m.nu) {
        e = cudaMalloc(&m.d_knots, m.knot_bytes);
        if (e == cudaSuccess) e = cudaMemcpy(m.d_knots, knot_buf.data(), m.knot_bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(m.d_rows);
            if (m.d_knots) cudaFree(m.d_knots);
            return fail(ctx, MFADVR_ENOMEM, "knot tables of %llu bytes: %s",
                        static_cast<unsigned long long>(m.knot_bytes), cudaGetErrorString(e));
        }
    }
    void *tmp = nullptr;
    if (m.rational) e = cudaMalloc(&m.d_wrows, rows_b);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, count * sizeof(float));
    // Power form: the span polynomials, beside the row array (a rational
    // model has two: of w P, then of w), built from each axis's span pieces
    // about the span centres (d_cp).  AUTO drops to the B-spline form when
    // the allocation fails.
    void *d_cp = nullptr;
    const double *cpd[3] = {nullptr, nullptr, nullptr};
    if (e == cudaSuccess && want_poly) {
        const cudaError_t ep = cudaMalloc(&m.d_poly, poly_b);
        if (ep == cudaSuccess) {
            m.poly_bytes = poly_b;
            m.bytes += poly_b;
            e = upload_centred_pieces(desc, m, &d_cp, cpd);
        } else {
            cudaGetLastError();
            m.d_poly = nullptr;
            if (desc->render_form == MFADVR_FORM_POWER) {
                cudaFree(m.d_rows);
                if (m.d_knots) cudaFree(m.d_knots);
                if (m.d_wrows) cudaFree(m.d_wrows);
                if (tmp) cudaFree(tmp);
                return fail(ctx, MFADVR_ENOMEM, "span polynomials: cudaMalloc(%llu): %s",
                            static_cast<unsigned long long>(poly_b), cudaGetErrorString(ep));
            }
        }
    }
    // the arrays of w P (or P), then those of the weights: tmp holds one source
    // lattice at a time
    char *poly = static_cast<char *>(m.d_poly);
    const uint64_t poly_one = m.rational ? poly_b / 2 : poly_b;  // bytes of one polynomial array
    const float *rows_src = m.rational ? wctrl.data() : desc->ctrl;
    if (e == cudaSuccess) e = cudaMemcpy(tmp, rows_src, count * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = build_arrays(m, static_cast<const float *>(tmp), m.d_rows, poly, 1.0f / m.scale, cpd);
    if (e == cudaSuccess && m.rational) {
        e = cudaDeviceSynchronize();  // tmp is reused
        if (e == cudaSuccess) e = cudaMemcpy(tmp, desc->weights, count * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = build_arrays(m, static_cast<const float *>(tmp), m.d_wrows, poly ? poly + poly_one : nullptr,
                             1.0f / m.wscale, cpd);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (d_cp) cudaFree(d_cp);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) {
        cudaFree(m.d_rows);
        if (m.d_knots) cudaFree(m.d_knots);
        if (m.d_wrows) cudaFree(m.d_wrows);
        if (m.d_poly) cudaFree(m.d_poly);
        return cuda_fail(ctx, e, "model upload");
    }
    const int32_t id = ctx->next_id++;
    ctx->models[id] = m;
    ctx->used += m.bytes;
    *model_id = id;
    return MFADVR_OK;
}

mfadvr_status mfadvr_unload_model(mfadvr_ctx *ctx, int32_t model_id)
{
    TraceRange trace("mfadvr_unload_model");
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    Model *m = nullptr;
    if (mfadvr_status st = find_model(ctx, model_id, &m)) return st;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    cudaFree(m->d_rows);
    if (m->d_knots) cudaFree(m->d_knots);
    if (m->d_wrows) cudaFree(m->d_wrows);
    if (m->d_poly) cudaFree(m->d_poly);
    ctx->used -= m->bytes;
    ctx->models.erase(model_id);
    return MFADVR_OK;
}

mfadvr_status mfadvr_model_info(mfadvr_ctx *ctx, int32_t model_id, float *pmin, float *pmax, float *scale,
                                uint64_t *bytes)
{
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    Model *m = nullptr;
    if (mfadvr_status st = find_model(ctx, model_id, &m)) return st;
    if (pmin) *pmin = m->pmin;
    if (pmax) *pmax = m->pmax;
    if (scale) *scale = m->scale;
    if (bytes) *bytes = m->bytes;
    return MFADVR_OK;
}

mfadvr_status mfadvr_eval_points(mfadvr_ctx *ctx, int32_t model_id, const float *params_dev, int64_t n,
                                 float *out_dev, int32_t *spans_dev, void *stream)
{
    TraceRange trace("mfadvr_eval_points");
    return query_device(ctx, model_id, params_dev, n, MFADVR_QUERY_BOTH, out_dev, spans_dev, stream);
}

mfadvr_status mfadvr_eval_points_host(mfadvr_ctx *ctx, int32_t model_id, const float *params_host, int64_t n,
                                      float *out_host, int32_t *spans_host, void *stream)
{
    TraceRange trace("mfadvr_eval_points_host");
    return query_host(ctx, model_id, params_host, n, MFADVR_QUERY_BOTH, out_host, spans_host, stream);
}

mfadvr_status mfadvr_query_points(mfadvr_ctx *ctx, int32_t model_id, const float *params_dev, int64_t n,
                                  int32_t query, float *out_dev, int32_t *spans_dev, void *stream)
{
    TraceRange trace("mfadvr_query_points");
    return query_device(ctx, model_id, params_dev, n, query, out_dev, spans_dev, stream);
}

mfadvr_status mfadvr_query_points_host(mfadvr_ctx *ctx, int32_t model_id, const float *params_host, int64_t n,
                                       int32_t query, float *out_host, int32_t *spans_host, void *stream)
{
    TraceRange trace("mfadvr_query_points_host");
    return query_host(ctx, model_id, params_host, n, query, out_host, spans_host, stream);
}

mfadvr_status mfadvr_query_points_host_async(mfadvr_ctx *ctx, int32_t model_id, const float *params_host, int64_t n,
                                             int32_t query, float *out_host, int32_t *spans_host, int32_t max_ctas,
                                             void *stream)
{
    TraceRange trace("mfadvr_query_points_host_async");
    return query_host_async(ctx, model_id, params_host, n, query, out_host, spans_host, max_ctas, stream);
}

mfadvr_status mfadvr_render(mfadvr_ctx *ctx, int32_t model_id, const mfadvr_camera *camera,
                            const mfadvr_render_params *params, float *rgba_dev, int32_t *nsamples_dev, void *stream)
{
    TraceRange trace("mfadvr_render");
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    Model *m = nullptr;
    if (mfadvr_status st = find_model(ctx, model_id, &m)) return st;
    RenderSetup rs;
    if (mfadvr_status st = make_setup(ctx, *m, camera, params, &rs)) return st;
    apply_tuning(ctx, *m, &rs);
    if (!rgba_dev || reinterpret_cast<uintptr_t>(rgba_dev) % 16 != 0)
        return fail(ctx, MFADVR_EINVAL, "rgba must be a 16-byte aligned device pointer");
    if (reinterpret_cast<uintptr_t>(nsamples_dev) % 4 != 0)
        return fail(ctx, MFADVR_EINVAL, "nsamples must be 4-byte aligned");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "cudaSetDevice");
    if (!is_device_ptr(rgba_dev) || !is_device_ptr(params->tf_rgba) || (nsamples_dev && !is_device_ptr(nsamples_dev)))
        return fail(ctx, MFADVR_EINVAL, "rgba, tf_rgba and nsamples must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mfadvr_status st = stage_tf(ctx, params->tf_rgba, params->tf_size, false, &rs, s)) return st;
    rs.out = reinterpret_cast<float4 *>(rgba_dev);
    rs.nsamples = nsamples_dev;
    int *counter = nullptr;
    if (mfadvr_status st = next_counter(ctx, &counter)) return st;
    int slot = -1;
    if (mfadvr_status st = take_order(ctx, &rs, s, &slot)) return st;
    cudaError_t e = launch_render(view_of(*m), rs, counter, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "render launch");
    return record_order(ctx, slot, s);
}

mfadvr_status mfadvr_render_trace(mfadvr_ctx *ctx, int32_t model_id, const mfadvr_camera *camera,
                                  const mfadvr_render_params *params, float *rgba_dev, int32_t *nsamples_dev,
                                  int32_t max_samples, float *pos_dev, int32_t *span_dev, void *stream)
{
    TraceRange trace("mfadvr_render_trace");
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    Model *m = nullptr;
    if (mfadvr_status st = find_model(ctx, model_id, &m)) return st;
    RenderSetup rs;
    if (mfadvr_status st = make_setup(ctx, *m, camera, params, &rs)) return st;
    apply_tuning(ctx, *m, &rs);
    if (m->dtype != MFADVR_F32 || m->rational || params->shading == 0)
        return fail(ctx, MFADVR_EUNSUPPORTED, "the render trace covers shaded renders of plain FP32 models");
    if (max_samples < 1 || static_cast<int64_t>(params->width) * params->height * max_samples > (int64_t(1) << 24))
        return fail(ctx, MFADVR_EINVAL, "max_samples must be >= 1 and width*height*max_samples <= 2^24");
    if (!rgba_dev || reinterpret_cast<uintptr_t>(rgba_dev) % 16 != 0 || !pos_dev || !span_dev ||
        reinterpret_cast<uintptr_t>(pos_dev) % 4 != 0 || reinterpret_cast<uintptr_t>(span_dev) % 4 != 0 ||
        reinterpret_cast<uintptr_t>(nsamples_dev) % 4 != 0)
        return fail(ctx, MFADVR_EINVAL, "rgba (16-byte aligned), pos and span must be set; pos, span, nsamples 4-byte aligned");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "cudaSetDevice");
    if (!is_device_ptr(rgba_dev) || !is_device_ptr(params->tf_rgba) || !is_device_ptr(pos_dev) ||
        !is_device_ptr(span_dev) || (nsamples_dev && !is_device_ptr(nsamples_dev)))
        return fail(ctx, MFADVR_EINVAL, "rgba, tf_rgba, pos, span and nsamples must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mfadvr_status st = stage_tf(ctx, params->tf_rgba, params->tf_size, false, &rs, s)) return st;
    rs.out = reinterpret_cast<float4 *>(rgba_dev);
    rs.nsamples = nsamples_dev;
    int *counter = nullptr;
    if (mfadvr_status st = next_counter(ctx, &counter)) return st;
    cudaError_t e = launch_render_trace(view_of(*m), rs, counter, TraceOn{pos_dev, span_dev, max_samples}, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "render trace launch");
    return MFADVR_OK;
}

mfadvr_status mfadvr_render_host(mfadvr_ctx *ctx, int32_t model_id, const mfadvr_camera *camera,
                                 const mfadvr_render_params *params, float *rgba_host, int32_t *nsamples_host,
                                 void *stream)
{
    TraceRange trace("mfadvr_render_host");
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    Model *m = nullptr;
    if (mfadvr_status st = find_model(ctx, model_id, &m)) return st;
    RenderSetup rs;
    if (mfadvr_status st = make_setup(ctx, *m, camera, params, &rs)) return st;
    apply_tuning(ctx, *m, &rs);
    if (!rgba_host) return fail(ctx, MFADVR_EINVAL, "rgba must not be NULL");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mfadvr_status st = stage_tf(ctx, params->tf_rgba, params->tf_size, true, &rs, s)) return st;
    const size_t npix = static_cast<size_t>(params->width) * params->height;
    const size_t img_b = npix * 16, ns_b = nsamples_host ? npix * 4 : 0;
    // page-locked outputs are written by the kernel directly; others staged
    void *zimg = pinned_alias(rgba_host), *zns = nsamples_host ? pinned_alias(nsamples_host) : nullptr;
    const bool direct = zimg && reinterpret_cast<uintptr_t>(zimg) % 16 == 0 && (!nsamples_host || zns);
    cudaError_t e = cudaSuccess;
    if (direct) {
        rs.out = static_cast<float4 *>(zimg);
        rs.nsamples = static_cast<int32_t *>(zns);
    } else {
        e = ctx->st_out.reserve(img_b + ns_b);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "staging allocation");
        rs.out = static_cast<float4 *>(ctx->st_out.ptr);
        rs.nsamples =
            nsamples_host ? reinterpret_cast<int32_t *>(static_cast<char *>(ctx->st_out.ptr) + img_b) : nullptr;
    }
    int *counter = nullptr;
    if (mfadvr_status st = next_counter(ctx, &counter)) return st;
    int slot = -1;
    if (mfadvr_status st = take_order(ctx, &rs, s, &slot)) return st;
    e = launch_render(view_of(*m), rs, counter, s);
    if (e == cudaSuccess) {
        if (mfadvr_status st = record_order(ctx, slot, s)) return st;
    }
    if (e == cudaSuccess && !direct) e = cudaMemcpyAsync(rgba_host, rs.out, img_b, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && !direct && nsamples_host)
        e = cudaMemcpyAsync(nsamples_host, rs.nsamples, ns_b, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "render_host");
    return MFADVR_OK;
}

mfadvr_status mfadvr_render_batch(mfadvr_ctx *ctx, int32_t njobs, const mfadvr_render_job *jobs, void *stream)
{
    TraceRange trace("mfadvr_render_batch");
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    if (njobs < 1 || njobs > MFADVR_MAX_BATCH || !jobs)
        return fail(ctx, MFADVR_EINVAL, "njobs must be in 1..%d and jobs not NULL", MFADVR_MAX_BATCH);
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "cudaSetDevice");
    // every argument first, then device work
    std::vector<RenderJob> table(njobs);
    for (int i = 0; i < njobs; ++i)
        if (mfadvr_status st = make_job(ctx, jobs[i], i, &table[i])) return st;
    if (!ctx->d_jobs) {
        const size_t bytes = sizeof(RenderJob) * MFADVR_MAX_BATCH * mfadvr_ctx::kJobSlots;
        cudaError_t e = cudaMalloc(&ctx->d_jobs, bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_jobs, bytes);
        for (unsigned k = 0; e == cudaSuccess && k < mfadvr_ctx::kJobSlots; ++k)
            e = cudaEventCreateWithFlags(&ctx->job_done[k], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "job-table allocation");
    }
    const unsigned slot = ctx->next_jobs++ % mfadvr_ctx::kJobSlots;
    cudaError_t e = cudaEventSynchronize(ctx->job_done[slot]);  // the slot's previous launches are done
    if (e != cudaSuccess) return cuda_fail(ctx, e, "job-table slot wait");
    RenderJob *hj = ctx->h_jobs + static_cast<size_t>(slot) * MFADVR_MAX_BATCH;
    RenderJob *dj = ctx->d_jobs + static_cast<size_t>(slot) * MFADVR_MAX_BATCH;
    std::vector<BatchGroup> groups = pack_jobs(table.data(), njobs, hj);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(dj, hj, sizeof(RenderJob) * njobs, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "job-table copy");
    for (const BatchGroup &gr : groups) {
        int *counter = nullptr;
        if (mfadvr_status st = next_counter(ctx, &counter)) return st;
        // the group's tiles costliest first (as mfadvr_render), on one scale
        // of cost levels: the largest sample count along a job's box diagonal
        int *order = nullptr, *hist = nullptr;
        unsigned char *level = nullptr;
        int oslot = -1;
        if (mfadvr_status st = take_order_slot(ctx, gr.tiles, s, &order, &level, &hist, &oslot)) return st;
        if (oslot >= 0) {
            float max_count = 1.0f;
            for (int i = gr.first; i < gr.first + gr.count; ++i) {
                const RenderSetup &r = hj[i].rs;
                double d2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    const double ext = static_cast<double>(r.box_max[a]) - r.box_min[a];
                    d2 += ext * ext;
                }
                max_count = std::max(max_count, static_cast<float>(std::sqrt(d2) / r.step + 1.0));
            }
            e = launch_tile_order_batch(dj + gr.first, gr.count, gr.tiles, max_count, order, level, hist, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "batched tile order");
        }
        e = launch_render_batch(gr.p, gr.dtype, gr.grad, gr.nu, gr.rat, dj + gr.first, gr.count, gr.tiles, 0, counter,
                                order, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batched render launch");
        if (mfadvr_status st = record_order(ctx, oslot, s)) return st;
    }
    e = cudaEventRecord(ctx->job_done[slot], s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "job-table slot event");
    return MFADVR_OK;
}

mfadvr_status mfadvr_autotune(mfadvr_ctx *ctx, int32_t model_id, const mfadvr_camera *camera,
                              const mfadvr_render_params *params, float *rgba_dev, int32_t *nsamples_dev, void *stream,
                              mfadvr_tuning *best)
{
    TraceRange trace("mfadvr_autotune");
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    Model *m = nullptr;
    if (mfadvr_status st = find_model(ctx, model_id, &m)) return st;
    RenderSetup rs;
    if (mfadvr_status st = make_setup(ctx, *m, camera, params, &rs)) return st;
    if (!rgba_dev || reinterpret_cast<uintptr_t>(rgba_dev) % 16 != 0 ||
        reinterpret_cast<uintptr_t>(nsamples_dev) % 4 != 0)
        return fail(ctx, MFADVR_EINVAL, "rgba must be 16-byte and nsamples 4-byte aligned");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "cudaSetDevice");
    if (!is_device_ptr(rgba_dev) || !is_device_ptr(params->tf_rgba) || (nsamples_dev && !is_device_ptr(nsamples_dev)))
        return fail(ctx, MFADVR_EINVAL, "rgba, tf_rgba and nsamples must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mfadvr_status st = stage_tf(ctx, params->tf_rgba, params->tf_size, false, &rs, s)) return st;
    rs.out = reinterpret_cast<float4 *>(rgba_dev);
    rs.nsamples = nsamples_dev;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event creation");
    const int tile_ws[] = {8, 4, 16, 2, 32, 1};
    const int ctas[] = {0, 2};
    mfadvr_tuning win{8, 0, INFINITY};
    for (int tw : tile_ws) {
        for (int c : ctas) {
            rs.tile_w_log2 = ilog2_u64(static_cast<uint64_t>(tw));
            rs.ctas_per_sm = c;
            float ms_best = INFINITY;
            // the fastest of 7 launches after a warm-up one: neighbouring
            // shapes differ by about 1-2%, which 3 launches did not resolve
            for (int rep = 0; rep < 8 && e == cudaSuccess; ++rep) {
                int *counter = nullptr;
                if (mfadvr_status st = next_counter(ctx, &counter)) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return st;
                }
                int slot = -1;
                if (mfadvr_status st = take_order(ctx, &rs, s, &slot)) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return st;
                }
                e = cudaEventRecord(e0, s);
                if (e == cudaSuccess) e = launch_render(view_of(*m), rs, counter, s);
                if (e == cudaSuccess && slot >= 0) e = cudaEventRecord(ctx->order_done[slot], s);
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && ms < ms_best) ms_best = ms;  // the first run warms up
            }
            if (e != cudaSuccess) break;
            if (ms_best < win.ms) win = mfadvr_tuning{tw, c, ms_best};
        }
        if (e != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
    ctx->tuning[tune_key(*m, rs.width, rs.height)] = win;
    if (best) *best = win;
    return MFADVR_OK;
}

mfadvr_status mfadvr_tuning_save(mfadvr_ctx *ctx, const char *path)
{
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    if (!path) return fail(ctx, MFADVR_EINVAL, "path must not be NULL");
    FILE *f = fopen(path, "w");
    if (!f) return fail(ctx, MFADVR_EINVAL, "cannot open %s for writing", path);
    for (const auto &kv : ctx->tuning)
        fprintf(f, "%d %d %d %d %d %d %.6f\n", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                std::get<3>(kv.first), kv.second.tile_w, kv.second.ctas_per_sm, kv.second.ms);
    const bool ok = fclose(f) == 0;
    return ok ? MFADVR_OK : fail(ctx, MFADVR_EINVAL, "cannot write %s", path);
}

mfadvr_status mfadvr_tuning_load(mfadvr_ctx *ctx, const char *path)
{
    if (!ctx) return fail(nullptr, MFADVR_EINVAL, "ctx must not be NULL");
    if (!path) return fail(ctx, MFADVR_EINVAL, "path must not be NULL");
    FILE *f = fopen(path, "r");
    if (!f) return fail(ctx, MFADVR_EINVAL, "cannot open %s", path);
    std::map<TuneKey, mfadvr_tuning> add;
    char line[256];
    int lineno = 0;
    while (fgets(line, sizeof line, f)) {
        ++lineno;
        int p, dt, lp, li, tw, c;
        float ms;
        if (sscanf(line, "%d %d %d %d %d %d %f", &p, &dt, &lp, &li, &tw, &c, &ms) != 7 || tw < 1 || tw > 32 ||
            (tw & (tw - 1)) != 0 || c < 0) {
            fclose(f);
            return fail(ctx, MFADVR_EINVAL, "%s:%d: malformed tuning line", path, lineno);
        }
        add[TuneKey(p, dt, lp, li)] = mfadvr_tuning{tw, c, ms};
    }
    fclose(f);
    for (const auto &kv : add) ctx->tuning[kv.first] = kv.second;
    return MFADVR_OK;
}

const char *mfadvr_status_string(mfadvr_status status)
{
    switch (status) {
    case MFADVR_OK: return "ok";
    case MFADVR_EINVAL: return "invalid argument";
    case MFADVR_ENOMEM: return "out of memory or over the HBM budget";
    case MFADVR_ECUDA: return "CUDA error";
    case MFADVR_ENOTFOUND: return "model not found";
    case MFADVR_ETIMEOUT: return "timed out";
    case MFADVR_EBUSY: return "busy";
    case MFADVR_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

const char *mfadvr_last_error(mfadvr_ctx *ctx)
{
    if (!ctx) {
        std::lock_guard<std::mutex> g(g_create_mu);
        return g_create_err.c_str();
    }
    return ctx->err.c_str();
}

}  // extern "C"
