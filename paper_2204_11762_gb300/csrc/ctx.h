// Internals of libmfadvr.so shared by its host-side translation units: the
// resident model store, the context, argument checks and render setup.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mfa_internal.h"
#include "mfadvr.h"

namespace mfadvr {
namespace api {

// A named NVTX range over a scope: each entry point and each serving batch
// shows up by name on a profiler's timeline (no cost without a tool attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

struct Model {
    void *d_rows = nullptr;   // row layout, see mfa_basis.cuh
    uint64_t bytes = 0;
    int p = 0;
    int n[3] = {0, 0, 0};
    int dtype = MFADVR_F32;
    float scale = 1.0f;
    float pmin = 0.0f, pmax = 0.0f, pabs = 0.0f;
    float box_min[3] = {0, 0, 0}, box_max[3] = {1, 1, 1};
    // General knots (nu = 1): one device buffer holding, per axis, the
    // breakpoints, inverse widths and per-span pieces at these float offsets.
    int nu = 0;
    void *d_knots = nullptr;
    // Rational model: d_rows holds w P (scale `scale`), d_wrows holds w
    // (scale wscale), both in the row layout and the storage type.
    int rational = 0;
    void *d_wrows = nullptr;
    float wscale = 1.0f;
    uint64_t knot_bytes = 0;
    size_t brk_off[3] = {0, 0, 0}, ih_off[3] = {0, 0, 0}, cell_off[3] = {0, 0, 0}, pc_off[3] = {0, 0, 0};
    // POWER render form: the span polynomials (layout in mfa_basis.cuh,
    // PolyCell), null in the B-spline form.
    void *d_poly = nullptr;
    uint64_t poly_bytes = 0;
};

// Device buffer owned by the context, grown on demand (host-buffer calls).
struct Staging {
    void *ptr = nullptr;
    size_t bytes = 0;
    cudaError_t reserve(size_t need)
    {
        if (need <= bytes) return cudaSuccess;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&ptr, need);
        if (e == cudaSuccess) bytes = need;
        return e;
    }
    void release()
    {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
};

// Tuning-table key: degree, storage type, log2 of the lattice size and of
// the image size.
using TuneKey = std::tuple<int, int, int, int>;

struct Server;  // serving loop, see serve.cu

}  // namespace api
}  // namespace mfadvr

struct mfadvr_ctx {
    using Model = mfadvr::api::Model;
    using Staging = mfadvr::api::Staging;
    using TuneKey = mfadvr::api::TuneKey;
    int device = 0;
    uint64_t budget = 0, used = 0;
    std::map<int32_t, Model> models;
    int32_t next_id = 0;
    std::string err;
    Staging st_in, st_out, st_aux;
    // Ray-tile counters of render launches: each call takes the next slot of
    // the ring, so calls queued on different streams do not share one.
    int *counters = nullptr;
    unsigned next_counter = 0;
    static constexpr unsigned kCounters = 1024;
    // Batched renders: a ring of job tables (pinned host + device), each
    // slot guarded by an event recorded after the launches that read it.
    static constexpr unsigned kJobSlots = 32;
    mfadvr::RenderJob *h_jobs = nullptr, *d_jobs = nullptr;
    cudaEvent_t job_done[kJobSlots] = {};
    unsigned next_jobs = 0;
    // Longest-first tile orders of mfadvr_render launches: a ring of scratch
    // areas for images of up to kOrderTiles ray tiles (larger images take
    // their tiles in row order), each reused only after the launch that last
    // read it has finished (its event).  Allocated at the first such render.
    static constexpr unsigned kOrderSlots = 8;
    static constexpr int64_t kOrderTiles = int64_t(1) << 19;
    char *order_pool = nullptr;
    cudaEvent_t order_done[kOrderSlots] = {};
    unsigned next_order = 0;
    std::map<TuneKey, mfadvr_tuning> tuning;
    mfadvr::api::Server *server = nullptr;
    // Host-buffer point queries: chunks are copied in, evaluated and copied
    // out on these streams in turn, so that the two copy directions and the
    // kernels of neighbouring chunks overlap (created on first use).
    static constexpr int kPipes = 3;
    cudaStream_t pipe[kPipes] = {};
    cudaEvent_t pipe_start = nullptr;
};

namespace mfadvr {
namespace api {

mfadvr_status fail(mfadvr_ctx *ctx, mfadvr_status st, const char *fmt, ...);
mfadvr_status cuda_fail(mfadvr_ctx *ctx, cudaError_t e, const char *what);

// Makes ctx->device current for the duration of a call and restores the
// caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool is_device_ptr(const void *p);
ModelView view_of(const Model &m);
mfadvr_status next_counter(mfadvr_ctx *ctx, int **out);
mfadvr_status find_model(mfadvr_ctx *ctx, int32_t id, Model **out);
mfadvr_status make_setup(mfadvr_ctx *ctx, const Model &m, const mfadvr_camera *cam, const mfadvr_render_params *rp,
                         RenderSetup *rs);
void apply_tuning(const mfadvr_ctx *ctx, const Model &m, RenderSetup *rs);
// Checks one render job and turns it into the kernel's job record
// (tile fields are set by pack_jobs).
mfadvr_status make_job(mfadvr_ctx *ctx, const mfadvr_render_job &job, int index, RenderJob *out);

// One launch of a batched render: jobs dst[first, first+count) of one degree
// and storage type, `tiles` tiles in all.
struct BatchGroup {
    int p, dtype, grad, nu, rat, first, count, tiles;
};
// Orders n jobs by (degree, storage type, shading, general knots, rational)
// into dst, fills their tile fields and returns the launch groups (grad =
// shading: the gradient is queried; nu: general knots; rat: weights).
std::vector<BatchGroup> pack_jobs(const RenderJob *jobs, int n, RenderJob *dst);
// Tears down a context's serving loop, if one runs (serve.cu).
void stop_server(mfadvr_ctx *ctx);

}  // namespace api
}  // namespace mfadvr
