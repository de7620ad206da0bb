// mfadvr_render_lattice_noalloc: the render path for callers that cannot
// allocate device memory.
//
// Some callers must not call cudaMalloc during a render:
//  - code that records work into a CUDA stream capture, where an allocation
//    is not part of the captured work;
//  - plug-in hosts whose device memory is owned by the host application's
//    pool allocator;
//  - real-time loops, where the implicit device synchronisation of an
//    allocation would stall a frame.
// The regular path allocates: mfadvr_create / mfadvr_load_model put the model
// in library-owned memory, and mfadvr_render allocates its ray-tile counter
// ring on first use.  This entry point allocates nothing.  The caller passes
// its own FP32 lattice, transfer function and outputs in device memory.  The
// row layout the render kernel reads and the ray-tile counter live in one
// file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "mfa_internal.h"
#include "mfadvr.h"

namespace {

// [0, 256): the ray-tile counter; [256, 256 + 32 * MFADVR_NOALLOC_MAX_POINTS):
// the FP32 row array of the lattice.
constexpr size_t kCounterBytes = 256;
constexpr size_t kScratchBytes = kCounterBytes + mfadvr::row_entry_bytes(MFADVR_F32) * MFADVR_NOALLOC_MAX_POINTS;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context id the address was looked up in

// Device memory of device `dev` (managed memory is reachable from any device).
bool device_pointer(const void *p, int dev)
{
    if (!p) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (attr.type == cudaMemoryTypeDevice && attr.device == dev) || attr.type == cudaMemoryTypeManaged;
}

// Unique id of the calling thread's current CUDA context, 0 if none or if the
// driver entry points cannot be found.  A cudaDeviceReset destroys the
// primary context; the next one gets a new id, so a cached symbol address is
// looked up again instead of being used stale.
unsigned long long current_context_id()
{
    using GetCurrent = int (*)(void **);
    using GetId = int (*)(void *, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &f, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPoint("cuCtxGetId", &f, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    void *c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != 0 || !c || get_id(c, &id) != 0) return 0;
    return id;
}

mfadvr_status err(mfadvr_status st, const char *msg) { return mfadvr::fail_noctx(st, msg); }

}  // namespace

extern "C" MFADVR_API mfadvr_status mfadvr_render_lattice_noalloc(
    const float *ctrl_dev, const int32_t degree[3], const int32_t ncp[3], const float box_min[3],
    const float box_max[3], const mfadvr_camera *camera, const mfadvr_render_params *params, float *rgba_dev,
    int32_t *nsamples_dev, void *stream)
{
    if (!degree || !ncp || !box_min || !box_max || !camera || !params)
        return err(MFADVR_EINVAL, "degree, ncp, box, camera and params must not be NULL");
    if (degree[0] != degree[1] || degree[0] != degree[2] || degree[0] < 1 || degree[0] > MFADVR_MAX_DEGREE)
        return err(MFADVR_EUNSUPPORTED, "degrees must be equal on the three axes and in 1..MFADVR_MAX_DEGREE");
    int n[3];
    for (int a = 0; a < 3; ++a) {
        if (ncp[a] < degree[a] + 1 || ncp[a] > (1 << 24)) return err(MFADVR_EINVAL, "ncp must be in degree+1..2^24");
        if (!std::isfinite(box_min[a]) || !std::isfinite(box_max[a]) || !(box_max[a] > box_min[a]))
            return err(MFADVR_EINVAL, "box_max must exceed box_min on every axis");
        n[a] = ncp[a];
    }
    // n0 n1 <= 2^48 cannot wrap in 64 bits; the third factor is checked by
    // division, so that no product of three sides wraps past the limit.
    const unsigned long long n01 = static_cast<unsigned long long>(n[0]) * static_cast<unsigned long long>(n[1]);
    if (n01 > static_cast<unsigned long long>(MFADVR_NOALLOC_MAX_POINTS) / static_cast<unsigned long long>(n[2])) {
        char msg[200];
        snprintf(msg, sizeof msg, "lattice of %d x %d x %d control points exceeds the allocation-free scratch "
                 "(at most %d)", n[0], n[1], n[2], MFADVR_NOALLOC_MAX_POINTS);
        return err(MFADVR_ENOMEM, msg);
    }
    if (std::isnan(params->tf_lo) || std::isnan(params->tf_hi))
        return err(MFADVR_EINVAL, "tf_lo and tf_hi must be given (the lattice range is not computed here)");
    if (params->tf_size < 2)
        return err(MFADVR_EINVAL, "tf_size must be at least 2 (a one-entry table would need a staged copy)");
    if (reinterpret_cast<uintptr_t>(ctrl_dev) % 4 != 0 || reinterpret_cast<uintptr_t>(params->tf_rgba) % 16 != 0 ||
        reinterpret_cast<uintptr_t>(rgba_dev) % 16 != 0 || reinterpret_cast<uintptr_t>(nsamples_dev) % 4 != 0)
        return err(MFADVR_EINVAL, "ctrl, tf_rgba, rgba and nsamples must be aligned (4, 16, 16, 4 bytes)");

    mfadvr::RenderSetup rs;
    if (mfadvr_status st = mfadvr::setup_for_lattice(degree[0], n, box_min, box_max, camera, params, &rs)) return st;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return err(MFADVR_ECUDA, "no usable current device");
    if (!device_pointer(ctrl_dev, dev) || !device_pointer(params->tf_rgba, dev) || !device_pointer(rgba_dev, dev) ||
        (nsamples_dev && !device_pointer(nsamples_dev, dev)))
        return err(MFADVR_EINVAL, "ctrl, tf_rgba, rgba and nsamples must be memory of the current device");

    // Set-up, once per device (and again after a cudaDeviceReset replaced
    // its context), with that device current: the device address of the
    // scratch array (its host-side name is only a stand-in).
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_setup_mu);
        const unsigned long long ctx_id = current_context_id();
        if (!g_scratch_ptr[dev] || ctx_id != g_scratch_ctx[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return err(MFADVR_ECUDA, "cudaGetSymbolAddress of the allocation-free scratch failed");
            }
            g_scratch_ptr[dev] = p;
            g_scratch_ctx[dev] = current_context_id();  // the lookup made the context current if none was
        }
        scratch = g_scratch_ptr[dev];
    }
    int *counter = static_cast<int *>(scratch);
    void *rows = static_cast<unsigned char *>(scratch) + kCounterBytes;

    mfadvr::ModelView mv;
    mv.rows = rows;
    mv.p = degree[0];
    mv.dtype = MFADVR_F32;
    mv.scale = 1.0f;
    mv.n01 = n[0] * n[1];
    mv.nu = 0;  // clamped uniform knots, non-rational
    mv.rational = 0;
    mv.wrows = nullptr;
    mv.wscale = 1.0f;
    mv.poly = nullptr;  // the B-spline form: nothing beyond the caller's lattice
    mv.wpoly = nullptr;
    for (int a = 0; a < 3; ++a) {
        mv.n[a] = n[a];
        mv.m[a] = n[a] - degree[0];
        mv.brk[a] = mv.ih[a] = mv.pieces[a] = nullptr;
        mv.cell[a] = nullptr;
        mv.grid[a] = 0;
    }
    rs.tf = reinterpret_cast<const float4 *>(params->tf_rgba);
    rs.out = reinterpret_cast<float4 *>(rgba_dev);
    rs.nsamples = nsamples_dev;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The rows are rebuilt and the counter zeroed (by the render launcher)
    // on every call, so nothing a previous call left in the array is read.
    e = mfadvr::launch_build_rows(ctrl_dev, rows, n[0], n[1], n[2], MFADVR_F32, 1.0f, s);
    if (e == cudaSuccess) e = mfadvr::launch_render(mv, rs, counter, s);
    if (e != cudaSuccess) {
        char msg[160];
        snprintf(msg, sizeof msg, "allocation-free render launch: %s", cudaGetErrorString(e));
        return err(MFADVR_ECUDA, msg);
    }
    return MFADVR_OK;
}
