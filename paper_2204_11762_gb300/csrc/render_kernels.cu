// mfadvr_render's launchers: pick the per-degree instantiation (the kernels
// are in render_kernels.cuh, one degree per render_pN.cu).
#include "mfa_internal.h"
#include "render_kernels.cuh"

namespace mfadvr {

cudaError_t launch_render(const ModelView &mv, const RenderSetup &rs, int *counter, cudaStream_t stream)
{
    switch (mv.p) {
    case 1: return launch_render_p1(mv, rs, counter, stream);
    case 2: return launch_render_p2(mv, rs, counter, stream);
    case 3: return launch_render_p3(mv, rs, counter, stream);
    case 4: return launch_render_p4(mv, rs, counter, stream);
    case 5: return launch_render_p5(mv, rs, counter, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_render_trace(const ModelView &mv, const RenderSetup &rs, int *counter, const TraceOn &tr,
                                cudaStream_t stream)
{
    switch (mv.p) {
    case 1: return launch_render_trace_p1(mv, rs, counter, tr, stream);
    case 2: return launch_render_trace_p2(mv, rs, counter, tr, stream);
    case 3: return launch_render_trace_p3(mv, rs, counter, tr, stream);
    case 4: return launch_render_trace_p4(mv, rs, counter, tr, stream);
    case 5: return launch_render_trace_p5(mv, rs, counter, tr, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_render_batch(int p, int dtype, int grad, int nu, int rat, const RenderJob *jobs_dev, int njobs,
                                int total_tiles, int ctas_per_sm, int *counter, cudaStream_t stream)
{
    switch (p) {
    case 1:
        return launch_render_batch_p1(dtype, grad, nu, rat, jobs_dev, njobs, total_tiles, ctas_per_sm, counter,
                                        stream);
    case 2:
        return launch_render_batch_p2(dtype, grad, nu, rat, jobs_dev, njobs, total_tiles, ctas_per_sm, counter,
                                        stream);
    case 3:
        return launch_render_batch_p3(dtype, grad, nu, rat, jobs_dev, njobs, total_tiles, ctas_per_sm, counter,
                                        stream);
    case 4:
        return launch_render_batch_p4(dtype, grad, nu, rat, jobs_dev, njobs, total_tiles, ctas_per_sm, counter,
                                        stream);
    case 5:
        return launch_render_batch_p5(dtype, grad, nu, rat, jobs_dev, njobs, total_tiles, ctas_per_sm, counter,
                                        stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mfadvr
