// mfadvr_probe_fma: the FP32 multiply-add throughput of this GPU, measured.
//
// The render and point-query kernels run on the FP32 FMA pipe, so their
// roofline is the number of multiply-adds an SM can retire per second.  The
// peak derived from unit counts (SMs x 128 FP32 lanes x clock) assumes every
// issue slot is a multiply-add; this kernel measures what the chip delivers:
// eight independent chains per thread (a chain's latency is hidden by the
// others and by 64 resident warps per SM), 128 multiply-adds per loop
// iteration (scalar FFMA or packed fma.rn.f32x2), nothing else in the loop
// but its counter.  The caller times the launch with events on `stream`.
#include <cstdio>

#include "mfa_internal.h"
#include "mfadvr.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 8;  // chain steps per loop iteration

template <bool Packed>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(float *sink, int iters, float seed)
{
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        a[k] = make_float2(seed + 1e-7f * static_cast<float>(threadIdx.x) + static_cast<float>(k), seed - k);
    const float2 mul = make_float2(0.9999999f, 1.0000001f);
    const float2 add = make_float2(1e-7f, -1e-7f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if constexpr (Packed) {
                    a[k] = __ffma2_rn(a[k], mul, add);
                } else {
                    a[k].x = fmaf(a[k].x, mul.x, add.x);
                    a[k].y = fmaf(a[k].y, mul.y, add.y);
                }
            }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    // The chains stay live through a store that never happens in practice.
    if (s == 1234.5f) sink[0] = s;
}

}  // namespace

extern "C" MFADVR_API mfadvr_status mfadvr_probe_fma(int32_t packed, int32_t iters, float *sink_dev, void *stream,
                                                    double *fma_count)
{
    if (!sink_dev || !fma_count) return mfadvr::fail_noctx(MFADVR_EINVAL, "sink_dev and fma_count must not be NULL");
    if (iters < 1 || iters > (1 << 24)) return mfadvr::fail_noctx(MFADVR_EINVAL, "iters must be in 1..2^24");
    if (packed != 0 && packed != 1) return mfadvr::fail_noctx(MFADVR_EINVAL, "packed must be 0 or 1");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaPointerAttributes attr;
    if (e == cudaSuccess) e = cudaPointerGetAttributes(&attr, sink_dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return mfadvr::fail_noctx(MFADVR_EINVAL, "sink_dev must be memory of the current device");
    }
    if (!((attr.type == cudaMemoryTypeDevice && attr.device == dev) || attr.type == cudaMemoryTypeManaged))
        return mfadvr::fail_noctx(MFADVR_EINVAL, "sink_dev must be memory of the current device");
    int per_sm = 0;
    e = packed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<true>, kProbeThreads, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<false>, kProbeThreads, 0);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return mfadvr::fail_noctx(MFADVR_ECUDA, "occupancy query of the FMA probe failed");
    }
    const int blocks = sms * per_sm;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (packed) fma_probe_kernel<true><<<blocks, kProbeThreads, 0, s>>>(sink_dev, iters, 1.0f);
    else fma_probe_kernel<false><<<blocks, kProbeThreads, 0, s>>>(sink_dev, iters, 1.0f);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        char msg[160];
        snprintf(msg, sizeof msg, "FMA probe launch: %s", cudaGetErrorString(e));
        return mfadvr::fail_noctx(MFADVR_ECUDA, msg);
    }
    *fma_count = static_cast<double>(blocks) * kProbeThreads * static_cast<double>(iters) * kUnroll * kChains * 2.0;
    return MFADVR_OK;
}
