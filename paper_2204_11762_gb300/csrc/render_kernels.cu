// mfadvr_render's launchers: pick the per-degree instantiation (the kernels
// are in render_kernels.cuh, one degree per render_pN.cu).
#include <algorithm>

#include "mfa_internal.h"
#include "render_kernels.cuh"

namespace mfadvr {

namespace {

constexpr int kTileLevels = 32;

// Lane-in-tile of corner c (0..3) of a tile of tw x 32/tw pixels.
__device__ __forceinline__ int corner_lane(int c, int tw)
{
    return c == 0 ? 0 : (c == 1 ? tw - 1 : (c == 2 ? 32 - tw : 31));
}

// Takes the largest of the sample counts n of the four lanes of a corner
// group (lanes 4g .. 4g + 3, all lanes of the warp calling) and, in the
// group's first lane, records the tile's level (kTileLevels levels of
// per_level samples, level 0 the costliest) and counts it in s_hist.
__device__ __forceinline__ void record_tile_level(int n, bool valid, int tile, float per_level,
                                                  unsigned char *__restrict__ level, int *s_hist)
{
    n = max(n, __shfl_xor_sync(kFull, n, 1));
    n = max(n, __shfl_xor_sync(kFull, n, 2));
    if ((threadIdx.x & 3) == 0 && valid) {
        const int q = min(static_cast<int>(static_cast<float>(n) / per_level), kTileLevels - 1);
        level[tile] = static_cast<unsigned char>(kTileLevels - 1 - q);
        atomicAdd(&s_hist[kTileLevels - 1 - q], 1);
    }
}

// Tile costs for the longest-first order.  Four lanes per tile, one per
// corner pixel of the tile (clamped into the image: a tile's first pixel is
// always inside it), each taking its ray's sample count (the chord through
// the box over the step: the samples it takes unless it terminates early);
// the tile's cost is the largest of the four, quantised to kTileLevels levels
// of the count along the box diagonal; level 0 holds the costliest tiles.
// level[tile] and per-level counts in hist[0 .. kTileLevels).
__global__ void __launch_bounds__(256) tile_level_kernel(RenderSetup rs, int tiles_x, int tiles,
                                                         unsigned char *__restrict__ level, int *__restrict__ hist)
{
    __shared__ int s_hist[kTileLevels];
    if (threadIdx.x < kTileLevels) s_hist[threadIdx.x] = 0;
    __syncthreads();
    float diag2 = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float e = rs.box_max[a] - rs.box_min[a];
        diag2 = fmaf(e, e, diag2);
    }
    const float per_level = fmaxf(sqrtf(diag2) / rs.step + 1.0f, 1.0f) / static_cast<float>(kTileLevels);
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    const int l = corner_lane(lane & 3, 1 << rs.tile_w_log2);
    for (int base = (blockIdx.x * warps + (threadIdx.x >> 5)) * 8; base < tiles; base += gridDim.x * warps * 8) {
        const int tile = base + (lane >> 2);
        int n = 0;
        if (tile < tiles) {
            int px, py;
            slot_pixel(tile * 32 + l, tiles_x, rs.tile_w_log2, px, py);
            float o[3], dir[3], t0;
            n = static_cast<int>(ray_chord(rs, min(px, rs.width - 1), min(py, rs.height - 1), o, dir, t0));
        }
        record_tile_level(n, tile < tiles, tile, per_level, level, s_hist);
    }
    __syncthreads();
    if (threadIdx.x < kTileLevels && s_hist[threadIdx.x]) atomicAdd(&hist[threadIdx.x], s_hist[threadIdx.x]);
}

// The same for a batched launch: tile t of the concatenated sequence belongs
// to the job whose tile_begin is the largest at or below t (jobs sorted by
// tile_begin); its corner rays use that job's camera, box and step.  One
// scale of levels for all jobs (per_level samples per level, the host's
// largest diagonal count over the jobs / kTileLevels), so that tiles of
// different jobs compare.
__global__ void __launch_bounds__(256) tile_level_batch_kernel(const RenderJob *__restrict__ jobs, int njobs, int tiles,
                                                               float per_level, unsigned char *__restrict__ level,
                                                               int *__restrict__ hist)
{
    __shared__ int s_hist[kTileLevels];
    if (threadIdx.x < kTileLevels) s_hist[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    for (int base = (blockIdx.x * warps + (threadIdx.x >> 5)) * 8; base < tiles; base += gridDim.x * warps * 8) {
        const int tile = base + (lane >> 2);
        int n = 0;
        if (tile < tiles) {
            int lo = 0, hi = njobs - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(&jobs[mid].tile_begin) <= tile) lo = mid;
                else hi = mid - 1;
            }
            const RenderSetup &rs = jobs[lo].rs;
            int px, py;
            slot_pixel((tile - jobs[lo].tile_begin) * 32 + corner_lane(lane & 3, 1 << rs.tile_w_log2),
                       jobs[lo].tiles_x, rs.tile_w_log2, px, py);
            float o[3], dir[3], t0;
            n = static_cast<int>(ray_chord(rs, min(px, rs.width - 1), min(py, rs.height - 1), o, dir, t0));
        }
        record_tile_level(n, tile < tiles, tile, per_level, level, s_hist);
    }
    __syncthreads();
    if (threadIdx.x < kTileLevels && s_hist[threadIdx.x]) atomicAdd(&hist[threadIdx.x], s_hist[threadIdx.x]);
}

// Counting sort of the tiles by level: order[] lists level 0's tiles first.
// Lanes of a warp with equal levels take consecutive places through one
// atomic on the level's cursor (hist[kTileLevels + level]); within a level
// the order is that of the atomics.
__global__ void __launch_bounds__(256) tile_order_kernel(int tiles, const unsigned char *__restrict__ level,
                                                         int *__restrict__ hist, int *__restrict__ order)
{
    __shared__ int s_base[kTileLevels];
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < kTileLevels) {
        const int c = hist[threadIdx.x];
        int x = c;
#pragma unroll
        for (int o = 1; o < kTileLevels; o <<= 1) {
            const int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        s_base[threadIdx.x] = x - c;
    }
    __syncthreads();
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < tiles; base += stride) {
        const int t = base + lane;
        const bool ok = t < tiles;
        const int lv = ok ? level[t] : kTileLevels;
        const unsigned peers = __match_any_sync(kFull, lv);
        const int leader = __ffs(peers) - 1;
        int first = 0;
        if (ok && lane == leader) first = atomicAdd(&hist[kTileLevels + lv], __popc(peers));
        first = __shfl_sync(kFull, first, leader);
        if (ok) order[s_base[lv] + first + __popc(peers & ((1u << lane) - 1u))] = t;
    }
}

}  // namespace

cudaError_t launch_tile_order(const RenderSetup &rs, int tiles_x, int tiles, cudaStream_t stream)
{
    if (tiles <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(rs.tile_hist, 0, 2 * kTileLevels * sizeof(int), stream);
    if (e != cudaSuccess) return e;
    const int cap = sm_count() * 8;
    const int lv_blocks = std::min((tiles + 63) / 64, cap);  // 8 warps of 8 tiles
    tile_level_kernel<<<lv_blocks, 256, 0, stream>>>(rs, tiles_x, tiles, rs.tile_level, rs.tile_hist);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int ord_blocks = std::min((tiles + 255) / 256, cap);
    tile_order_kernel<<<ord_blocks, 256, 0, stream>>>(tiles, rs.tile_level, rs.tile_hist, rs.tile_order);
    return cudaGetLastError();
}

cudaError_t launch_tile_order_batch(const RenderJob *jobs_dev, int njobs, int tiles, float max_count, int *order,
                                    unsigned char *level, int *hist, cudaStream_t stream)
{
    if (tiles <= 0 || njobs <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(hist, 0, 2 * kTileLevels * sizeof(int), stream);
    if (e != cudaSuccess) return e;
    const int cap = sm_count() * 8;
    const float per_level = fmaxf(max_count, 1.0f) / static_cast<float>(kTileLevels);
    const int lv_blocks = std::min((tiles + 63) / 64, cap);
    tile_level_batch_kernel<<<lv_blocks, 256, 0, stream>>>(jobs_dev, njobs, tiles, per_level, level, hist);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int ord_blocks = std::min((tiles + 255) / 256, cap);
    tile_order_kernel<<<ord_blocks, 256, 0, stream>>>(tiles, level, hist, order);
    return cudaGetLastError();
}

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
                                int total_tiles, int ctas_per_sm, int *counter, const int *order, cudaStream_t stream)
{
    switch (p) {
    case 1:
        return launch_render_batch_p1(dtype, grad, nu, rat, jobs_dev, njobs, total_tiles, ctas_per_sm, counter, order,
                                        stream);
    case 2:
        return launch_render_batch_p2(dtype, grad, nu, rat, jobs_dev, njobs, total_tiles, ctas_per_sm, counter, order,
                                        stream);
    case 3:
        return launch_render_batch_p3(dtype, grad, nu, rat, jobs_dev, njobs, total_tiles, ctas_per_sm, counter, order,
                                        stream);
    case 4:
        return launch_render_batch_p4(dtype, grad, nu, rat, jobs_dev, njobs, total_tiles, ctas_per_sm, counter, order,
                                        stream);
    case 5:
        return launch_render_batch_p5(dtype, grad, nu, rat, jobs_dev, njobs, total_tiles, ctas_per_sm, counter, order,
                                        stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mfadvr
