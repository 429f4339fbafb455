// rt_render.cu -- instantiations and launchers of the render and medium
// kernels (the kernels themselves are in rt_trace.cuh).
#include "rt_trace.cuh"

namespace grt {

template <class R>
static cudaError_t occupancy_t(int variant, int* bps)
{
    switch (variant) {
        case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, render_kernel<R, kVariantBlocks[1]>, kRenderBlock, 0);
        case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, render_kernel<R, kVariantBlocks[2]>, kRenderBlock, 0);
        default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, render_kernel<R, kVariantBlocks[0]>, kRenderBlock, 0);
    }
}

template <class R>
static void launch_t(const DevScene& sc, int variant, int min_active, float* rgb, uint8_t* rgb8, rt_ray_record* rec,
                     unsigned long long* counters, int grid, cudaStream_t stream)
{
    switch (variant) {
        case 1: render_kernel<R, kVariantBlocks[1]><<<grid, kRenderBlock, 0, stream>>>(sc, rgb, rgb8, rec, counters, min_active); break;
        case 2: render_kernel<R, kVariantBlocks[2]><<<grid, kRenderBlock, 0, stream>>>(sc, rgb, rgb8, rec, counters, min_active); break;
        default: render_kernel<R, kVariantBlocks[0]><<<grid, kRenderBlock, 0, stream>>>(sc, rgb, rgb8, rec, counters, min_active); break;
    }
}

cudaError_t render_occupancy(int precision, int variant, int* blocks_per_sm)
{
    return precision == RT_FP64 ? occupancy_t<double>(variant, blocks_per_sm) : occupancy_t<float>(variant, blocks_per_sm);
}

cudaError_t launch_render(const DevScene& sc, int precision, int variant, int min_active, float* rgb, uint8_t* rgb8,
                          rt_ray_record* rec, unsigned long long* counters, int grid, cudaStream_t stream)
{
    if (precision == RT_FP64) launch_t<double>(sc, variant, min_active, rgb, rgb8, rec, counters, grid, stream);
    else launch_t<float>(sc, variant, min_active, rgb, rgb8, rec, counters, grid, stream);
    return cudaGetLastError();
}

cudaError_t launch_medium(int precision, double kA, double Lambda, const double* xy, int64_t n, double* out,
                          cudaStream_t stream)
{
    const int block = 128;
    const int64_t grid = (n + block - 1) / block;
    if (grid == 0) return cudaSuccess;
    if (precision == RT_FP64) medium_kernel<double><<<(unsigned)grid, block, 0, stream>>>(kA, Lambda, xy, n, out);
    else medium_kernel<float><<<(unsigned)grid, block, 0, stream>>>(kA, Lambda, xy, n, out);
    return cudaGetLastError();
}

}  // namespace grt
