// rt_render.cu -- instantiations and launchers of the render and medium
// kernels (the kernels themselves are in rt_trace.cuh).
#include "rt_trace.cuh"

namespace grt {

// Register-budget variants are compiled for the FP32 RK4 kernel, the one the
// benchmark times; the other (precision, integrator) pairs have one each.
template <class R, int INTEG>
static cudaError_t occupancy_t(int variant, int* bps)
{
    if constexpr (sizeof(R) == 4 && INTEG == RT_RK4) {
        if (variant == 1)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, render_kernel<R, kVariantBlocks[1], INTEG>, kRenderBlock, 0);
        if (variant == 2)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, render_kernel<R, kVariantBlocks[2], INTEG>, kRenderBlock, 0);
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, render_kernel<R, kVariantBlocks[0], INTEG>, kRenderBlock, 0);
}

template <class R, int INTEG>
static void launch_t(const DevScene& sc, int variant, int min_active, float* rgb, uint8_t* rgb8, rt_ray_record* rec,
                     unsigned long long* counters, int grid, cudaStream_t stream)
{
    if constexpr (sizeof(R) == 4 && INTEG == RT_RK4) {
        if (variant == 1) {
            render_kernel<R, kVariantBlocks[1], INTEG><<<grid, kRenderBlock, 0, stream>>>(sc, rgb, rgb8, rec, counters, min_active);
            return;
        }
        if (variant == 2) {
            render_kernel<R, kVariantBlocks[2], INTEG><<<grid, kRenderBlock, 0, stream>>>(sc, rgb, rgb8, rec, counters, min_active);
            return;
        }
    }
    render_kernel<R, kVariantBlocks[0], INTEG><<<grid, kRenderBlock, 0, stream>>>(sc, rgb, rgb8, rec, counters, min_active);
}

cudaError_t render_occupancy(int precision, int integrator, int variant, int* blocks_per_sm)
{
    if (precision == RT_FP64)
        return integrator == RT_DP45 ? occupancy_t<double, RT_DP45>(variant, blocks_per_sm)
                                     : occupancy_t<double, RT_RK4>(variant, blocks_per_sm);
    return integrator == RT_DP45 ? occupancy_t<float, RT_DP45>(variant, blocks_per_sm)
                                 : occupancy_t<float, RT_RK4>(variant, blocks_per_sm);
}

cudaError_t launch_render(const DevScene& sc, int precision, int variant, int min_active, float* rgb, uint8_t* rgb8,
                          rt_ray_record* rec, unsigned long long* counters, int grid, cudaStream_t stream)
{
    if (precision == RT_FP64) {
        if (sc.integrator == RT_DP45) launch_t<double, RT_DP45>(sc, variant, min_active, rgb, rgb8, rec, counters, grid, stream);
        else launch_t<double, RT_RK4>(sc, variant, min_active, rgb, rgb8, rec, counters, grid, stream);
    } else {
        if (sc.integrator == RT_DP45) launch_t<float, RT_DP45>(sc, variant, min_active, rgb, rgb8, rec, counters, grid, stream);
        else launch_t<float, RT_RK4>(sc, variant, min_active, rgb, rgb8, rec, counters, grid, stream);
    }
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
