// rt_render.cu -- instantiations and launchers of the render and medium
// kernels (the kernels themselves are in rt_trace.cuh and rt_wave.cuh).
#include <atomic>

#include "rt_wave.cuh"

namespace grt {

// The wavefront kernels keep their pixel pool in dynamic shared memory above
// the default 48 KB; the limit is raised once per kernel and device.
template <class K>
static cudaError_t allow_smem(K kernel, size_t bytes, std::atomic<unsigned long long>& done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
}

template <class R, int INTEG, bool OPT>
static cudaError_t wave_prepare()
{
    static std::atomic<unsigned long long> done{0};
    return allow_smem(wave_kernel<R, INTEG, OPT>, wave_smem_bytes<R>(), done);
}

// Register-budget variants of the per-lane loop are compiled for the FP32 RK4
// kernel, the one the benchmark times; the other (precision, integrator)
// pairs have one each, but for the time form (RT_RK4T), which has none.
// Every pair has the wavefront loop.
template <class R, int INTEG>
static cudaError_t occupancy_t(int variant, bool opt, int* bps)
{
    if (variant == kVariantWave) {
        if (opt) {
            const cudaError_t e = wave_prepare<R, INTEG, true>();
            if (e != cudaSuccess) return e;
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, wave_kernel<R, INTEG, true>, kWaveBlock,
                                                                 wave_smem_bytes<R>());
        }
        const cudaError_t e = wave_prepare<R, INTEG, false>();
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, wave_kernel<R, INTEG, false>, kWaveBlock,
                                                             wave_smem_bytes<R>());
    }
    if constexpr (INTEG == RT_RK4T) {
        return cudaErrorInvalidValue;                // the time form runs in the wavefront loop only
    } else {
    if constexpr (sizeof(R) == 4 && INTEG == RT_RK4) {
        if (variant == 1)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, render_kernel<R, kVariantBlocks[1], INTEG>, kRenderBlock, 0);
        if (variant == 2)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, render_kernel<R, kVariantBlocks[2], INTEG>, kRenderBlock, 0);
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, render_kernel<R, kVariantBlocks[0], INTEG>, kRenderBlock, 0);
    }
}

template <class R, int INTEG>
static cudaError_t launch_t(const DevScene& sc, int variant, int min_active, float* rgb, uint8_t* rgb8,
                            rt_ray_record* rec, unsigned long long* counters, int grid, const SampleScratch& ss,
                            cudaStream_t stream)
{
    if (variant == kVariantWave) {
        // scenes with options (RT_FLAG_*) take the options build of the loop
        if (sc.flags) {
            const cudaError_t e = wave_prepare<R, INTEG, true>();
            if (e != cudaSuccess) return e;
            wave_kernel<R, INTEG, true><<<grid, kWaveBlock, wave_smem_bytes<R>(), stream>>>(
                sc, rgb, rgb8, rec, counters, min_active, ss.col, ss.cnt, ss.br);
            return cudaGetLastError();
        }
        const cudaError_t e = wave_prepare<R, INTEG, false>();
        if (e != cudaSuccess) return e;
        wave_kernel<R, INTEG, false><<<grid, kWaveBlock, wave_smem_bytes<R>(), stream>>>(
            sc, rgb, rgb8, rec, counters, min_active, ss.col, ss.cnt, ss.br);
        return cudaGetLastError();
    }
    if constexpr (INTEG == RT_RK4T) {
        return cudaErrorInvalidValue;
    } else {
    if constexpr (sizeof(R) == 4 && INTEG == RT_RK4) {
        if (variant == 1) {
            render_kernel<R, kVariantBlocks[1], INTEG><<<grid, kRenderBlock, 0, stream>>>(sc, rgb, rgb8, rec, counters, min_active);
            return cudaGetLastError();
        }
        if (variant == 2) {
            render_kernel<R, kVariantBlocks[2], INTEG><<<grid, kRenderBlock, 0, stream>>>(sc, rgb, rgb8, rec, counters, min_active);
            return cudaGetLastError();
        }
    }
    render_kernel<R, kVariantBlocks[0], INTEG><<<grid, kRenderBlock, 0, stream>>>(sc, rgb, rgb8, rec, counters, min_active);
    return cudaGetLastError();
    }
}

size_t branch_queue_bytes(int precision, int grid)
{
    return precision == RT_FP64 ? wave_branch_bytes<double>(grid) : wave_branch_bytes<float>(grid);
}

bool variant_compiled(int precision, int integrator, int variant)
{
    if (variant == kVariantWave) return true;
    if (integrator == RT_RK4T) return false;
    if (variant == 0) return true;
    return precision == RT_FP32 && integrator == RT_RK4 && variant >= 0 && variant < kLaneVariants;
}

cudaError_t render_occupancy(int precision, int integrator, int variant, bool opt, int* blocks_per_sm)
{
    if (precision == RT_FP64) {
        if (integrator == RT_DP45) return occupancy_t<double, RT_DP45>(variant, opt, blocks_per_sm);
        if (integrator == RT_RK4T) return occupancy_t<double, RT_RK4T>(variant, opt, blocks_per_sm);
        return occupancy_t<double, RT_RK4>(variant, opt, blocks_per_sm);
    }
    if (integrator == RT_DP45) return occupancy_t<float, RT_DP45>(variant, opt, blocks_per_sm);
    if (integrator == RT_RK4T) return occupancy_t<float, RT_RK4T>(variant, opt, blocks_per_sm);
    return occupancy_t<float, RT_RK4>(variant, opt, blocks_per_sm);
}

cudaError_t launch_render(const DevScene& sc, int precision, int variant, int min_active, float* rgb, uint8_t* rgb8,
                          rt_ray_record* rec, unsigned long long* counters, int grid, const SampleScratch& ss,
                          cudaStream_t stream)
{
    if (precision == RT_FP64) {
        if (sc.integrator == RT_DP45)
            return launch_t<double, RT_DP45>(sc, variant, min_active, rgb, rgb8, rec, counters, grid, ss, stream);
        if (sc.integrator == RT_RK4T)
            return launch_t<double, RT_RK4T>(sc, variant, min_active, rgb, rgb8, rec, counters, grid, ss, stream);
        return launch_t<double, RT_RK4>(sc, variant, min_active, rgb, rgb8, rec, counters, grid, ss, stream);
    }
    if (sc.integrator == RT_DP45)
        return launch_t<float, RT_DP45>(sc, variant, min_active, rgb, rgb8, rec, counters, grid, ss, stream);
    if (sc.integrator == RT_RK4T)
        return launch_t<float, RT_RK4T>(sc, variant, min_active, rgb, rgb8, rec, counters, grid, ss, stream);
    return launch_t<float, RT_RK4>(sc, variant, min_active, rgb, rgb8, rec, counters, grid, ss, stream);
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
