// rt_render.cu -- instantiations and launchers of the render and medium
// kernels (the kernels themselves are in rt_trace.cuh and rt_wave.cuh).
#include <atomic>
#include <cmath>
#include <mutex>

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
    return allow_smem(wave_kernel<R, INTEG, OPT>, wave_smem_bytes<R, INTEG>(), done);
}

// Register-budget variants of the per-lane loop are compiled for the FP32 RK4
// kernel, the one the benchmark times; the other (precision, integrator)
// pairs have one each, but for the time form (RT_RK4T) and the Gaussian
// bump, which have none.  Every pair has the wavefront loop; the Gaussian
// bump has its plain build only.
template <class R, int INTEG>
static cudaError_t occupancy_t(int variant, bool opt, int* bps)
{
    if (variant == kVariantWave) {
        if constexpr (!gauss_of(INTEG)) {
            if (opt) {
                const cudaError_t e = wave_prepare<R, INTEG, true>();
                if (e != cudaSuccess) return e;
                return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, wave_kernel<R, INTEG, true>,
                                                                     WaveShape<R, INTEG>::kBlock,
                                                                     wave_smem_bytes<R, INTEG>());
            }
        }
        const cudaError_t e = wave_prepare<R, INTEG, false>();
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, wave_kernel<R, INTEG, false>,
                                                             WaveShape<R, INTEG>::kBlock, wave_smem_bytes<R, INTEG>());
    }
    if constexpr (integ_of(INTEG) == RT_RK4T || gauss_of(INTEG)) {
        return cudaErrorInvalidValue;                // the wavefront loop only
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
                            const WaitLimit& wl, cudaStream_t stream)
{
    if (variant == kVariantWave) {
        // scenes with options (RT_FLAG_*) take the options build of the loop;
        // the Gaussian bump has none
        if constexpr (!gauss_of(INTEG)) {
            if (sc.flags) {
                const cudaError_t e = wave_prepare<R, INTEG, true>();
                if (e != cudaSuccess) return e;
                wave_kernel<R, INTEG, true><<<grid, WaveShape<R, INTEG>::kBlock, wave_smem_bytes<R, INTEG>(), stream>>>(
                    sc, rgb, rgb8, rec, counters, min_active, ss.col, ss.cnt, ss.br, WaveWait{wl.spin, wl.hold});
                return cudaGetLastError();
            }
        }
        const cudaError_t e = wave_prepare<R, INTEG, false>();
        if (e != cudaSuccess) return e;
        wave_kernel<R, INTEG, false><<<grid, WaveShape<R, INTEG>::kBlock, wave_smem_bytes<R, INTEG>(), stream>>>(
            sc, rgb, rgb8, rec, counters, min_active, ss.col, ss.cnt, ss.br, WaveWait{wl.spin, wl.hold});
        return cudaGetLastError();
    }
    if constexpr (integ_of(INTEG) == RT_RK4T || gauss_of(INTEG)) {
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

// Coefficients a_1..a_N of Weideman's series for the Faddeeva function
// (rt_gauss.cuh), then L = 2^(-1/4) N^(1/2): a_n is the n-th Fourier
// coefficient of (L^2 + t^2) exp(-t^2), t = L tan(theta/2), by the midpoint
// rule on 8192 angles (the integrand is smooth and periodic).
static void weideman_coefficients(int N, double* out)
{
    const int M = 8192;
    const double L = std::pow(2.0, -0.25) * std::sqrt((double)N);
    for (int n = 1; n <= N; ++n) {
        double acc = 0.0;
        for (int j = 0; j < M; ++j) {
            const double th = -kPi + (j + 0.5) * (2.0 * kPi / M);
            const double t = L * std::tan(0.5 * th);
            acc += (L * L + t * t) * std::exp(-t * t) * std::cos(n * th);
        }
        out[n - 1] = acc / M;
    }
    out[N] = L;
}

cudaError_t gauss_upload()
{
    static std::once_flag once;
    static double ad[kWNd + 1];
    static float af[kWNf + 1];
    std::call_once(once, [] {
        double tf[kWNf + 1];
        weideman_coefficients(kWNd, ad);
        weideman_coefficients(kWNf, tf);
        for (int n = 0; n <= kWNf; ++n) af[n] = (float)tf[n];
    });
    static std::atomic<unsigned long long> done{0};
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return cudaSuccess;
    std::lock_guard<std::mutex> lock(mu);
    if (done.load() & bit) return cudaSuccess;
    e = cudaMemcpyToSymbol(kWad, ad, sizeof ad);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(kWaf, af, sizeof af);
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
}

size_t branch_queue_bytes(int precision, int integrator, int grid)
{
    if (precision == RT_FP64) return wave_branch_bytes<double, RT_RK4>(grid);
    return integ_of(integrator) == RT_DP45 ? wave_branch_bytes<float, RT_DP45>(grid)
                                           : wave_branch_bytes<float, RT_RK4>(grid);
}

bool variant_compiled(int precision, int integrator, int variant)
{
    if (variant == kVariantWave) return true;
    if (integrator == RT_RK4T || (integrator & kModeGauss)) return false;
    if (variant == 0) return true;
    return precision == RT_FP32 && integrator == RT_RK4 && variant >= 0 && variant < kLaneVariants;
}

cudaError_t render_occupancy(int precision, int integrator, int variant, bool opt, int* blocks_per_sm)
{
    constexpr int G = kModeGauss;
    if (precision == RT_FP64) {
        switch (integrator) {
            case RT_DP45: return occupancy_t<double, RT_DP45>(variant, opt, blocks_per_sm);
            case RT_RK4T: return occupancy_t<double, RT_RK4T>(variant, opt, blocks_per_sm);
            case RT_RK4 | G: return occupancy_t<double, RT_RK4 | G>(variant, false, blocks_per_sm);
            case RT_DP45 | G: return occupancy_t<double, RT_DP45 | G>(variant, false, blocks_per_sm);
            default: return occupancy_t<double, RT_RK4>(variant, opt, blocks_per_sm);
        }
    }
    switch (integrator) {
        case RT_DP45: return occupancy_t<float, RT_DP45>(variant, opt, blocks_per_sm);
        case RT_RK4T: return occupancy_t<float, RT_RK4T>(variant, opt, blocks_per_sm);
        case RT_RK4 | G: return occupancy_t<float, RT_RK4 | G>(variant, false, blocks_per_sm);
        case RT_DP45 | G: return occupancy_t<float, RT_DP45 | G>(variant, false, blocks_per_sm);
        default: return occupancy_t<float, RT_RK4>(variant, opt, blocks_per_sm);
    }
}

cudaError_t launch_render(const DevScene& sc, int precision, int variant, int min_active, float* rgb, uint8_t* rgb8,
                          rt_ray_record* rec, unsigned long long* counters, int grid, const SampleScratch& ss,
                          const WaitLimit& wl, cudaStream_t stream)
{
    constexpr int G = kModeGauss;
    const int mode = sc.integrator | (sc.mirror == RT_MIRROR_GAUSS ? G : 0);
#define RT_LAUNCH(RR, M) return launch_t<RR, M>(sc, variant, min_active, rgb, rgb8, rec, counters, grid, ss, wl, stream)
    if (precision == RT_FP64) {
        switch (mode) {
            case RT_DP45: RT_LAUNCH(double, RT_DP45);
            case RT_RK4T: RT_LAUNCH(double, RT_RK4T);
            case RT_RK4 | G: RT_LAUNCH(double, RT_RK4 | G);
            case RT_DP45 | G: RT_LAUNCH(double, RT_DP45 | G);
            default: RT_LAUNCH(double, RT_RK4);
        }
    }
    switch (mode) {
        case RT_DP45: RT_LAUNCH(float, RT_DP45);
        case RT_RK4T: RT_LAUNCH(float, RT_RK4T);
        case RT_RK4 | G: RT_LAUNCH(float, RT_RK4 | G);
        case RT_DP45 | G: RT_LAUNCH(float, RT_DP45 | G);
        default: RT_LAUNCH(float, RT_RK4);
    }
#undef RT_LAUNCH
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
