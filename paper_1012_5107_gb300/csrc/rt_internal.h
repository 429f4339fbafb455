// rt_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "rt.h"
#include "rt_device.cuh"

namespace grt {

constexpr int kRenderBlock = 128;
// Launch variants of the render: 0..2 are the per-lane loop (rt_trace.cuh)
// compiled for 4, 5 and 6 resident blocks of kRenderBlock threads per SM;
// kVariantWave is the wavefront loop (rt_wave.cuh).
constexpr int kVariants = 4;
constexpr int kLaneVariants = 3;
constexpr int kVariantBlocks[kLaneVariants] = {4, 5, 6};
constexpr int kVariantWave = 3;
constexpr int kDefaultVariant = kVariantWave;
// An integration task continues while at least this many of its 32 rays are
// inside the cloak.  Measured on the current kernels (CUDA events): the FP32
// RK4 grating loop is fastest at 24 (the step's batched launch 7.25 ms, 7.34
// at 28, 7.87 at 30); the FP32 time form and Gaussian medium at 28 (time form
// 9.21 ms, 9.35 at 24, 9.47 at 30; Gaussian 9.39 / 9.49 ms at 28 / 24); the
// FP64 loops, bound by the FP64 pipe, with full warps only (FP64 cloaked
// render 590 ms at 32, 595 at 30, 605 at 28, 623 at 24).
constexpr int kMinActive = 28;
constexpr int kMinActiveRK4F32 = 24;
constexpr int kMinActiveF64 = 32;
// Dormand-Prince steps are longer: a task holding fewer rays is still worth
// running (1920 x 1080 x 16 with one block of 384 threads per SM, E = 8 / 32:
// 133.0 / 214.8 ms at 8, 135.1 / 221.5 ms at 16; 2 to 10 within 1 %)
constexpr int kMinActiveDP45 = 8;
// The default for a precision (RT_FP32 / RT_FP64) and render mode (the
// integrator, with kModeGauss for the Gaussian bump).
inline int default_min_active(int precision, int mode)
{
    if ((mode & 7) == RT_DP45) return kMinActiveDP45;
    if (precision == RT_FP64) return kMinActiveF64;
    if (mode == RT_RK4) return kMinActiveRK4F32;
    return kMinActive;
}
constexpr int kMaxWindows = 16;
// Render mode: the integrator (RT_RK4, RT_DP45, RT_RK4T), with kModeGauss set
// for scenes of the Gaussian bump, whose box holds the Gaussian map's medium.
constexpr int kModeGauss = 8;
inline int render_mode(const rt_scene_desc& d)
{
    return d.integrator | (d.mirror == RT_MIRROR_GAUSS ? kModeGauss : 0);
}
// Coefficients of the Faddeeva series of the Gaussian cloak, uploaded once
// per device before its first Gaussian scene.
cudaError_t gauss_upload();
constexpr int kCounters = 17;      // [0] work counter, [1..11] statistics, [12..15] optional profile,
                                   // [16] wavefront-loop waits that timed out

#ifndef RT_PROFILE
#define RT_PROFILE 0
#endif

struct Windows {
    int n;
    int j0[kMaxWindows], j1[kMaxWindows];
};

// Whether launch variant `variant` exists for this precision and render mode.
bool variant_compiled(int precision, int mode, int variant);
// opt: the options build of the wavefront loop (scenes with RT_FLAG_* set)
cudaError_t render_occupancy(int precision, int mode, int variant, bool opt, int* blocks_per_sm);
// Scratch of the wavefront loop for pixels of several samples: 3 floats per
// sample (col) and one counter per pixel (cnt, zero at launch).
struct SampleScratch {
    float* col;
    int* cnt;
    void* br;        // Fresnel branch queues (RT_FLAG_FRESNEL), see wave_branch_bytes
};
// Bytes of the Fresnel branch queues a wavefront launch of `grid` blocks of
// this precision and integrator needs.
size_t branch_queue_bytes(int precision, int integrator, int grid);
constexpr size_t kScratchBytesPerSample = 3 * sizeof(float);
constexpr size_t kScratchBytesPerPixel = sizeof(int);
// The colours of a pixel's samples sit in one block of whole 128-byte L2
// lines, 16 bytes a sample (three floats and a pad, so that every 32-byte
// sector is written in full): once the pixel's last sample has summed them,
// the lines are discarded from L2 without being written back to DRAM.
__host__ __device__ constexpr int64_t col_block_bytes(int spp) { return ((int64_t)spp * 16 + 127) / 128 * 128; }

// Bounds of the wavefront loop's waits on its work queues: attempts per wait
// and whether every block starts with its queue lock held (rt_scene_set_wait_limit).
constexpr int kDefaultWaitSpin = 1 << 24;
struct WaitLimit {
    int spin;
    int hold;
};
cudaError_t launch_render(const DevScene& sc, int precision, int variant, int min_active, float* rgb, uint8_t* rgb8,
                          rt_ray_record* rec, unsigned long long* counters, int grid, const SampleScratch& ss,
                          const WaitLimit& wl, cudaStream_t stream);
cudaError_t launch_medium(int precision, double kA, double Lambda, const double* xy, int64_t n, double* out,
                          cudaStream_t stream);

// Cross-correlation: column moments per row chunk (nchunks x W*C double4,
// padded to 256 bytes), then window slices (kXcorrTailBytes), then C.
// `scratch` holds xcorr_scratch_bytes(H, W, C) bytes, 256-byte aligned (none
// for the small images that one block takes).
constexpr size_t kXcorrTailBytes = 129 * 1024;
int xcorr_chunks(int H);
size_t xcorr_scratch_bytes(int H, int W, int C);
cudaError_t launch_xcorr(const float* f, const float* g, int H, int W, int C, const Windows& win, void* scratch,
                         double* out, cudaStream_t stream);

// Columns of a width-W image inside each field of view (host).
void fov_windows(int W, double hfov_deg, const double* fov_deg, int n_fov, Windows* win);

void set_error(const char* fmt, ...);

}  // namespace grt

struct rt_scene;

namespace grt {

// Scene table, precision, integrator and device of a scene.
int scene_info(rt_scene* s, DevScene* dev, int* precision, int* integrator, int* device);
void counters_to_stats(const unsigned long long* c, rt_stats* out);

// Autotuner cache (process lifetime, optionally the RT_AUTOTUNE_CACHE file).
}  // namespace grt
#include <string>
namespace grt {
bool tune_lookup(const std::string& key, int* variant, int* min_active);
// Scene table of a validated descriptor (texture pointer left to the caller).
void build_scene_table(const rt_scene_desc* d, DevScene* s);
cudaError_t batch_occupancy(int precision, int integrator, bool opt, int* bps);
// One launch of the wavefront loop over the pixels of n scenes (device tables).
struct BatchLaunch {
    const DevScene* scenes;
    const int64_t* offsets;      // n + 1: first pixel of each scene
    const int64_t* soffsets;     // n + 1: first sample of each scene
    float* const* rgbs;          // n output images
    int n;
    int64_t total, total_samples;
    SampleScratch scratch;       // for total_samples samples and total pixels
    unsigned long long* counters;
    int min_active, grid;
    bool opt;                    // a scene has options (RT_FLAG_*): the options build
};
cudaError_t launch_batch(int precision, int integrator, const BatchLaunch& L, cudaStream_t stream);
void tune_record(const std::string& key, int variant, int min_active);

}  // namespace grt
