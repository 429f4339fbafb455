// rt_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "rt.h"
#include "rt_device.cuh"

namespace grt {

constexpr int kRenderBlock = 128;
// Compiled register budgets of the render kernel: resident blocks of
// kRenderBlock threads per SM that each variant is sized for.
constexpr int kVariants = 3;
constexpr int kVariantBlocks[kVariants] = {4, 5, 6};
constexpr int kDefaultVariant = 0;
constexpr int kMinActive = 24;   // step while at least this many lanes of a warp are inside the cloak
constexpr int kMaxWindows = 16;
constexpr int kCounters = 16;      // [0] work counter, [1..11] statistics, [12..15] optional profile

#ifndef RT_PROFILE
#define RT_PROFILE 0
#endif

struct Windows {
    int n;
    int j0[kMaxWindows], j1[kMaxWindows];
};

cudaError_t render_occupancy(int precision, int integrator, int variant, int* blocks_per_sm);
cudaError_t launch_render(const DevScene& sc, int precision, int variant, int min_active, float* rgb, uint8_t* rgb8,
                          rt_ray_record* rec, unsigned long long* counters, int grid, cudaStream_t stream);
cudaError_t launch_medium(int precision, double kA, double Lambda, const double* xy, int64_t n, double* out,
                          cudaStream_t stream);

// Cross-correlation: column moments into `partial` (nchunks x W*C double4),
// then one block per window.
int xcorr_chunks(int H);
cudaError_t launch_xcorr(const float* f, const float* g, int H, int W, int C, const Windows& win, void* partial,
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
cudaError_t batch_occupancy(int precision, int integrator, int* bps);
cudaError_t launch_batch(int precision, int integrator, const DevScene* scenes, const int64_t* offsets,
                         float* const* rgbs, int n, int64_t total, unsigned long long* counters, int min_active,
                         int grid, cudaStream_t stream);
void tune_record(const std::string& key, int variant, int min_active);

}  // namespace grt
