// rt_batch.cu -- many scenes in one persistent launch replayed from a CUDA
// graph, and the autotuner of the launch configuration.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <atomic>

#include "rt_internal.h"
#include "rt_wave.cuh"

namespace grt {

// Many scenes in one launch of the wavefront loop: their samples form one
// work list, so the warps balance across scenes of uneven size.
template <class R, int INTEG, bool OPT>
static cudaError_t batch_prepare()
{
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(wave_batch_kernel<R, INTEG, OPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)wave_smem_bytes<R, INTEG>());
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
}

template <class R, int INTEG, bool OPT>
static cudaError_t batch_occupancy_t(int* bps)
{
    const cudaError_t e = batch_prepare<R, INTEG, OPT>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, wave_batch_kernel<R, INTEG, OPT>,
                                                         WaveShape<R, INTEG>::kBlock, wave_smem_bytes<R, INTEG>());
}

template <bool OPT>
static cudaError_t batch_occupancy_o(int precision, int integrator, int* bps)
{
    if (precision == RT_FP64) {
        if (integrator == RT_DP45) return batch_occupancy_t<double, RT_DP45, OPT>(bps);
        if (integrator == RT_RK4T) return batch_occupancy_t<double, RT_RK4T, OPT>(bps);
        return batch_occupancy_t<double, RT_RK4, OPT>(bps);
    }
    if (integrator == RT_DP45) return batch_occupancy_t<float, RT_DP45, OPT>(bps);
    if (integrator == RT_RK4T) return batch_occupancy_t<float, RT_RK4T, OPT>(bps);
    return batch_occupancy_t<float, RT_RK4, OPT>(bps);
}

cudaError_t batch_occupancy(int precision, int integrator, bool opt, int* bps)
{
    return opt ? batch_occupancy_o<true>(precision, integrator, bps)
               : batch_occupancy_o<false>(precision, integrator, bps);
}

template <class R, int INTEG, bool OPT>
static cudaError_t launch_batch_t(const BatchLaunch& L, cudaStream_t stream)
{
    const cudaError_t e = batch_prepare<R, INTEG, OPT>();
    if (e != cudaSuccess) return e;
    wave_batch_kernel<R, INTEG, OPT><<<L.grid, WaveShape<R, INTEG>::kBlock, wave_smem_bytes<R, INTEG>(), stream>>>(
        L.scenes, L.offsets, L.soffsets, L.rgbs, L.n, L.total, L.total_samples, L.scratch.col, L.scratch.cnt,
        L.scratch.br, L.counters, L.min_active);
    return cudaGetLastError();
}

template <bool OPT>
static cudaError_t launch_batch_o(int precision, int integrator, const BatchLaunch& L, cudaStream_t stream)
{
    if (precision == RT_FP64) {
        if (integrator == RT_DP45) return launch_batch_t<double, RT_DP45, OPT>(L, stream);
        if (integrator == RT_RK4T) return launch_batch_t<double, RT_RK4T, OPT>(L, stream);
        return launch_batch_t<double, RT_RK4, OPT>(L, stream);
    }
    if (integrator == RT_DP45) return launch_batch_t<float, RT_DP45, OPT>(L, stream);
    if (integrator == RT_RK4T) return launch_batch_t<float, RT_RK4T, OPT>(L, stream);
    return launch_batch_t<float, RT_RK4, OPT>(L, stream);
}

cudaError_t launch_batch(int precision, int integrator, const BatchLaunch& L, cudaStream_t stream)
{
    return L.opt ? launch_batch_o<true>(precision, integrator, L, stream)
                 : launch_batch_o<false>(precision, integrator, L, stream);
}

// ------------------------------------------------------------------------
// Autotuner cache: key -> (variant, min_active), for the process and
// optionally in the text file named by RT_AUTOTUNE_CACHE ("key variant
// min_active" per line).
// ------------------------------------------------------------------------
static std::mutex g_tune_mutex;
static std::map<std::string, std::pair<int, int>> g_tune;
static bool g_tune_loaded = false;

static void tune_load_locked()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = getenv("RT_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char key[256];
    int v, m;
    while (fscanf(f, "%255s %d %d", key, &v, &m) == 3) g_tune[key] = {v, m};
    fclose(f);
}

static void tune_store_locked()
{
    const char* path = getenv("RT_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "w");
    if (!f) return;
    for (const auto& kv : g_tune) fprintf(f, "%s %d %d\n", kv.first.c_str(), kv.second.first, kv.second.second);
    fclose(f);
}

bool tune_lookup(const std::string& key, int* variant, int* min_active)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    *variant = it->second.first;
    *min_active = it->second.second;
    return true;
}

void tune_record(const std::string& key, int variant, int min_active)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_load_locked();
    g_tune[key] = {variant, min_active};
    tune_store_locked();
}

}  // namespace grt

using namespace grt;

#define RT_CK(call)                                                                                   \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            set_error("%s:%d: %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));            \
            return RT_ECUDA;                                                                          \
        }                                                                                             \
    } while (0)

#define RT_REQ(cond, ...)                                                                             \
    do {                                                                                              \
        if (!(cond)) {                                                                                \
            set_error(__VA_ARGS__);                                                                   \
            return RT_EINVAL;                                                                         \
        }                                                                                             \
    } while (0)

struct rt_batch {
    int n, device, precision, integrator, grid, nsm, min_active;
    // The kernel's work list takes the scenes in slot order: slot j holds the
    // caller's scene order[j].  Cloaked scenes (rays that integrate) come
    // first, then bare gratings, then flat mirrors; within a kind the scene
    // with fewer samples first.  A scene's samples then start early enough
    // that its longest rays do not make the launch's tail: a centre line of
    // a cloaked render, taken after a million samples of cheap renders,
    // would.  The cheap air-only renders fill the end of the launch.
    std::vector<int> order;
    int64_t total, total_samples;
    DevScene* d_scenes;
    int64_t* d_offsets;      // first pixel of each scene
    int64_t* d_soffsets;     // first sample of each scene
    float* d_samp;           // per-sample colours of multi-sample pixels
    int* d_pcnt;             // per-pixel sample counters
    void* d_br;              // Fresnel branch queues (when a scene has RT_FLAG_FRESNEL)
    bool opt;                // a scene has options (RT_FLAG_*): the options build of the loop
    std::vector<DevScene> h_scenes;    // the table last uploaded
    DevScene* h_stage;       // pinned staging of rt_batch_update
    cudaEvent_t staged;      // the last staging copy is done
    float** d_rgbs;
    std::vector<float*> h_rgbs;        // output pointers last uploaded
    unsigned long long* d_counters;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int graph_min_active;
    cudaEvent_t done;
};

extern "C" {

int rt_batch_create(rt_scene* const* scenes, int32_t n, rt_batch** out)
{
    RT_REQ(out, "out is NULL");
    *out = nullptr;
    RT_REQ(scenes && n >= 1, "need at least one scene");
    std::vector<DevScene> user(n), dev(n);
    std::vector<int64_t> off(n + 1, 0), soff(n + 1, 0);
    int precision = -1, integrator = -1, device = -1;
    bool fresnel = false, opt = false;
    for (int i = 0; i < n; ++i) {
        RT_REQ(scenes[i], "scene %d is NULL", i);
        int p, g, d;
        if (scene_info(scenes[i], &user[i], &p, &g, &d) != RT_OK) return RT_EINVAL;
        RT_REQ(user[i].pix_list == nullptr, "scene %d", i);
        RT_REQ(user[i].mirror != RT_MIRROR_GAUSS, "scene %d: scenes of the Gaussian bump are rendered alone", i);
        if (i == 0) { precision = p; integrator = g; device = d; }
        RT_REQ(p == precision && g == integrator, "scenes of a batch must share precision and integrator (scene %d)", i);
        RT_REQ(d == device, "scenes of a batch must live on one device (scene %d)", i);
        fresnel = fresnel || (user[i].flags & RT_FLAG_FRESNEL);
        opt = opt || user[i].flags != 0;
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const DevScene &x = user[a], &y = user[c];
        if (x.cloak != y.cloak) return x.cloak > y.cloak;
        if (x.mirror != y.mirror) return x.mirror > y.mirror;
        return x.nwork * x.spp < y.nwork * y.spp;
    });
    int64_t cols = 0;                         // floats of pixel colour blocks
    for (int j = 0; j < n; ++j) {
        dev[j] = user[order[j]];
        off[j + 1] = off[j] + dev[j].nwork;
        soff[j + 1] = soff[j] + dev[j].nwork * dev[j].spp;
        dev[j].col_base = cols;
        if (dev[j].spp > 1) cols += dev[j].nwork * (col_block_bytes(dev[j].spp) >> 2);
    }
    int cur = -1;
    RT_CK(cudaGetDevice(&cur));
    RT_REQ(cur == device, "current device %d, scenes live on device %d", cur, device);
    rt_batch* b = new (std::nothrow) rt_batch();
    if (!b) { set_error("host allocation failed"); return RT_ENOMEM; }
    b->n = n;
    b->order = order;
    b->device = device;
    b->precision = precision;
    b->integrator = integrator;
    b->total = off[n];
    b->total_samples = soff[n];
    b->min_active = default_min_active(precision, integrator);
    b->graph_min_active = -1;
    b->h_rgbs.assign(n, nullptr);
    cudaError_t e = cudaMalloc(&b->d_scenes, sizeof(DevScene) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_offsets, sizeof(int64_t) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_soffsets, sizeof(int64_t) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_samp, sizeof(float) * (size_t)(cols > 0 ? cols : 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_pcnt, kScratchBytesPerPixel * (size_t)b->total);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_rgbs, sizeof(float*) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, sizeof(unsigned long long) * kCounters);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_scenes, dev.data(), sizeof(DevScene) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_offsets, off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_soffsets, soff.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_rgbs, 0, sizeof(float*) * n);
    if (e == cudaSuccess) e = cudaMemset(b->d_counters, 0, sizeof(unsigned long long) * kCounters);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    int bps = 0;
    b->opt = opt;
    b->h_scenes = dev;
    if (e == cudaSuccess) e = batch_occupancy(precision, integrator, opt, &bps);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        set_error("rt_batch_create: %s", cudaGetErrorString(e));
        rt_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA;
    }
    b->grid = (bps > 0 ? bps : 1) * b->nsm;
    if (fresnel) {
        e = cudaMalloc(&b->d_br, branch_queue_bytes(precision, integrator, b->grid));
        if (e != cudaSuccess) {
            set_error("rt_batch_create: %s", cudaGetErrorString(e));
            rt_batch_destroy(b);
            return RT_ENOMEM;
        }
    }
    *out = b;
    return RT_OK;
}

void rt_batch_destroy(rt_batch* b)
{
    if (!b) return;
    if (b->done) cudaEventSynchronize(b->done);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->d_scenes) cudaFree(b->d_scenes);
    if (b->d_offsets) cudaFree(b->d_offsets);
    if (b->d_soffsets) cudaFree(b->d_soffsets);
    if (b->d_samp) cudaFree(b->d_samp);
    if (b->d_pcnt) cudaFree(b->d_pcnt);
    if (b->d_br) cudaFree(b->d_br);
    if (b->staged) { cudaEventSynchronize(b->staged); cudaEventDestroy(b->staged); }
    if (b->h_stage) cudaFreeHost(b->h_stage);
    if (b->d_rgbs) cudaFree(b->d_rgbs);
    if (b->d_counters) cudaFree(b->d_counters);
    if (b->done) cudaEventDestroy(b->done);
    delete b;
}

int rt_batch_update(rt_batch* b, const rt_scene_desc* descs, int32_t n, void* stream, uint64_t* h2d_bytes)
{
    RT_REQ(b && descs, "batch and descs must not be NULL");
    RT_REQ(n == b->n, "the batch holds %d scenes, got %d descriptors", b->n, n);
    std::vector<DevScene> dev(n);
    for (int j = 0; j < n; ++j) {
        const int i = b->order[j];           // the caller's index of slot j
        if (rt_validate_desc(&descs[i]) != RT_OK) return RT_EINVAL;
        const DevScene& old = b->h_scenes[j];
        build_scene_table(&descs[i], &dev[j]);
        RT_REQ(descs[i].precision == b->precision && descs[i].integrator == b->integrator,
               "scene %d: precision and integrator must stay", i);
        RT_REQ(dev[j].nwork == old.nwork && dev[j].spp == old.spp && dev[j].wout == old.wout,
               "scene %d: image size and samples per pixel must stay", i);
        RT_REQ(dev[j].background == old.background && dev[j].flags == old.flags &&
                   dev[j].cloak == old.cloak && dev[j].mirror == old.mirror,
               "scene %d: background kind, flags, mirror and cloak must stay", i);
        dev[j].tex = old.tex;
        dev[j].tex_size = old.tex_size;
        dev[j].pix_list = nullptr;
        dev[j].col_base = old.col_base;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(DevScene) * (size_t)n;
    if (!b->h_stage) {
        RT_CK(cudaMallocHost((void**)&b->h_stage, bytes));
        RT_CK(cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming));
    } else {
        RT_CK(cudaEventSynchronize(b->staged));     // the previous copy has left the staging buffer
    }
    memcpy(b->h_stage, dev.data(), bytes);
    RT_CK(cudaMemcpyAsync(b->d_scenes, b->h_stage, bytes, cudaMemcpyHostToDevice, st));
    RT_CK(cudaEventRecord(b->staged, st));
    b->h_scenes = dev;
    if (h2d_bytes) *h2d_bytes = bytes;
    return RT_OK;
}

int rt_batch_render(rt_batch* b, float* const* d_rgb, void* stream)
{
    RT_REQ(b && d_rgb, "batch and d_rgb must not be NULL");
    for (int i = 0; i < b->n; ++i) RT_REQ(d_rgb[i], "d_rgb[%d] is NULL", i);
    cudaStream_t st = (cudaStream_t)stream;
    // a change of output images is a small upload outside the graph
    bool changed = false;
    for (int j = 0; j < b->n; ++j) changed = changed || (b->h_rgbs[j] != d_rgb[b->order[j]]);
    if (changed) {
        for (int j = 0; j < b->n; ++j) b->h_rgbs[j] = d_rgb[b->order[j]];
        RT_CK(cudaMemcpyAsync(b->d_rgbs, b->h_rgbs.data(), sizeof(float*) * b->n, cudaMemcpyHostToDevice, st));
        RT_CK(cudaStreamSynchronize(st));
    }
    if (!b->exec || b->graph_min_active != b->min_active) {
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        // record the launch (counter reset and the persistent kernel) once
        cudaStream_t cap;
        RT_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned long long) * kCounters, cap);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_pcnt, 0, kScratchBytesPerPixel * (size_t)b->total, cap);
        const BatchLaunch L = {b->d_scenes, b->d_offsets, b->d_soffsets, b->d_rgbs, b->n, b->total,
                               b->total_samples, {b->d_samp, b->d_pcnt, b->d_br}, b->d_counters, b->min_active,
                               b->grid, b->opt};
        if (e == cudaSuccess) e = launch_batch(b->precision, b->integrator, L, cap);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        RT_CK(e);
        RT_CK(e2);
        b->graph = g;
        RT_CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
        b->graph_min_active = b->min_active;
    }
    RT_CK(cudaGraphLaunch(b->exec, st));
    RT_CK(cudaEventRecord(b->done, st));
    return RT_OK;
}

int rt_batch_stats(rt_batch* b, rt_stats* out)
{
    RT_REQ(b && out, "batch and out must not be NULL");
    unsigned long long c[kCounters];
    RT_CK(cudaEventSynchronize(b->done));
    RT_CK(cudaMemcpy(c, b->d_counters, sizeof c, cudaMemcpyDeviceToHost));
    counters_to_stats(c, out);
    if (out->sched_timeouts) {
        set_error("the last render of this batch gave up %llu bounded waits of its work queues; its images are "
                  "incomplete", (unsigned long long)out->sched_timeouts);
        return RT_ETIMEDOUT;
    }
    return RT_OK;
}

int rt_batch_set_launch(rt_batch* b, int32_t min_active)
{
    RT_REQ(b, "batch is NULL");
    RT_REQ(min_active >= 1 && min_active <= 32, "min_active must be 1..32");
    b->min_active = min_active;
    return RT_OK;
}

int rt_batch_get_launch(rt_batch* b, int32_t* min_active, int32_t* grid, int64_t* total)
{
    RT_REQ(b, "batch is NULL");
    if (min_active) *min_active = b->min_active;
    if (grid) *grid = b->grid;
    if (total) *total = b->total;
    return RT_OK;
}

// Time one configuration: median of `trials` renders (after one warm-up).
static int time_batch(rt_batch* b, float* const* d_rgb, cudaStream_t st, int trials, float* ms)
{
    cudaEvent_t e0, e1;
    RT_CK(cudaEventCreate(&e0));
    RT_CK(cudaEventCreate(&e1));
    std::vector<float> t;
    int rc = rt_batch_render(b, d_rgb, st);
    for (int k = 0; rc == RT_OK && k < trials; ++k) {
        cudaEventRecord(e0, st);
        rc = rt_batch_render(b, d_rgb, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float x = 0.0f;
        cudaEventElapsedTime(&x, e0, e1);
        t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != RT_OK) return rc;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return RT_OK;
}

int rt_batch_autotune(rt_batch* b, float* const* d_rgb, int32_t trials, void* stream, int32_t* min_active_out)
{
    RT_REQ(b && d_rgb, "batch and d_rgb must not be NULL");
    RT_REQ(trials >= 1 && trials <= 64, "trials must be 1..64");
    char key[128];
    snprintf(key, sizeof key, "batch/p%d/i%d/n%d", b->precision, b->integrator, b->n);
    int v = 0, m = 0;
    if (!tune_lookup(key, &v, &m)) {
        const int cand[] = {12, 16, 20, 24, 28};
        float best = 1e30f;
        m = default_min_active(b->precision, b->integrator);
        for (int c : cand) {
            b->min_active = c;
            float ms = 0.0f;
            const int rc = time_batch(b, d_rgb, (cudaStream_t)stream, trials, &ms);
            if (rc != RT_OK) return rc;
            if (ms < best) { best = ms; m = c; }
        }
        tune_record(key, 0, m);
    }
    b->min_active = m;
    if (min_active_out) *min_active_out = m;
    return RT_OK;
}

}  // extern "C"
