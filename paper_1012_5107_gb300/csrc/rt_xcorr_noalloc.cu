// rt_xcorr_noalloc.cu -- the image cross-correlation of rt_xcorr for callers
// that cannot allocate device memory.
//
// Some callers cannot allocate: hosts that hand all device memory to their
// own pool and forbid allocations behind its back, and latency-bound loops
// in which an allocation call (which can synchronise the device or take a
// driver lock) is not acceptable.  This entry point runs the same
// kernels as rt_xcorr but keeps their scratch -- the per-chunk column
// moments and the window slices -- in the file-scope device array below
// instead of allocating it.
//
// The array is a fixed 16 MiB (and the slices' 129 KiB) that every GPU
// which loads the library holds until the process exits.  Host code must not pass the array's name to a
// kernel: in host code it names a host-side stand-in, not device memory.  The
// device address is taken with cudaGetSymbolAddress, once per device, with
// that device current, by the first call of rt_xcorr_noalloc on the device,
// and kept for the life of the process: a cudaDeviceReset of that device
// invalidates it (the module is loaded again, possibly elsewhere), so the
// entry point must not be used on a device after resetting it.
#include <cstdio>
#include <mutex>

#include "rt_internal.h"

namespace grt {

struct alignas(32) NoallocMoments {
    double v[4];
};

// Largest column-moment scratch in 32-byte moment records: 16 MiB; the array
// adds the window slices and the padding between the two.
constexpr size_t kNoallocMoments = (size_t)16 << 20 >> 5;
constexpr size_t kNoallocRecords = kNoallocMoments + (kXcorrTailBytes + 256) / sizeof(NoallocMoments);

static __device__ __align__(256) NoallocMoments g_xcorr_scratch[kNoallocRecords];

constexpr int kNoallocMaxDevices = 64;
static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[kNoallocMaxDevices];

// Device address of the scratch array on device `dev` (current), looked up on
// first use and cached; nullptr with the error in `err` on failure.
static void* noalloc_scratch(int dev, cudaError_t* err)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_xcorr_scratch);
        if (e != cudaSuccess) {
            *err = e;
            return nullptr;
        }
        g_noalloc_ptr[dev] = p;
    }
    *err = cudaSuccess;
    return g_noalloc_ptr[dev];
}

}  // namespace grt

using namespace grt;

extern "C" int rt_xcorr_noalloc(const float* d_f, const float* d_g, int32_t height, int32_t width, int32_t channels,
                                const double* fov_deg, int32_t n_fov, double hfov_deg, double* d_out, void* stream)
{
    set_error("%s", "");             // no stale message from an earlier call
    if (!d_f || !d_g || !d_out || !fov_deg) { set_error("null pointer argument"); return RT_EINVAL; }
    if (height < 1 || width < 1) { set_error("height and width must be >= 1"); return RT_EINVAL; }
    if (channels < 1 || channels > 4) { set_error("channels must be 1..4"); return RT_EINVAL; }
    if (n_fov < 1 || n_fov > kMaxWindows) { set_error("n_fov must be 1..%d", kMaxWindows); return RT_EINVAL; }
    if (!(hfov_deg > 0.0 && hfov_deg < 180.0)) { set_error("hfov_deg must be in (0, 180)"); return RT_EINVAL; }
    for (int q = 0; q < n_fov; ++q)
        if (!(fov_deg[q] >= 0.0)) { set_error("fov_deg must be >= 0"); return RT_EINVAL; }
    const size_t need = (size_t)xcorr_chunks(height) * (size_t)width * (size_t)channels;
    if (need > kNoallocMoments || xcorr_scratch_bytes(height, width, channels) > sizeof(g_xcorr_scratch)) {
        set_error("rt_xcorr_noalloc: %d x %d x %d images need %zu bytes of scratch; the fixed scratch holds %zu "
                  "bytes (min(ceil(height / 64), 64) * width * channels must be <= %zu)",
                  height, width, channels, need * sizeof(NoallocMoments), kNoallocMoments * sizeof(NoallocMoments),
                  kNoallocMoments);
        return RT_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_error("no CUDA device: %s", cudaGetErrorString(e)); return RT_ENODEV; }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) {
        set_error("device %d is sm_%d%d; this library is built for sm_103a only", dev, major, minor);
        return RT_ENODEV;
    }
    if (dev < 0 || dev >= kNoallocMaxDevices) { set_error("device index %d out of range", dev); return RT_EINVAL; }
    void* scratch = noalloc_scratch(dev, &e);
    if (!scratch) {
        set_error("rt_xcorr_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return RT_ECUDA;
    }
    Windows win;
    fov_windows(width, hfov_deg, fov_deg, n_fov, &win);
    // each kernel reads only scratch records that an earlier kernel of the
    // same call wrote, so nothing has to be cleared between calls
    e = launch_xcorr(d_f, d_g, height, width, channels, win, scratch, d_out, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error("rt_xcorr_noalloc: %s", cudaGetErrorString(e));
        return RT_ECUDA;
    }
    return RT_OK;
}
