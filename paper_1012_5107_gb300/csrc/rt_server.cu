// rt_server.cu -- a render server with continuous batching over a
// device-resident request ring.
//
// Requests (scene descriptors plus a caller-owned output image) are queued by
// rt_submit.  A worker thread admits them in arrival order while the sum of
// their ray-state footprints stays within the budget and publishes each
// admitted request into a ring of request slots in device memory: its scene
// table, output and scratch pointers, and a counter of the samples handed
// out.  A persistent launch of the wavefront loop takes samples from the
// published requests, so a launch that is running picks up requests
// published while it runs, as its lanes free up.  Of the oldest requests
// with samples left (a window of kRingWindow), each grab takes from the one
// with the fewest left (shortest remaining work first): a small request that
// arrives while a large one renders is taken up at once and finishes first.
// A launch ends when it finds no sample left; the worker launches again when
// samples are published and fewer than max_inflight launches are running (a
// second launch takes over the SMs as the blocks of the first one end).  The last pixel of a request to finish
// writes the request's completion record into host-mapped memory, which the
// worker polls.
//
// Consistency of the ring.  The worker copies a slot, then the request count,
// in that order on one copy stream; a lane that reads the request count
// (acquire) finds every slot below it.  A slot is reused only after its
// request completed; a grab that raced with a reuse is clipped to the new
// request's samples.  This file is compiled with global loads cached in L2
// only, and the background texels are loaded from L2 as well, so that no SM
// holds a stale copy of a reused slot or of memory that a later request's
// texture was copied into.
//
// Scratch comes from two device arenas allocated with the server: the pixel
// counters from one kept at zero (each pixel's last sample clears its
// counter), the per-sample colours and textures from the other.  Nothing is
// allocated or cleared per request, so the copy stream carries copies only:
// a memset is a kernel, which would wait for the running launch to end.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#define RT_TEX_LOAD __ldcg
#include "rt_wave.cuh"

namespace grt {

constexpr int kRingSlots = 1024;          // requests a ring holds in flight
constexpr int kRingGrabTries = 4096;      // scans of one grab before it gives up
constexpr int kRingWindow = 64;           // oldest requests with samples left that a grab chooses from
constexpr int kRingLocalBits = 40;        // a grabbed sample: slot << 40 | its index in the request
constexpr int kRingKinds = 6;             // precision x integrator (RK4, DP45, RK4T)

// One published request (device memory).
struct RingSlot {
    DevScene sc;                 // its scene table (nwork = pixels)
    float* out;                  // caller's image
    float* samp;                 // the pixels' colour blocks (col_block_bytes each; spp > 1)
    int* pcnt;                   // one counter per pixel (spp > 1), zero at publication and after
    long long nsamples;
    long long npix;
    unsigned long long grabbed;  // samples handed out (zero at publication)
    unsigned long long pix_done; // pixels finished (zero at publication)
    unsigned long long seq;      // its request number k in the ring (slot k % kRingSlots)
};

struct RingCtl {
    unsigned long long nreq;          // requests published (host)
    unsigned long long first_active;  // no request below this one has samples left (device)
    unsigned long long grabbed;       // samples handed out over all requests (device)
    unsigned long long pad;
};

// Completion records (host-mapped memory): seq[k % kRingSlots] = k + 1 once
// request k is finished.
struct RingDone {
    unsigned long long seq[kRingSlots];
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p)
{
    return *(const volatile unsigned long long*)p;
}

// The ring as a work source of the wavefront loop (rt_wave.cuh).
struct RingScenes {
    static constexpr bool kParamScene = false;
    RingSlot* slots;
    RingCtl* ctl;
    RingDone* done;
    void* branches;               // no scene options: no branch queues

    __device__ __forceinline__ const DevScene& scene(int s) const { return slots[s].sc; }
    // Warp-aggregated grab: the calling lanes look at the oldest kRingWindow
    // published requests from first_active on (each lane at every n-th of
    // them, n the number of calling lanes, then two warp reductions), and the
    // leader takes up to one sample per calling lane from the one with the
    // fewest samples left, by an atomic add on its counter; -1 for every lane
    // when none is left (or the attempts run out).  The result is
    // slot << 40 | sample index.  Remaining counts compare up to 2^26 - 1
    // (larger ones as equal, the older first).
    __device__ __forceinline__ int64_t grab(unsigned long long*, unsigned lane) const
    {
        const unsigned m = __activemask();
        const int leader = __ffs(m) - 1;
        const unsigned rank = __popc(m & ((1u << lane) - 1u));
        const unsigned cnt = __popc(m);
        constexpr long long kRemCap = (1ll << 26) - 1;
        long long base = -1;
        unsigned n = 0;
        for (int it = 0; it < kRingGrabTries; ++it) {
            long long nreq = 0, lo = 0;
            if ((int)lane == leader) {
                nreq = (long long)ld_acquire_u64(&ctl->nreq);
                lo = (long long)ld_volatile_u64(&ctl->first_active);
                if (lo < nreq - kRingSlots) lo = nreq - kRingSlots;
                if (lo < 0) lo = 0;
            }
            nreq = __shfl_sync(m, nreq, leader);
            lo = __shfl_sync(m, lo, leader);
            const long long wend = (nreq - lo < kRingWindow) ? nreq - lo : kRingWindow;
            unsigned key = 0xffffffffu, fq = kRingWindow;          // (remaining << 6 | q), first q with samples left
            for (long long q = rank; q < wend; q += cnt) {
                const int s = (int)((lo + q) % kRingSlots);
                const long long rem = slots[s].nsamples - (long long)ld_volatile_u64(&slots[s].grabbed);
                if (rem > 0) {                                       // <= 0 once the counter ran past
                    if ((unsigned)q < fq) fq = (unsigned)q;
                    const unsigned kk = ((unsigned)(rem < kRemCap ? rem : kRemCap) << 6) | (unsigned)q;
                    if (kk < key) key = kk;
                }
            }
            key = __reduce_min_sync(m, key);
            fq = __reduce_min_sync(m, fq);
            int again = 0;
            if ((int)lane == leader) {
                // requests before the first one with samples left are done with
                const long long adv = (fq < (unsigned)kRingWindow) ? lo + fq
                                                                    : (lo + kRingWindow < nreq ? lo + kRingWindow : nreq);
                if (adv > lo) atomicMax(&ctl->first_active, (unsigned long long)adv);
                if (key == 0xffffffffu) {
                    again = (lo + kRingWindow < nreq) ? 1 : 0;      // look further on, or none left
                } else {
                    // an atomic add always succeeds: the counter may run past the
                    // request's samples, and what lies past them is not taken
                    // (after a reuse of the slot: the new request's samples)
                    const int s = (int)((lo + (long long)(key & 63u)) % kRingSlots);
                    const unsigned long long want = cnt;
                    const unsigned long long c = atomicAdd(&slots[s].grabbed, want);
                    const long long have = slots[s].nsamples - (long long)c;
                    if (have <= 0) {
                        again = 1;
                    } else {
                        const unsigned long long t = (unsigned long long)have < want ? (unsigned long long)have : want;
                        atomicAdd(&ctl->grabbed, t);
                        base = ((long long)s << kRingLocalBits) | (long long)c;
                        n = (unsigned)t;
                    }
                }
            }
            again = __shfl_sync(m, again, leader);
            base = __shfl_sync(m, base, leader);
            if (base >= 0 || !again) break;
        }
        n = __shfl_sync(m, n, leader);
        return (base >= 0 && rank < n) ? (int64_t)(base + rank) : -1;
    }
    __device__ __forceinline__ void map_sample(int64_t ws, int& s, int64_t& pix, int64_t& out, int& sample) const
    {
        s = (int)(ws >> kRingLocalBits);
        const int64_t l = ws & ((1ll << kRingLocalBits) - 1);
        const int spp = slots[s].sc.spp;
        const int64_t w = l / spp;
        sample = (int)(l - w * spp);
        out = pix = w;
    }
    __device__ __forceinline__ float* sample_col(int s, int64_t out, int sample) const
    {
        return slots[s].samp + (col_block_bytes(slots[s].sc.spp) >> 2) * out + 4 * sample;
    }
    __device__ __forceinline__ int* pixel_count(int s, int64_t out) const { return slots[s].pcnt + out; }
    // The pixel's last sample sets its counter back to zero: the counters
    // come from an arena kept at zero, so a request needs no clearing before
    // it is published (a clearing kernel would wait for the running launch).
    __device__ __forceinline__ void release_count(int s, int64_t out) const { slots[s].pcnt[out] = 0; }
    // After a pixel is written: count it; the request's last pixel writes the
    // completion record to host-mapped memory.
    __device__ __forceinline__ void pixel_done(int s) const
    {
        __threadfence();                                  // this pixel's colours before the count
        const unsigned long long d = atomicAdd(&slots[s].pix_done, 1ull) + 1ull;
        if (d == (unsigned long long)slots[s].npix) {
            __threadfence_system();                       // every pixel of the request before the record
            *(volatile unsigned long long*)&done->seq[s] = slots[s].seq + 1ull;
        }
    }
    __device__ __forceinline__ float* rgb_of(int s) const { return slots[s].out; }
    __device__ __forceinline__ uint8_t* rgb8_of(int) const { return nullptr; }
    __device__ __forceinline__ rt_ray_record* rec_of(int) const { return nullptr; }
};

template <class R, int INTEG>
__global__ void __launch_bounds__(WaveShape<R, INTEG>::kBlock, WaveShape<R, INTEG>::kMinBlocks) wave_ring_kernel(
    RingSlot* slots, RingCtl* ctl, RingDone* done, unsigned long long* counters, int min_active)
{
    const RingScenes src{slots, ctl, done, nullptr};
    wave_loop<R, INTEG, false>(src, counters, min_active, WaveWait{kWaveSpin, 0});
}

template <class R, int INTEG>
static cudaError_t ring_launch_t(int grid, RingSlot* slots, RingCtl* ctl, RingDone* done,
                                 unsigned long long* counters, cudaStream_t st)
{
    static std::atomic<unsigned long long> set{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(set.load() & bit)) {
        e = cudaFuncSetAttribute(wave_ring_kernel<R, INTEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)wave_smem_bytes<R, INTEG>());
        if (e != cudaSuccess) return e;
        set.fetch_or(bit);
    }
    wave_ring_kernel<R, INTEG><<<grid, WaveShape<R, INTEG>::kBlock, wave_smem_bytes<R, INTEG>(), st>>>(slots, ctl, done, counters,
                                                                               default_min_active(sizeof(R) == 4 ? RT_FP32 : RT_FP64, INTEG));
    return cudaGetLastError();
}

template <class R, int INTEG>
static cudaError_t ring_occupancy_t(int* bps)
{
    cudaError_t e = cudaFuncSetAttribute(wave_ring_kernel<R, INTEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)wave_smem_bytes<R, INTEG>());
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, wave_ring_kernel<R, INTEG>,
                                                         WaveShape<R, INTEG>::kBlock, wave_smem_bytes<R, INTEG>());
}

static int kind_of(int precision, int integrator) { return precision * 3 + integrator; }

static cudaError_t ring_launch(int kind, int grid, RingSlot* slots, RingCtl* ctl, RingDone* done,
                               unsigned long long* counters, cudaStream_t st)
{
    switch (kind) {
        case 0: return ring_launch_t<float, RT_RK4>(grid, slots, ctl, done, counters, st);
        case 1: return ring_launch_t<float, RT_DP45>(grid, slots, ctl, done, counters, st);
        case 2: return ring_launch_t<float, RT_RK4T>(grid, slots, ctl, done, counters, st);
        case 3: return ring_launch_t<double, RT_RK4>(grid, slots, ctl, done, counters, st);
        case 4: return ring_launch_t<double, RT_DP45>(grid, slots, ctl, done, counters, st);
        default: return ring_launch_t<double, RT_RK4T>(grid, slots, ctl, done, counters, st);
    }
}

static cudaError_t ring_occupancy(int kind, int* bps)
{
    switch (kind) {
        case 0: return ring_occupancy_t<float, RT_RK4>(bps);
        case 1: return ring_occupancy_t<float, RT_DP45>(bps);
        case 2: return ring_occupancy_t<float, RT_RK4T>(bps);
        case 3: return ring_occupancy_t<double, RT_RK4>(bps);
        case 4: return ring_occupancy_t<double, RT_DP45>(bps);
        default: return ring_occupancy_t<double, RT_RK4T>(bps);
    }
}

}  // namespace grt

using namespace grt;

namespace {

using Clock = std::chrono::steady_clock;

// Bytes of ray state a request holds while it is in flight: every sample of
// the image carries its state through the ring (position, direction,
// cloak state, accumulators), 64 bytes per sample, plus its colour slot and
// its pixel's sample counter in the scratch and its output image.
constexpr size_t kStateBytesPerSample = 64;
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over the device arena (host bookkeeping only).
struct Arena {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;          // offset -> bytes
    void init(char* b, size_t n)
    {
        base = b;
        size = n;
        free_.clear();
        if (n) free_[0] = n;
    }
    bool alloc(size_t bytes, size_t* off)
    {
        bytes = align_up(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = align_up(bytes ? bytes : 1);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
};

struct Request {
    uint64_t ticket;
    rt_scene_desc desc;
    std::vector<float> tex;            // copy of the host texture, if any
    float* d_out;
    size_t bytes;                      // footprint in the budget
    size_t arena_off, arena_bytes;     // colours and texture in the data arena
    size_t cnt_off, cnt_bytes;         // pixel counters in the counter arena
    int kind;
    uint64_t seq;                      // request number in its ring
    long long nsamples;
    Clock::time_point submitted, published, finished;
    int status;                        // RT_PENDING until done
    uint64_t rays;
    int passed = 0;                    // later requests admitted before it (kMaxPassed)
};

// Admission takes queued requests in arrival order, but a request that fits
// may pass queued ones that do not fit yet: a small request then need not
// wait behind a large one for the budget a third holds.  No request is passed
// more than kMaxPassed times; after that, admission waits for it.  The
// worker looks kAdmitLookahead requests deep.
constexpr int kMaxPassed = 32;
constexpr size_t kAdmitLookahead = 64;

struct Ring {
    int kind = -1;
    bool ready = false;
    RingSlot* d_slots = nullptr;
    RingCtl* d_ctl = nullptr;
    RingDone* h_done = nullptr;        // host-mapped
    RingDone* d_done = nullptr;
    RingSlot* h_slot_stage = nullptr;  // pinned, one per slot
    unsigned long long* h_ctl_stage = nullptr;   // pinned, two per slot (the request count)
    unsigned long long* d_stats = nullptr;       // kCounters per launch stream
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t published_ev = nullptr;
    std::vector<cudaStream_t> kstreams;
    std::vector<cudaEvent_t> kdone;
    std::vector<bool> krunning;
    std::vector<uint64_t> slot_ticket;           // ticket in each slot (0: free)
    uint64_t nreq = 0;
    unsigned long long published = 0;
    int grid = 0;
    bool timed_out = false;                      // a launch gave up bounded waits
};

}  // namespace

struct rt_server {
    int nsm;
    int device;
    size_t budget, in_use;
    int max_inflight;
    size_t max_queue;
    char* d_arena;
    Arena arena;                       // colours and textures
    Arena counters;                    // pixel counters (kept at zero)
    Ring rings[kRingKinds];
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;                    // submitted, not admitted
    std::map<uint64_t, Request> req;
    uint64_t next_ticket;
    uint64_t completed, failed, in_flight;
    bool stop;
    std::thread worker;
};

static size_t request_bytes(const rt_scene_desc* d)
{
    const size_t wout = d->centre_line ? 1 : (size_t)d->width;
    const size_t pixels = (size_t)d->height * wout;
    return pixels * (size_t)d->spp * (kStateBytesPerSample + kScratchBytesPerSample) +
           pixels * (3 * sizeof(float) + kScratchBytesPerPixel);
}

static void ring_free(Ring& g)
{
    if (g.copy_stream) cudaStreamSynchronize(g.copy_stream);
    for (size_t i = 0; i < g.kstreams.size(); ++i) {
        cudaStreamSynchronize(g.kstreams[i]);
        cudaStreamDestroy(g.kstreams[i]);
        cudaEventDestroy(g.kdone[i]);
    }
    g.kstreams.clear();
    g.kdone.clear();
    g.krunning.clear();
    if (g.published_ev) cudaEventDestroy(g.published_ev);
    if (g.copy_stream) cudaStreamDestroy(g.copy_stream);
    if (g.d_slots) cudaFree(g.d_slots);
    if (g.d_ctl) cudaFree(g.d_ctl);
    if (g.d_stats) cudaFree(g.d_stats);
    if (g.h_done) cudaFreeHost(g.h_done);
    if (g.h_slot_stage) cudaFreeHost(g.h_slot_stage);
    if (g.h_ctl_stage) cudaFreeHost(g.h_ctl_stage);
    g = Ring();
}

// Device ring, streams and staging of one kind (worker thread, lock held).
static cudaError_t ring_init(rt_server* S, Ring& g, int kind)
{
    g.kind = kind;
    int bps = 0;
    cudaError_t e = ring_occupancy(kind, &bps);
    g.grid = (bps > 0 ? bps : 1) * S->nsm;
    if (e == cudaSuccess) e = cudaMalloc(&g.d_slots, sizeof(RingSlot) * kRingSlots);
    if (e == cudaSuccess) e = cudaMalloc(&g.d_ctl, sizeof(RingCtl));
    if (e == cudaSuccess) e = cudaMemset(g.d_ctl, 0, sizeof(RingCtl));
    if (e == cudaSuccess) e = cudaMalloc(&g.d_stats, sizeof(unsigned long long) * kCounters * S->max_inflight);
    if (e == cudaSuccess) e = cudaHostAlloc(&g.h_done, sizeof(RingDone), cudaHostAllocMapped);
    if (e == cudaSuccess) memset(g.h_done, 0, sizeof(RingDone));
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&g.d_done, g.h_done, 0);
    if (e == cudaSuccess) e = cudaHostAlloc(&g.h_slot_stage, sizeof(RingSlot) * kRingSlots, cudaHostAllocDefault);
    if (e == cudaSuccess)
        e = cudaHostAlloc(&g.h_ctl_stage, sizeof(unsigned long long) * 2 * kRingSlots, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.published_ev, cudaEventDisableTiming);
    for (int i = 0; i < S->max_inflight && e == cudaSuccess; ++i) {
        cudaStream_t st;
        cudaEvent_t ev;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) break;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) { cudaStreamDestroy(st); break; }
        g.kstreams.push_back(st);
        g.kdone.push_back(ev);
        g.krunning.push_back(false);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    g.slot_ticket.assign(kRingSlots, 0);
    g.ready = (e == cudaSuccess);
    return e;
}

static void finish_request(rt_server* S, Request& r, int status, Clock::time_point now)
{
    r.status = status;
    r.finished = now;
    const size_t wout = r.desc.centre_line ? 1 : (size_t)r.desc.width;
    r.rays = (uint64_t)r.desc.height * wout * r.desc.spp;
    r.tex.clear();
    S->in_use -= r.bytes;
    if (r.arena_bytes) S->arena.release(r.arena_off, r.arena_bytes);
    r.arena_bytes = 0;
    if (r.cnt_bytes) {
        // a request that did not finish leaves counters behind: clear them
        // (a failure path only; it waits for the device)
        if (status != RT_OK) cudaMemset(S->counters.base + r.cnt_off, 0, r.cnt_bytes);
        S->counters.release(r.cnt_off, r.cnt_bytes);
    }
    r.cnt_bytes = 0;
    if (status == RT_OK) S->completed++;
    else S->failed++;
}

// Publish an admitted request into its ring (worker thread, lock held):
// scratch and texture from the arena, the slot copied to the device.
static cudaError_t publish(rt_server* S, Ring& g, Request& r)
{
    const uint64_t k = g.nreq;
    const int s = (int)(k % kRingSlots);
    RingSlot& h = g.h_slot_stage[s];
    memset(&h, 0, sizeof h);
    build_scene_table(&r.desc, &h.sc);
    const long long npix = (long long)h.sc.nwork;
    const long long ns = npix * h.sc.spp;
    char* base = S->arena.base + r.arena_off;
    size_t at = 0;
    cudaError_t e = cudaSuccess;
    if (h.sc.spp > 1) {
        h.samp = (float*)(base + at);
        at += align_up((size_t)col_block_bytes(h.sc.spp) * (size_t)npix);
        h.pcnt = (int*)(S->counters.base + r.cnt_off);
    }
    if (e == cudaSuccess && !r.tex.empty()) {
        float* t = (float*)(base + at);
        e = cudaMemcpyAsync(t, r.tex.data(), r.tex.size() * sizeof(float), cudaMemcpyHostToDevice, g.copy_stream);
        h.sc.tex = t;
    }
    h.out = r.d_out;
    h.nsamples = ns;
    h.npix = npix;
    h.grabbed = 0;
    h.pix_done = 0;
    h.seq = k;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g.d_slots + s, &h, sizeof h, cudaMemcpyHostToDevice, g.copy_stream);
    if (e != cudaSuccess) return e;
    g.h_done->seq[s] = 0;
    g.slot_ticket[s] = r.ticket;
    r.seq = k;
    r.nsamples = ns;
    g.nreq = k + 1;
    g.published += (unsigned long long)ns;
    // the slot first, then the request count (in that order on the copy
    // stream): a lane that sees the count finds the slot
    unsigned long long* cs = g.h_ctl_stage + 2 * s;
    cs[0] = g.nreq;
    return cudaMemcpyAsync(&g.d_ctl->nreq, cs, sizeof(unsigned long long), cudaMemcpyHostToDevice, g.copy_stream);
}

// Launch the ring's kernel on a free stream once the publications are on the
// device (worker thread, lock held).
static cudaError_t launch(rt_server* S, Ring& g)
{
    int i = -1;
    for (size_t q = 0; q < g.krunning.size(); ++q)
        if (!g.krunning[q]) { i = (int)q; break; }
    if (i < 0) return cudaSuccess;
    cudaStream_t st = g.kstreams[i];
    unsigned long long* stats = g.d_stats + (size_t)kCounters * i;
    cudaError_t e = cudaEventRecord(g.published_ev, g.copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, g.published_ev, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(stats, 0, sizeof(unsigned long long) * kCounters, st);
    if (e == cudaSuccess) e = ring_launch(g.kind, g.grid, g.d_slots, g.d_ctl, g.d_done, stats, st);
    if (e == cudaSuccess) e = cudaEventRecord(g.kdone[i], st);
    if (e == cudaSuccess) g.krunning[i] = true;
    return e;
}

// Completions, ended launches and lost requests of one ring (worker thread, lock held).
static void ring_progress(rt_server* S, Ring& g)
{
    const Clock::time_point now = Clock::now();
    for (int s = 0; s < kRingSlots; ++s) {
        const uint64_t t = g.slot_ticket[s];
        if (!t) continue;
        Request& r = S->req[t];
        if (*(volatile unsigned long long*)&g.h_done->seq[s] == r.seq + 1) {
            finish_request(S, r, RT_OK, now);
            g.slot_ticket[s] = 0;
            S->in_flight--;
            S->cv_done.notify_all();
        }
    }
    bool any_running = false;
    for (size_t i = 0; i < g.krunning.size(); ++i) {
        if (!g.krunning[i]) continue;
        const cudaError_t q = cudaEventQuery(g.kdone[i]);
        if (q == cudaErrorNotReady) { any_running = true; continue; }
        g.krunning[i] = false;
        unsigned long long timeouts = 0;
        if (q != cudaSuccess ||
            cudaMemcpy(&timeouts, g.d_stats + (size_t)kCounters * i + (kCounters - 1), sizeof timeouts,
                       cudaMemcpyDeviceToHost) != cudaSuccess)
            g.timed_out = true;
        else if (timeouts)
            g.timed_out = true;
    }
    bool pending = false;
    for (int s = 0; s < kRingSlots && !pending; ++s) pending = g.slot_ticket[s] != 0;
    if (!pending || any_running) return;
    // no launch running: samples left over need a launch; requests whose
    // samples were all handed out but never finished are lost
    unsigned long long grabbed = 0;
    if (!g.timed_out &&
        cudaMemcpy(&grabbed, &g.d_ctl->grabbed, sizeof grabbed, cudaMemcpyDeviceToHost) != cudaSuccess)
        g.timed_out = true;
    if (!g.timed_out && grabbed < g.published) {
        if (launch(S, g) != cudaSuccess) g.timed_out = true;
        if (!g.timed_out) return;
    }
    // look again for records written just before the launches ended
    for (int s = 0; s < kRingSlots; ++s) {
        const uint64_t t = g.slot_ticket[s];
        if (!t) continue;
        Request& r = S->req[t];
        const bool done = *(volatile unsigned long long*)&g.h_done->seq[s] == r.seq + 1;
        finish_request(S, r, done ? RT_OK : (g.timed_out ? RT_ETIMEDOUT : RT_ECUDA), Clock::now());
        g.slot_ticket[s] = 0;
        S->in_flight--;
    }
    g.timed_out = false;
    S->cv_done.notify_all();
}

static bool any_launch_running(rt_server* S)
{
    for (Ring& g : S->rings)
        for (bool b : g.krunning)
            if (b) return true;
    return false;
}

static void worker_main(rt_server* S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    for (;;) {
        for (Ring& g : S->rings)
            if (g.ready) ring_progress(S, g);
        if (S->stop && S->in_flight == 0 && !any_launch_running(S)) break;
        // admit in arrival order while the budget, the ring and the arena
        // allow, letting a request that fits pass ones that do not (kMaxPassed)
        bool touched[kRingKinds] = {false, false, false, false, false, false};
        size_t qi = 0;
        while (!S->stop && qi < S->queue.size() && qi < kAdmitLookahead) {
            Request& r = S->req[S->queue[qi]];
            if (S->in_use + r.bytes > S->budget) {
                if (r.passed >= kMaxPassed) break;
                ++qi;
                continue;
            }
            Ring& g = S->rings[r.kind];
            if (!g.ready && ring_init(S, g, r.kind) != cudaSuccess) {
                ring_free(g);
                finish_request(S, r, RT_ECUDA, Clock::now());
                S->queue.erase(S->queue.begin() + (std::ptrdiff_t)qi);
                S->cv_done.notify_all();
                continue;
            }
            if (g.slot_ticket[g.nreq % kRingSlots] != 0) {               // its ring is full
                if (r.passed >= kMaxPassed) break;
                ++qi;
                continue;
            }
            const rt_scene_desc& d = r.desc;
            const size_t npix = (size_t)d.height * (d.centre_line ? 1 : (size_t)d.width);
            size_t need = 0, need_cnt = 0;
            if (d.spp > 1) {
                need += align_up((size_t)col_block_bytes(d.spp) * npix);
                need_cnt = align_up(kScratchBytesPerPixel * npix);
            }
            need += align_up(r.tex.size() * sizeof(float));
            size_t off = 0, coff = 0;
            bool ok = !need || S->arena.alloc(need, &off);
            if (ok && need_cnt && !S->counters.alloc(need_cnt, &coff)) {
                if (need) S->arena.release(off, need);
                ok = false;
            }
            if (!ok) {
                if (S->in_flight == 0) {                                  // can never fit
                    finish_request(S, r, RT_ENOMEM, Clock::now());
                    S->queue.erase(S->queue.begin() + (std::ptrdiff_t)qi);
                    S->cv_done.notify_all();
                    continue;
                }
                if (r.passed >= kMaxPassed) break;
                ++qi;
                continue;
            }
            r.arena_off = off;
            r.arena_bytes = need;
            r.cnt_off = coff;
            r.cnt_bytes = need_cnt;
            S->in_use += r.bytes;
            for (size_t j = 0; j < qi; ++j) S->req[S->queue[j]].passed++;
            S->queue.erase(S->queue.begin() + (std::ptrdiff_t)qi);
            S->in_flight++;
            if (publish(S, g, r) != cudaSuccess) {
                g.slot_ticket[g.nreq % kRingSlots] = 0;
                finish_request(S, r, RT_ECUDA, Clock::now());
                S->in_flight--;
                S->cv_done.notify_all();
                continue;
            }
            r.published = Clock::now();
            touched[r.kind] = true;
        }
        for (int q = 0; q < kRingKinds; ++q) {
            Ring& g = S->rings[q];
            if (!touched[q]) continue;
            // a running launch takes the new samples itself; another launch
            // starts if a stream is free, and takes over SMs as the running
            // launch's blocks end
            if (launch(S, g) != cudaSuccess) g.timed_out = true;
        }
        S->cv_work.wait_for(lock, std::chrono::microseconds(S->in_flight ? 100 : 2000));
    }
}

extern "C" {

int rt_request_bytes(const rt_scene_desc* desc, uint64_t* bytes)
{
    if (!desc || !bytes) { set_error("desc and bytes must not be NULL"); return RT_EINVAL; }
    const int rc = rt_validate_desc(desc);
    if (rc != RT_OK) return rc;
    *bytes = request_bytes(desc);
    return RT_OK;
}

int rt_server_create(size_t ray_state_budget_bytes, int32_t max_inflight, rt_server** out)
{
    if (!out) { set_error("out is NULL"); return RT_EINVAL; }
    *out = nullptr;
    set_error("%s", "");
    if (ray_state_budget_bytes == 0) { set_error("budget must be > 0"); return RT_EINVAL; }
    if (max_inflight < 1 || max_inflight > 16) { set_error("max_inflight must be 1..16"); return RT_EINVAL; }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_error("no CUDA device: %s", cudaGetErrorString(e)); return RT_ENODEV; }
    rt_server* S = new (std::nothrow) rt_server();
    if (!S) { set_error("host allocation failed"); return RT_ENOMEM; }
    S->device = dev;
    S->budget = ray_state_budget_bytes;
    S->in_use = 0;
    S->max_inflight = max_inflight;
    S->max_queue = 1 << 16;
    S->next_ticket = 1;
    S->completed = S->failed = S->in_flight = 0;
    S->stop = false;
    S->d_arena = nullptr;
    // the arena holds the scratch and textures of the requests in flight: at
    // most the budget (whose footprints count 76 bytes per sample against 12
    // of scratch) and at most half of the free device memory
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    size_t arena = std::min(ray_state_budget_bytes, fr / 2);
    arena = align_up(std::max(arena, (size_t)(1 << 20)));
    e = cudaMalloc(&S->d_arena, arena);
    if (e != cudaSuccess) {
        delete S;
        set_error("rt_server_create: arena of %zu bytes: %s", arena, cudaGetErrorString(e));
        return RT_ENOMEM;
    }
    // a seventh for the pixel counters (4 bytes a pixel against at least 24
    // of colours at two samples a pixel), the rest for colours and textures
    const size_t ncnt = align_up(arena / 7);
    e = cudaMemset(S->d_arena, 0, ncnt);
    if (e != cudaSuccess) {
        cudaFree(S->d_arena);
        delete S;
        set_error("rt_server_create: %s", cudaGetErrorString(e));
        return RT_ECUDA;
    }
    S->counters.init(S->d_arena, ncnt);
    S->arena.init(S->d_arena + ncnt, arena - ncnt);
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    S->nsm = nsm > 0 ? nsm : 1;
    S->worker = std::thread(worker_main, S);
    *out = S;
    return RT_OK;
}

void rt_server_destroy(rt_server* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        // requests never admitted fail; those in flight are finished
        for (uint64_t t : S->queue) {
            Request& r = S->req[t];
            r.status = RT_ETIMEDOUT;
            r.finished = Clock::now();
            S->failed++;
        }
        S->queue.clear();
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Ring& g : S->rings) ring_free(g);
    if (S->d_arena) cudaFree(S->d_arena);
    delete S;
}

int rt_submit(rt_server* S, const rt_scene_desc* desc, float* d_out, uint64_t* ticket)
{
    if (!S || !desc || !d_out || !ticket) { set_error("null argument"); return RT_EINVAL; }
    // validate on the caller's thread: a bad descriptor is reported at once
    rt_scene_desc d = *desc;
    const int vr = rt_validate_desc(&d);
    if (vr != RT_OK) return vr;
    if (d.mirror == RT_MIRROR_GAUSS) {
        set_error("scenes of the Gaussian bump are rendered alone (rt_render), not served");
        return RT_EINVAL;
    }
    if (d.flags != 0) {
        set_error("scenes with options (RT_FLAG_*) are rendered alone or in batches, not served");
        return RT_EINVAL;
    }
    Request r;
    r.desc = d;
    r.d_out = d_out;
    r.bytes = request_bytes(&d);
    r.arena_off = r.arena_bytes = 0;
    r.cnt_off = r.cnt_bytes = 0;
    r.kind = kind_of(d.precision, d.integrator);
    r.seq = 0;
    r.nsamples = 0;
    r.status = RT_PENDING;
    r.rays = 0;
    if (d.background == RT_BG_TEXTURE && d.tex) {
        r.tex.assign(d.tex, d.tex + (size_t)d.tex_size * d.tex_size);
    }
    r.desc.tex = nullptr;
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stop) { set_error("server is shutting down"); return RT_EBUSY; }
    if (r.bytes > S->budget) {
        set_error("request needs %zu bytes of ray state; the budget is %zu", r.bytes, S->budget);
        return RT_EBUSY;
    }
    if (S->queue.size() >= S->max_queue) { set_error("submission queue full"); return RT_EBUSY; }
    r.ticket = S->next_ticket++;
    r.submitted = Clock::now();
    *ticket = r.ticket;
    S->queue.push_back(r.ticket);
    S->req.emplace(r.ticket, std::move(r));
    S->cv_work.notify_all();
    return RT_OK;
}

int rt_poll(rt_server* S, uint64_t ticket, int32_t timeout_us, rt_result* out)
{
    if (!S || !out) { set_error("null argument"); return RT_EINVAL; }
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->req.find(ticket);
    if (it == S->req.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return RT_EINVAL; }
    if (it->second.status == RT_PENDING && timeout_us > 0) {
        S->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), [&] {
            auto j = S->req.find(ticket);
            return j == S->req.end() || j->second.status != RT_PENDING;
        });
        it = S->req.find(ticket);
        if (it == S->req.end()) { set_error("ticket %llu was reported already", (unsigned long long)ticket); return RT_EINVAL; }
    }
    Request& r = it->second;
    if (r.status == RT_PENDING) return timeout_us > 0 ? RT_ETIMEDOUT : RT_PENDING;
    out->status = r.status;
    out->latency_ms = (float)std::chrono::duration<double, std::milli>(r.finished - r.submitted).count();
    out->queue_ms = (r.published.time_since_epoch().count() > 0)
                        ? (float)std::chrono::duration<double, std::milli>(r.published - r.submitted).count()
                        : out->latency_ms;
    out->rays = r.rays;
    const int st = r.status;
    S->req.erase(ticket);          // a finished ticket is reported once
    return st == RT_OK ? RT_OK : st;
}

int rt_server_stats(rt_server* S, rt_server_info* out)
{
    if (!S || !out) { set_error("null argument"); return RT_EINVAL; }
    std::lock_guard<std::mutex> lock(S->mu);
    out->queued = S->queue.size();
    out->in_flight = S->in_flight;
    out->completed = S->completed;
    out->failed = S->failed;
    out->bytes_in_use = S->in_use;
    out->budget = S->budget;
    return RT_OK;
}

}  // extern "C"
