// rt_server.cu -- a render server with continuous batching.
//
// Requests (scene descriptors plus a caller-owned output image) are queued by
// rt_submit.  A worker thread admits them in arrival order while the sum of
// their ray-state footprints stays within the budget, groups the newly
// admitted requests into a batch (one persistent launch for all of them) and
// launches it on a free stream, so requests that arrive while other batches
// run are admitted as budget and streams free up and their work overlaps on
// the device.  Completion is detected with non-blocking event queries; every
// wait of the host is bounded.
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

#include "rt_internal.h"

using namespace grt;

namespace {

using Clock = std::chrono::steady_clock;

// Bytes of ray state a request holds while it is in flight: every sample of
// the image carries its state through the batch (position, direction,
// cloak state, accumulators), 64 bytes per sample, plus its colour slot and
// its pixel's sample counter in the launch's scratch and its output image.
constexpr size_t kStateBytesPerSample = 64;

struct Request {
    uint64_t ticket;
    rt_scene_desc desc;
    std::vector<float> tex;            // copy of the host texture, if any
    float* d_out;
    size_t bytes;
    Clock::time_point submitted, launched, finished;
    int status;                        // RT_PENDING until done
    uint64_t rays;
};

struct Flight {
    std::vector<uint64_t> tickets;
    std::vector<void*> allocs;          // stream-ordered device allocations of the flight
    unsigned long long* d_counters;
    int stream;
    cudaEvent_t done;
};

}  // namespace

struct rt_server {
    int precision_of(uint64_t t) { return req[t].desc.precision; }
    int integrator_of(uint64_t t) { return req[t].desc.integrator; }
    int nsm;
    int device;
    size_t budget, in_use;
    int max_inflight;
    size_t max_queue;
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;                    // submitted, not admitted
    std::map<uint64_t, Request> req;
    std::vector<Flight> flights;
    uint64_t next_ticket;
    uint64_t completed, failed;
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

// Launch one batch of admitted requests on stream `si` (worker thread, lock
// held).  Every device allocation of the flight is stream-ordered on its
// stream, so starting and retiring flights never synchronises the device.
static void launch_flight(rt_server* S, const std::vector<uint64_t>& admitted, int si)
{
    cudaStream_t st = S->streams[si];
    // the flight's work list in the batch order: cloaked scenes first, then
    // bare gratings, then flat mirrors, fewer samples first within a kind
    std::vector<uint64_t> tickets = admitted;
    auto samples = [&](uint64_t t) {
        const rt_scene_desc& d = S->req[t].desc;
        return (int64_t)d.height * (d.centre_line ? 1 : d.width) * d.spp;
    };
    std::stable_sort(tickets.begin(), tickets.end(), [&](uint64_t a, uint64_t c) {
        const rt_scene_desc &x = S->req[a].desc, &y = S->req[c].desc;
        if (x.cloak != y.cloak) return x.cloak > y.cloak;
        if (x.mirror != y.mirror) return x.mirror > y.mirror;
        return samples(a) < samples(c);
    });
    Flight f;
    f.stream = si;
    f.done = nullptr;
    f.d_counters = nullptr;
    const int n = (int)tickets.size();
    std::vector<DevScene> dev(n);
    std::vector<int64_t> off(n + 1, 0), soff(n + 1, 0);
    std::vector<float*> outs(n);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMallocAsync(p, bytes, st);
        if (e == cudaSuccess) f.allocs.push_back(*p);
    };
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        Request& r = S->req[tickets[i]];
        build_scene_table(&r.desc, &dev[i]);
        if (!r.tex.empty()) {
            void* t = nullptr;
            alloc(&t, r.tex.size() * sizeof(float));
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(t, r.tex.data(), r.tex.size() * sizeof(float), cudaMemcpyHostToDevice, st);
            dev[i].tex = (const float*)t;
        }
        off[i + 1] = off[i] + dev[i].nwork;
        soff[i + 1] = soff[i] + dev[i].nwork * dev[i].spp;
        outs[i] = r.d_out;
    }
    void *d_scenes = nullptr, *d_off = nullptr, *d_soff = nullptr, *d_rgbs = nullptr, *d_cnt = nullptr;
    void *d_samp = nullptr, *d_pcnt = nullptr, *d_br = nullptr;
    bool fresnel = false, opt = false;
    for (int i = 0; i < n; ++i) {
        fresnel = fresnel || (dev[i].flags & RT_FLAG_FRESNEL);
        opt = opt || dev[i].flags != 0;
    }
    // one persistent block per resident slot of the build the flight takes
    int bps = 0;
    if (e == cudaSuccess) e = batch_occupancy(S->precision_of(tickets[0]), S->integrator_of(tickets[0]), opt, &bps);
    const int grid = (bps > 0 ? bps : 1) * S->nsm;
    if (fresnel) alloc(&d_br, branch_queue_bytes(S->precision_of(tickets[0]), grid));
    alloc(&d_scenes, sizeof(DevScene) * n);
    alloc(&d_off, sizeof(int64_t) * (n + 1));
    alloc(&d_soff, sizeof(int64_t) * (n + 1));
    alloc(&d_rgbs, sizeof(float*) * n);
    alloc(&d_cnt, sizeof(unsigned long long) * kCounters);
    alloc(&d_samp, kScratchBytesPerSample * (size_t)soff[n]);
    alloc(&d_pcnt, kScratchBytesPerPixel * (size_t)off[n]);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_scenes, dev.data(), sizeof(DevScene) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_soff, soff.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_rgbs, outs.data(), sizeof(float*) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * kCounters, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_pcnt, 0, kScratchBytesPerPixel * (size_t)off[n], st);
    if (e == cudaSuccess) {
        const BatchLaunch L = {(const DevScene*)d_scenes, (const int64_t*)d_off, (const int64_t*)d_soff,
                               (float* const*)d_rgbs, n, off[n], soff[n], {(float*)d_samp, (int*)d_pcnt, d_br},
                               (unsigned long long*)d_cnt, kMinActive, grid, opt};
        e = launch_batch(S->precision_of(tickets[0]), S->integrator_of(tickets[0]), L, st);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(f.done, st);
    // pageable-memory copies are staged before cudaMemcpyAsync returns, so the
    // host tables can go now
    const Clock::time_point now = Clock::now();
    if (e != cudaSuccess) {
        for (void* p : f.allocs) cudaFreeAsync(p, st);
        if (f.done) cudaEventDestroy(f.done);
        for (uint64_t t : tickets) {
            Request& r = S->req[t];
            r.status = RT_ECUDA;
            r.finished = now;
            S->in_use -= r.bytes;
            S->failed++;
        }
        S->cv_done.notify_all();
        return;
    }
    f.d_counters = (unsigned long long*)d_cnt;
    for (uint64_t t : tickets) S->req[t].launched = now;
    f.tickets = tickets;
    S->stream_busy[si] = true;
    S->flights.push_back(std::move(f));
}

// Retire finished batches (worker thread, lock held).
static void retire(rt_server* S)
{
    for (size_t i = 0; i < S->flights.size();) {
        Flight& f = S->flights[i];
        const cudaError_t q = cudaEventQuery(f.done);
        if (q == cudaErrorNotReady) { ++i; continue; }
        int status = (q == cudaSuccess) ? RT_OK : RT_ECUDA;
        if (status == RT_OK) {
            // a bounded wait of the work queues that gave up leaves images incomplete
            unsigned long long timeouts = 0;
            cudaStream_t st = S->streams[f.stream];
            if (cudaMemcpyAsync(&timeouts, f.d_counters + (kCounters - 1), sizeof timeouts, cudaMemcpyDeviceToHost,
                                st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                status = RT_ECUDA;
            else if (timeouts)
                status = RT_ETIMEDOUT;
        }
        const Clock::time_point now = Clock::now();
        for (size_t k = 0; k < f.tickets.size(); ++k) {
            Request& r = S->req[f.tickets[k]];
            r.status = status;
            r.finished = now;
            const size_t wout = r.desc.centre_line ? 1 : (size_t)r.desc.width;
            r.rays = (uint64_t)r.desc.height * wout * r.desc.spp;
            r.tex.clear();
            S->in_use -= r.bytes;
            if (status == RT_OK) S->completed++;
            else S->failed++;
        }
        cudaStream_t st = S->streams[f.stream];
        for (void* p : f.allocs) cudaFreeAsync(p, st);
        cudaEventDestroy(f.done);
        S->stream_busy[f.stream] = false;
        S->flights.erase(S->flights.begin() + i);
        S->cv_done.notify_all();
    }
}

static void worker_main(rt_server* S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    for (;;) {
        retire(S);
        if (S->stop && S->flights.empty()) break;
        // admit in arrival order while the budget allows
        std::vector<uint64_t> admit;
        if (!S->stop) {
            // a batch shares precision and integrator: take the queue head's
            // kind, in arrival order, up to the first request of another kind
            int kind = -1;
            while (!S->queue.empty() && admit.size() < 256) {
                Request& r = S->req[S->queue.front()];
                const int k = r.desc.precision * 4 + r.desc.integrator;
                if (kind >= 0 && k != kind) break;
                if (S->in_use + r.bytes > S->budget) break;
                kind = k;
                S->in_use += r.bytes;
                admit.push_back(r.ticket);
                S->queue.pop_front();
            }
        }
        if (!admit.empty()) {
            int si = -1;
            for (int k = 0; k < S->max_inflight; ++k)
                if (!S->stream_busy[k]) { si = k; break; }
            if (si >= 0) {
                launch_flight(S, admit, si);
                continue;
            }
            // no free stream: return the admissions and wait for a batch to finish
            for (auto it = admit.rbegin(); it != admit.rend(); ++it) {
                S->in_use -= S->req[*it].bytes;
                S->queue.push_front(*it);
            }
        }
        S->cv_work.wait_for(lock, std::chrono::microseconds(S->flights.empty() ? 2000 : 200));
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
    S->completed = S->failed = 0;
    S->stop = false;
    for (int k = 0; k < max_inflight; ++k) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
            delete S;
            set_error("stream creation failed");
            return RT_ECUDA;
        }
        S->streams.push_back(st);
        S->stream_busy.push_back(false);
    }
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
        // requests never admitted fail
        for (uint64_t t : S->queue) {
            Request& r = S->req[t];
            r.status = RT_ETIMEDOUT;
            r.finished = Clock::now();
        }
        S->queue.clear();
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
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
    Request r;
    r.desc = d;
    r.d_out = d_out;
    r.bytes = request_bytes(&d);
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
    out->queue_ms = (r.launched.time_since_epoch().count() > 0)
                        ? (float)std::chrono::duration<double, std::milli>(r.launched - r.submitted).count()
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
    size_t inflight = 0;
    for (const Flight& f : S->flights) inflight += f.tickets.size();
    out->in_flight = inflight;
    out->completed = S->completed;
    out->failed = S->failed;
    out->bytes_in_use = S->in_use;
    out->budget = S->budget;
    return RT_OK;
}

}  // extern "C"
