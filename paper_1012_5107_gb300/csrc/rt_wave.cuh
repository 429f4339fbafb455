// rt_wave.cuh -- the wavefront form of the render loop.
//
// The persistent loop of rt_trace.cuh keeps one pixel per lane, so a warp
// integrates only while enough of its own lanes are inside the cloak and the
// others wait.  Here a block keeps a pool of pixels in flight in shared memory
// (each with its ray state in the cloak and everything else a lane would own)
// and two queues of pool entries: rays inside the cloak, ready to step, and
// rays that need service (an event located, a sample finished, a new pixel).
// Each warp repeatedly takes one task:
//   * integrate: up to 32 rays from the cloak queue, stepped together until
//     fewer than min_active (scaled to the rays taken) are still inside or the
//     step cap of a task is reached; the rays still inside go back to the
//     cloak queue, the others to the service queue;
//   * serve: up to 32 entries of the service queue, filled up with free pool
//     entries that take new samples; each lane runs the service steps of
//     rt_trace.cuh until its ray is inside the cloak again (back to the cloak
//     queue) or the work list is exhausted (back to the free list).
// The work items are samples, not pixels: the samples of a pixel are traced
// at the same time, so the longest unit of work is one ray (a pixel of 4
// samples in a row would be up to four times longer and set the end of the
// launch).  Each finished sample leaves its colour in a scratch slot and
// counts itself in its pixel's counter; the last one adds the pixel's colours
// in sample order, the order of the per-lane loop, so the images are the same
// and only the grouping of rays into warps changes.
//
// The queues are rings of 16-bit pool indices guarded by a block-level lock
// (an atomic flag in shared memory) that one lane per warp takes for a few
// dozen cycles per task; every wait on it is bounded (WaveWait) and a timeout
// is counted in counters[kCounters - 1] (reported as an error by the host).
#pragma once

#include "rt_trace.cuh"

namespace grt {

// Step cap of one integration task: the rays still inside go back to the
// cloak queue after it, and the warp takes its next task (the step's batched
// launch, CUDA events: 7.10 ms at 128, 7.14 at 96, 7.29 at 64, 7.16 at 256,
// 7.28 at 512, 7.34 at 1024)
constexpr int kWaveTaskSteps = 128;
constexpr int kWaveSpin = kDefaultWaitSpin;  // attempts (with a short sleep) before a wait gives up

// The block shape of the loop for a precision and integrator: threads per
// block, blocks per SM (which sets the registers a thread may use: 65536 /
// (threads x blocks)) and P, the samples in flight per block -- more than the
// block's lanes, so that a warp always finds work while the other warps hold
// theirs.  FP32 RK4: two blocks of 256 threads, 128 registers.  FP32
// Dormand-Prince keeps the running sums of its stages and two states live
// through a step, which spills at 128 registers: one block of 384 threads
// (12 warps, up to 168 registers).  FP64: one block of 256 threads.
template <class R, int INTEG>
struct WaveShape {
    static constexpr bool kWide = sizeof(R) == 4 && integ_of(INTEG) == RT_DP45;
    static constexpr int kBlock = kWide ? 384 : 256;
    static constexpr int kMinBlocks = (sizeof(R) == 4 && !kWide) ? 2 : 1;
    static constexpr int P = kWide ? 576 : (sizeof(R) == 4 ? 384 : 320);
};

template <class R, int INTEG>
constexpr size_t wave_smem_bytes()
{
    constexpr int P = WaveShape<R, INTEG>::P;
    return (sizeof(Cold<R>) + sizeof(Box<R>)) * P + 3 * sizeof(short) * P;
}

// Bytes of the Fresnel branch queues of a launch of `grid` blocks.
template <class R, int INTEG>
constexpr size_t wave_branch_bytes(int grid)
{
    return (size_t)grid * WaveShape<R, INTEG>::P * kMaxBranches * sizeof(Branch<R>);
}

struct WaveCtl {
    int lock;
    int in_head, in_cnt;     // cloak queue
    int sv_head, sv_cnt;     // service queue
    int fr_cnt;              // free list (stack)
    int exhausted;           // the work list has no pixels left
    int error;
};

enum : int { WT_WAIT = 0, WT_INT = 1, WT_SRV = 2, WT_DONE = 3, WT_ERR = 4 };
enum : int { WD_NONE = 0, WD_IN = 1, WD_SRV = 2, WD_FREE = 3 };

// How the waits of a launch are bounded: `spin` attempts per wait (kWaveSpin
// unless the scene asks for fewer) and, with `hold` set, every block starts
// with its queue lock taken, so that every wait runs out and the launch ends
// with the timeouts counted (a test of failure detection; nothing faults).
struct WaveWait {
    int spin;
    int hold;
};

__device__ __forceinline__ bool wave_acquire(int* lock, int spin)
{
    for (int it = 0; it < spin; ++it) {
        if (atomicCAS(lock, 0, 1) == 0) {
            __threadfence_block();
            return true;
        }
        __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void wave_release(int* lock)
{
    __threadfence_block();
    atomicExch(lock, 0);
}

// Publish the pool entries of the calling warp's lanes to the queue each
// names (dest); lanes with WD_NONE take part without publishing.  Returns
// false if the lock could not be taken.
template <int P>
__device__ __forceinline__ bool wave_push(WaveCtl& Q, short* inq, short* svq, short* frq, unsigned lane, int p,
                                          int dest, int spin)
{
    __threadfence_block();      // this lane's pool writes before its index is published
    const unsigned mi = __ballot_sync(0xffffffffu, dest == WD_IN);
    const unsigned ms = __ballot_sync(0xffffffffu, dest == WD_SRV);
    const unsigned mf = __ballot_sync(0xffffffffu, dest == WD_FREE);
    if ((mi | ms | mf) == 0u) return true;
    int ok = 1, ti = 0, ts = 0, tf = 0;
    if (lane == 0) {
        ok = wave_acquire(&Q.lock, spin) ? 1 : 0;
        if (ok) {
            ti = Q.in_head + Q.in_cnt;
            ts = Q.sv_head + Q.sv_cnt;
            tf = Q.fr_cnt;
            Q.in_cnt += __popc(mi);
            Q.sv_cnt += __popc(ms);
            Q.fr_cnt += __popc(mf);
            if (mf) Q.exhausted = 1;
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return false;
    ti = __shfl_sync(0xffffffffu, ti, 0);
    ts = __shfl_sync(0xffffffffu, ts, 0);
    tf = __shfl_sync(0xffffffffu, tf, 0);
    const unsigned lt = (1u << lane) - 1u;
    if (dest == WD_IN) inq[(ti + __popc(mi & lt)) % P] = (short)p;
    else if (dest == WD_SRV) svq[(ts + __popc(ms & lt)) % P] = (short)p;
    else if (dest == WD_FREE) frq[tf + __popc(mf & lt)] = (short)p;
    __threadfence_block();
    __syncwarp();
    if (lane == 0) wave_release(&Q.lock);
    return true;
}

// A finished sample (its colour in C.acc): with one sample per pixel the pixel
// is written at once; otherwise the colour goes to the sample's scratch slot
// and the last sample of the pixel to finish writes the pixel.
template <class R, class Src>
__device__ __forceinline__ void wave_finish_sample(const Src& src, const DevScene& sc, const Cold<R>& C)
{
    float acc[3] = {C.acc[0], C.acc[1], C.acc[2]};
    const int spp = sc.spp;
    if (spp > 1) {
        float* col = src.sample_col(C.scene, C.work, C.sample);
        __stcg(reinterpret_cast<float4*>(col), make_float4(acc[0], acc[1], acc[2], 0.0f));
        __threadfence();                                     // the colour before the count
        if (atomicAdd(src.pixel_count(C.scene, C.work), 1) != spp - 1) return;
        __threadfence();                                     // the count before the other colours
        const float4* base = reinterpret_cast<const float4*>(col) - C.sample;
        acc[0] = acc[1] = acc[2] = 0.0f;
        for (int q = 0; q < spp; ++q) {
            const float4 v = __ldcg(base + q);
            acc[0] += v.x;
            acc[1] += v.y;
            acc[2] += v.z;
        }
        src.release_count(C.scene, C.work);
        // the block is dead: drop its lines from L2 without a write-back
        const char* blk = reinterpret_cast<const char*>(base);
        for (int64_t b = 0; b < col_block_bytes(spp); b += 128)
            asm volatile("discard.global.L2 [%0], 128;" ::"l"(blk + b) : "memory");
    }
    const float inv = 1.0f / (float)spp;
    float c[3];
    for (int a = 0; a < 3; ++a) c[a] = acc[a] * inv;
    float* o = src.rgb_of(C.scene) + 3 * C.work;
    o[0] = c[0]; o[1] = c[1]; o[2] = c[2];
    uint8_t* q8 = src.rgb8_of(C.scene);
    if (q8) {
        uint8_t* q = q8 + 3 * C.work;
        q[0] = quantize8(c[0]); q[1] = quantize8(c[1]); q[2] = quantize8(c[2]);
    }
    src.pixel_done(C.scene);
}

template <class R, int INTEG, bool OPT, class Src>
__device__ __forceinline__ void wave_loop(const Src& src, unsigned long long* counters, int min_active, WaveWait ww)
{
    constexpr int P = WaveShape<R, INTEG>::P;
    extern __shared__ __align__(16) unsigned char wave_smem[];
    Cold<R>* cold = reinterpret_cast<Cold<R>*>(wave_smem);
    Box<R>* boxes = reinterpret_cast<Box<R>*>(wave_smem + sizeof(Cold<R>) * P);
    short* inq = reinterpret_cast<short*>(wave_smem + (sizeof(Cold<R>) + sizeof(Box<R>)) * P);
    short* svq = inq + P;
    short* frq = svq + P;
    __shared__ WaveCtl Q;

    Branch<R>* branches = reinterpret_cast<Branch<R>*>(src.branches);
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        Cold<R>& C = cold[p];
        C.rays = 0;
        C.nevents = 0;
        C.scene = 0;
        for (int q = 0; q < 5; ++q) C.stat[q] = 0;
        C.br = branches ? branches + ((int64_t)blockIdx.x * P + p) * kMaxBranches : nullptr;
        frq[p] = (short)p;
    }
    if (threadIdx.x == 0) {
        Q.lock = ww.hold ? 1 : 0;
        Q.in_head = Q.in_cnt = Q.sv_head = Q.sv_cnt = 0;
        Q.fr_cnt = P;
        Q.exhausted = 0;
        Q.error = 0;
    }
    __syncthreads();

    const unsigned lane = threadIdx.x & 31u;
    LaneStats st = {0u, 0u, 0u, 0u};
#if RT_PROFILE
    // per warp (lane 0): cycles in integration tasks, cycles in service
    // tasks, integration iterations, cycles from the start to the exit
    unsigned long long prof[4] = {0, 0, 0, 0};
    const long long t_start = clock64();
#endif
    int idle = 0;
    bool failed = false;
    for (;;) {
        // ---- take a task (the leader decides under the lock) ----
        int task = WT_WAIT, m1 = 0, m2 = 0, b1 = 0, b2 = 0, locked = 0;
        if (lane == 0) {
            if (!wave_acquire(&Q.lock, ww.spin)) {
                task = WT_ERR;
            } else {
                locked = 1;
                const int nin = Q.in_cnt, nsv = Q.sv_cnt, nfr = Q.fr_cnt;
                const bool fresh = !Q.exhausted && nfr > 0;
                if (Q.error) {
                    task = WT_ERR;
                } else if (nsv >= 32 || (nin < 32 && (nsv > 0 || fresh))) {
                    task = WT_SRV;
                    m1 = min(32, nsv);
                    b1 = Q.sv_head;
                    Q.sv_head = (Q.sv_head + m1) % P;
                    Q.sv_cnt -= m1;
                    m2 = fresh ? min(32 - m1, nfr) : 0;
                    Q.fr_cnt -= m2;
                    b2 = Q.fr_cnt;
                } else if (nin > 0) {
                    task = WT_INT;
                    m1 = min(32, nin);
                    b1 = Q.in_head;
                    Q.in_head = (Q.in_head + m1) % P;
                    Q.in_cnt -= m1;
                } else if (Q.exhausted) {
                    // nothing queued and no new pixels: whatever other warps
                    // hold, they finish themselves
                    task = WT_DONE;
                }
            }
        }
        task = __shfl_sync(0xffffffffu, task, 0);
        m1 = __shfl_sync(0xffffffffu, m1, 0);
        m2 = __shfl_sync(0xffffffffu, m2, 0);
        b1 = __shfl_sync(0xffffffffu, b1, 0);
        b2 = __shfl_sync(0xffffffffu, b2, 0);
        int p = -1;
        bool fresh = false;
        if (task == WT_INT && (int)lane < m1) p = inq[(b1 + (int)lane) % P];
        if (task == WT_SRV) {
            if ((int)lane < m1) {
                p = svq[(b1 + (int)lane) % P];
            } else if ((int)lane < m1 + m2) {
                p = frq[b2 + (int)lane - m1];
                fresh = true;
            }
        }
        __syncwarp();
        if (lane == 0 && locked) wave_release(&Q.lock);
        if (task == WT_ERR) { failed = true; break; }
        if (task == WT_DONE) break;
        if (task == WT_WAIT) {
            if (++idle > ww.spin) { failed = true; break; }
            __nanosleep(256);
            continue;
        }
        idle = 0;
#if RT_PROFILE
        const long long t_task = clock64();
#endif

        Cold<R>& C = cold[p >= 0 ? p : 0];
        const DevScene& sc = src.scene(C.scene);
        Box<R> b;
        int phase = PH_IDLE, surf = EV_NONE, steps = 0;
        int dest = WD_NONE;
        if (task == WT_INT) {
            // ---- integrate ----
            if (p >= 0) {
                b = boxes[p];
                phase = PH_BOX;
                surf = C.surf;
                steps = C.steps;
            }
            const int need = max(1, m1 - (32 - min_active));
            // step constants: read in place from the kernel parameters, or
            // copied once per task from a scene table in device memory
            const StepConst<R>* kp = &step_const<R>(sc);
            StepConst<R> kc;
            if constexpr (!Src::kParamScene) {
                kc = *kp;
                kp = &kc;
            }
            const int64_t max_steps = sc.max_steps;
            int safe = 0;                          // steps without the faces' tests (box_step_into)
            for (int it = 0; it < kWaveTaskSteps; ++it) {
#if RT_PROFILE
                prof[2] += 1;
#endif
                if (phase == PH_BOX) box_step<R, INTEG>(*kp, max_steps, C, b, phase, surf, steps, st, safe);
                if (__popc(__ballot_sync(0xffffffffu, phase == PH_BOX)) < need) break;
            }
            if (p >= 0) {
                boxes[p] = b;
                C.surf = surf;
                C.steps = steps;
                C.phase = phase;
                dest = (phase == PH_BOX) ? WD_IN : WD_SRV;
            }
        } else {
            // ---- serve ----
            if (p >= 0) {
                if (!fresh) {
                    b = boxes[p];
                    phase = C.phase;
                    surf = C.surf;
                    steps = C.steps;
                }
                while (phase != PH_BOX && phase != PH_EXIT) {
                    if (phase == PH_EVENT || phase == PH_GUARD)
                        service_event<R, INTEG, OPT>(src.scene(C.scene), C, b, phase, surf, steps, src.rec_of(C.scene), st);
                    if (phase == PH_IDLE) {
                        const int64_t ws = src.grab(counters, lane);
                        if (ws < 0) { phase = PH_EXIT; break; }
                        int s, sample;
                        int64_t pix, out;
                        src.map_sample(ws, s, pix, out, sample);
                        C.scene = s;
                        C.work = out;
                        C.pix = pix;
                        C.sample = sample;
                        C.acc[0] = C.acc[1] = C.acc[2] = 0.0f;
                        start_sample<R, OPT>(src.scene(s), C, phase, surf, steps);
                    }
                    const DevScene& scs = src.scene(C.scene);
                    if (phase == PH_AIR) air_segment<R, INTEG, OPT>(scs, C, b, phase, surf, steps, src.rec_of(C.scene), st);
                    if (phase == PH_DONE) {
                        if (OPT && C.ibr < C.nbr) {
                            start_branch<R, INTEG>(scs, C, b, phase, surf, steps, st);   // next Fresnel branch
                        } else {
                            rt_ray_record* rec = src.rec_of(C.scene);
                            if (rec && (opt_flags<OPT>(scs) & RT_FLAG_FRESNEL)) {
                                // the record's colour: the sample's, summed over its paths
                                rt_ray_record* o = rec + C.work * scs.spp + C.sample;
                                o->rgb[0] = C.acc[0]; o->rgb[1] = C.acc[1]; o->rgb[2] = C.acc[2];
                            }
                            wave_finish_sample(src, scs, C);
                            phase = PH_IDLE;
                        }
                    }
                }
                if (phase == PH_BOX) {
                    boxes[p] = b;
                    C.surf = surf;
                    C.steps = steps;
                    C.phase = PH_BOX;
                    dest = WD_IN;
                } else {
                    dest = WD_FREE;
                }
            }
        }
        __syncwarp();
#if RT_PROFILE
        prof[task == WT_INT ? 0 : 1] += (unsigned long long)(clock64() - t_task);
#endif
        if (!wave_push<P>(Q, inq, svq, frq, lane, p, dest, ww.spin)) { failed = true; break; }
    }
#if RT_PROFILE
    prof[3] = (unsigned long long)(clock64() - t_start);
#endif
    if (failed && lane == 0) {
        atomicExch(&Q.error, 1);
        atomicAdd(&counters[kCounters - 1], 1ull);
    }
    __syncthreads();

    // counters: per-thread integration counters and the pool's per-pixel ones
    uint32_t v[11] = {0u, st.steps, st.evals, st.newton, 0u, st.refine, 0u, 0u, 0u, 0u, 0u};
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const Cold<R>& C = cold[p];
        v[0] += C.rays;
        v[4] += C.nevents;
        for (int q = 0; q < 5; ++q) v[6 + q] += C.stat[q];
    }
#pragma unroll
    for (int q = 0; q < 11; ++q) {
        unsigned long long x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0 && x) atomicAdd(&counters[1 + q], x);
    }
#if RT_PROFILE
    for (int q = 0; q < 4; ++q) {
        unsigned long long x = prof[q];
        if (lane == 0 && x) atomicAdd(&counters[12 + q], x);
    }
#endif
}

template <class R, int INTEG, bool OPT>
__global__ void __launch_bounds__(WaveShape<R, INTEG>::kBlock, WaveShape<R, INTEG>::kMinBlocks) wave_kernel(const __grid_constant__ DevScene sc,
                                                            float* __restrict__ rgb, uint8_t* __restrict__ rgb8,
                                                            rt_ray_record* rec, unsigned long long* counters,
                                                            int min_active, float* samp_col, int* pix_cnt,
                                                            void* branches, WaveWait ww)
{
    const OneScene src{sc, rgb, rgb8, rec, samp_col, pix_cnt, branches};
    wave_loop<R, INTEG, OPT>(src, counters, min_active, ww);
}

template <class R, int INTEG, bool OPT>
__global__ void __launch_bounds__(WaveShape<R, INTEG>::kBlock, WaveShape<R, INTEG>::kMinBlocks) wave_batch_kernel(
    const DevScene* __restrict__ scenes, const int64_t* __restrict__ offsets, const int64_t* __restrict__ soffsets,
    float* const* __restrict__ rgbs, int n, int64_t total, int64_t total_samples, float* samp_col, int* pix_cnt,
    void* branches, unsigned long long* counters, int min_active)
{
    const ManyScenes src{scenes, offsets, soffsets, rgbs, n, total, total_samples, samp_col, pix_cnt, branches};
    wave_loop<R, INTEG, OPT>(src, counters, min_active, WaveWait{kWaveSpin, 0});
}

}  // namespace grt
