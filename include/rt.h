/*
 * rt.h -- C ABI of the GB300 (sm_103a) renderer for Newtonian ray tracing of
 * the conformal grating cloak (Halimeh, Schmied & Wegener, Opt. Express 2010).
 *
 * Method (paper section / equation):
 *   - refractive index n = 1/|1 + W0(i c k exp(i k (x + i y)))|, c = i A,
 *     k = 2 pi / Lambda (Sec. 2, Eq. 1; W0 is the principal Lambert branch,
 *     Eq. 13) and its gradient (Sec. 3, Eq. 12);
 *   - each ray is a particle obeying Newton's law derived from Fermat's
 *     principle (Sec. 3, Eqs. 9-11), integrated numerically inside the cloak
 *     and straight in air, refracted by Snell's law at the cloak boundary
 *     (Sec. 3);
 *   - the metal grating is the trochoid of Eq. 2 (Sec. 2), a mirror;
 *   - frames are compared by the image cross-correlation C of Eqs. 14-15
 *     (Sec. 5), C(0,0) over central horizontal fields of view (Table 1).
 *
 * Conventions.  All lengths are world units; Lambda sets the scale (renders
 * are invariant under a common scaling of every length).  x runs across the
 * grooves, y is the mirror normal, z runs along the grooves.  The cloak is
 * the box |x| <= E/2, |z| <= E/2, -A <= y <= -A + H; n = 1 outside it.
 *
 * Ownership.  Every pointer argument named d_* is device memory owned by the
 * caller; h_* is host memory owned by the caller.  The library owns what it
 * allocates inside an rt_scene (texture copy, work counters, statistics) and
 * frees it in rt_destroy_scene.  Scenes may be used from one host thread at
 * a time.
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Device-side work is enqueued asynchronously on it unless the
 * function says otherwise.
 *
 * Errors.  Functions return RT_OK (0) or a negative code; rt_last_error()
 * gives a message for the calling thread.  Nothing exits or aborts.  There is
 * no CPU fallback: without an sm_103 device the compute functions return
 * RT_ENODEV.
 */
#ifndef GRATINGRT_RT_H
#define GRATINGRT_RT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define RT_OK 0
#define RT_PENDING 1          /* rt_poll: the request is not finished yet      */
#define RT_EINVAL (-22)       /* invalid argument or descriptor                */
#define RT_ENOMEM (-12)       /* device or host allocation failed              */
#define RT_ENODEV (-19)       /* no sm_103 device current                      */
#define RT_EBUSY (-16)        /* rt_submit: over the ray-state budget          */
#define RT_ETIMEDOUT (-110)   /* a bounded wait ran out                        */
#define RT_ECUDA (-5)         /* a CUDA runtime call failed (see message)      */

/* scene kinds and options */
#define RT_MIRROR_FLAT 0      /* plane y = 0 (Fig. 3a)                         */
#define RT_MIRROR_TROCHOID 1  /* trochoid grating, Eq. 2 (Fig. 3b, 3c)         */
#define RT_MIRROR_GAUSS 2     /* Gaussian bump (Fig. 4b, 4c): the image of the
                                 flat mirror under z(w) = w + i A F(w/gauss_w),
                                 F the Faddeeva function; Eq. 5 in its shallow
                                 limit.  Height A, width gauss_w                */
#define RT_BG_CHECKER 0       /* two-colour checkerboard                       */
#define RT_BG_TEXTURE 1       /* greyscale texture, bilinear, wrapping         */
#define RT_RK4 0              /* classical Runge-Kutta, fixed step h           */
#define RT_DP45 1             /* Dormand-Prince 5(4), adaptive (rtol, atol)    */
#define RT_RK4T 2             /* classical Runge-Kutta on Eq. 11 in physical
                                 time t (state r, v with |v| = c0/n), fixed
                                 step h in t; wavefront loop only              */
#define RT_FP32 0             /* single precision bulk arithmetic              */
#define RT_FP64 1             /* double precision throughout                   */

/* per-ray status */
#define RT_RAY_OK 0           /* reached the background                        */
#define RT_RAY_SKY 1          /* left the scene away from the background       */
#define RT_RAY_MAX_BOUNCES 2  /* more than max_bounces reflections             */
#define RT_RAY_MAX_STEPS 3    /* more than max_steps integrator steps          */
#define RT_RAY_NAN 4          /* non-finite state                              */

/* rt_scene_desc.flags (Sec. 3, Sec. 4 and Figs. 5-7):
   RT_FLAG_REFERENCED  the cloak's index divided by n_min = 1/(1 + kA), so it is
                       >= 1 everywhere; the air keeps n = 1
   RT_FLAG_PLATE       no cloak: a homogeneous dielectric plate of index
                       1/n_min = 1 + kA on the flat mirror, filling the cloak's
                       box from the mirror (y = 0) to the box top (the ideal
                       reference of the referenced cloak); needs
                       mirror = RT_MIRROR_FLAT and cloak = 0
   RT_FLAG_FRESNEL     Fresnel weights at the box faces: a crossing keeps the
                       unpolarised transmittance on the refracted ray, and the
                       camera's path also traces each reflected ray (weight R,
                       at most 8 per sample), which is not split again (rays
                       Fresnel-reflected more than once are neglected); total
                       internal reflection keeps the full weight.
   Scenes with any of these are rendered by the wavefront loop (launch
   variant 3) only, in a build of it that the scenes without options do not
   pay for. */
#define RT_FLAG_REFERENCED 1
#define RT_FLAG_PLATE 2
#define RT_FLAG_FRESNEL 4

/*
 * Scene descriptor.  The camera is a pinhole at distance cam_dist from the
 * origin at elevation elev_deg and azimuth azim_deg, looking at the origin,
 * with horizontal full field of view hfov_deg and square pixels (Sec. 4).
 * The background stands in for the photograph of Fig. 2(a): a plane normal to
 * the mirrored view axis, cam_dist from the origin.  Ray directions of sample
 * s of pixel (i, j): pixel centre for spp = 1, one uniform offset in each cell
 * of an m x m grid for spp = m^2 and two uniforms otherwise, drawn from
 * SplitMix64 outputs 2c+1 and 2c+2 with c = ((scene_id*height + i)*width_out
 * + j)*spp + s (width_out = 1 for centre_line).
 */
typedef struct rt_scene_desc {
    double Lambda;            /* grating period (> 0)                           */
    double A;                 /* half peak-to-peak amplitude, 0 <= kA < 1       */
    double H, E;              /* cloak box height above y=-A (y=0 for the
                                 Gaussian bump) and x/z extent                 */
    double cam_dist, elev_deg, azim_deg, hfov_deg;
    double bg_cell;           /* checkerboard cell size                         */
    double tex_texel;         /* texture texel size                             */
    double colour0[3], colour1[3];  /* checkerboard colours, linear [0, 1]      */
    double h;                 /* RK4 step (in the ray parameter tau, |dr/dtau| = n); DP45 first step */
    double rtol, atol;        /* DP45 tolerances (atol in world length units)   */
    double h_max;             /* DP45 largest step                              */
    double gauss_w;           /* Gaussian bump width (RT_MIRROR_GAUSS), > 0;
                                 0 <= A < 0.8 gauss_w keeps the map one to one */
    uint64_t seed, scene_id;  /* jitter stream                                  */
    int64_t max_steps;        /* guard on integrator steps per ray              */
    const float* tex;         /* host, tex_size^2 row-major greyscale (TEXTURE) */
    int32_t mirror;           /* RT_MIRROR_*                                    */
    int32_t cloak;            /* 1: graded-index cloak box present (Eq. 1 on the
                                 trochoid, the Gaussian map on the bump)        */
    int32_t width, height;    /* image size                                     */
    int32_t spp;              /* samples per pixel                              */
    int32_t centre_line;      /* 1: render only the vertical centre line
                                 (height x 1 image, horizontal offset 0)        */
    int32_t background;       /* RT_BG_*                                        */
    int32_t tex_size;         /* texture side                                   */
    int32_t integrator;       /* RT_RK4 | RT_DP45 | RT_RK4T (RK4T: not with the
                                 Gaussian bump)                                 */
    int32_t precision;        /* RT_FP32 | RT_FP64                              */
    int32_t max_bounces;      /* guard on reflections per ray                   */
    int32_t flags;            /* RT_FLAG_* (0: the plain method; 0 for the
                                 Gaussian bump)                                 */
} rt_scene_desc;

/* Per-sample exit record: the start of the ray's final straight segment (its
   last reflection or cloak-exit point; the camera for a ray that meets
   nothing; the point where a guard stopped it), the segment's unit direction,
   the sample's colour and counters. */
typedef struct rt_ray_record {
    double pos[3];
    double dir[3];
    float rgb[3];
    int32_t status;           /* RT_RAY_*                                       */
    int32_t bounces;          /* reflections (grating, mirror, total)           */
    int32_t events;           /* located events inside the cloak                */
    int64_t steps;            /* integrator steps (accepted + rejected)         */
} rt_ray_record;

/* Counters accumulated over one rt_render call. */
typedef struct rt_stats {
    uint64_t rays;            /* camera samples traced                          */
    uint64_t steps;           /* integrator steps                               */
    uint64_t evals;           /* index/gradient evaluations                     */
    uint64_t newton;          /* W0 iterations                                  */
    uint64_t events;          /* located events                                 */
    uint64_t fp64_refine;     /* W0 refinements in FP64 near the branch point   */
    uint64_t status[5];       /* rays per RT_RAY_* status                       */
    uint64_t profile[4];      /* zero unless built with RT_PROFILE: per-warp
                                 cycles in the service pass and in the
                                 integration loop, loop iterations, and lanes
                                 inside the cloak summed over the iterations
                                 (wavefront variant: integration tasks, rays
                                 they took, service tasks, rays they took)     */
    uint64_t sched_timeouts;  /* wavefront variant: bounded waits on its work
                                 queues that gave up (the image is then
                                 incomplete and rt_scene_stats fails)           */
} rt_stats;

typedef struct rt_scene rt_scene;

/*
 * rt_create_scene: validate `desc` and build a scene on the current device:
 * copies the texture (if any) to device memory and allocates the scene's work
 * counters.  Synchronous.  Returns RT_EINVAL for an invalid descriptor
 * (message names the field), RT_ENODEV without an sm_103 device, RT_ENOMEM.
 */
int rt_create_scene(const rt_scene_desc* desc, rt_scene** out);

/* rt_destroy_scene: free the scene (waits for its outstanding work). NULL is a no-op. */
void rt_destroy_scene(rt_scene* scene);

/*
 * rt_render: render the whole image (Sec. 4; Figs. 3-7).
 *   d_rgb   height x width_out x 3 float, mean colour per pixel (linear)
 *   d_rgb8  nullable, height x width_out x 3 bytes, q = floor(clamp(c)*255+1/2)
 *   d_rec   nullable, height x width_out x spp records in sample order
 * Asynchronous on `stream`.  Counters of the call can be read with
 * rt_scene_stats once the stream has completed.
 */
int rt_render(rt_scene* scene, float* d_rgb, uint8_t* d_rgb8, rt_ray_record* d_rec, void* stream);

/*
 * rt_render_pixels: render the listed pixels only (flat indices i*width_out+j,
 * device array d_pix of npix entries); d_rgb is npix x 3, d_rec (nullable)
 * npix x spp.  Same arithmetic as rt_render for those pixels.
 */
int rt_render_pixels(rt_scene* scene, const int64_t* d_pix, int64_t npix, float* d_rgb,
                     rt_ray_record* d_rec, void* stream);

/*
 * rt_render_host: rt_render into library-owned device buffers followed by the
 * copy of the colours (height x width_out x 3 float) and, if h_rgb8 is not
 * NULL, the 8-bit image to host memory; waits for `stream`.
 */
int rt_render_host(rt_scene* scene, float* h_rgb, uint8_t* h_rgb8, void* stream);

/* rt_scene_stats: counters of the last render of this scene (waits for it).
   Returns RT_ETIMEDOUT (counters filled in) if that render gave up a bounded
   wait of the wavefront loop's work queues. */
int rt_scene_stats(rt_scene* scene, rt_stats* out);

/*
 * rt_scene_set_launch: launch configuration of the scene's render kernel (the
 * knobs of the autotuner; results are identical for every setting).
 *   variant     0, 1, 2: the per-lane loop (one pixel per lane) compiled for
 *               4, 5, 6 resident blocks of 128 threads per SM (1 and 2 for
 *               FP32 RK4 only); 3: the wavefront loop (a pool of pixels in
 *               flight per block, rays inside the cloak regrouped into full
 *               warps; the only one for RT_RK4T and for scenes with
 *               flags); -1 keeps the current one
 *   min_active  the integration loop of a warp continues while at least this
 *               many of its 32 lanes are inside the cloak (1..32); 0 keeps it
 * Returns RT_EINVAL for values out of range or a variant not compiled for the
 * scene's precision and integrator.
 */
int rt_scene_set_launch(rt_scene* scene, int32_t variant, int32_t min_active);

/* rt_scene_get_launch: the current variant, min_active and grid size (blocks). */
int rt_scene_get_launch(rt_scene* scene, int32_t* variant, int32_t* min_active, int32_t* grid);

/*
 * rt_scene_set_wait_limit: bounds of the waits of the wavefront loop
 * (variant 3) on its per-block work queues, for this scene's later renders.
 * The paper has no counterpart: this is the runtime's failure detection.
 *   spin_limit  attempts (each followed by a short sleep) a wait makes before
 *               the launch gives it up: 1..2^24; 0 restores the default 2^24
 *               (about a second of waiting)
 *   hold_lock   0 for normal renders; nonzero starts every block with its
 *               queue lock taken and never released, so that every wait of
 *               the launch runs out after spin_limit attempts.  This makes a
 *               bounded wait expire on purpose, for tests of failure
 *               detection: no GPU fault is involved, every block returns,
 *               the image is left incomplete and rt_scene_stats reports
 *               RT_ETIMEDOUT with the timeouts counted in sched_timeouts.
 * Host only (takes effect at the next render).  Returns RT_EINVAL for a
 * spin_limit out of range.
 */
int rt_scene_set_wait_limit(rt_scene* scene, int32_t spin_limit, int32_t hold_lock);

/*
 * rt_scene_autotune: time the scene's launch configurations (every
 * register-budget variant compiled for its precision and integrator, times
 * min_active in {12, 16, 20, 24, 28}; median of `trials` full renders into
 * d_rgb, which must hold one image) and keep the fastest.  The choice is
 * cached per scene class (precision, integrator, mirror, cloak and the power
 * of two of width * height * spp) for the process, and in the text file named
 * by the environment variable RT_AUTOTUNE_CACHE if set; a cached class is not
 * timed again.  Synchronous.  Outputs (nullable) report the choice.
 */
int rt_scene_autotune(rt_scene* scene, float* d_rgb, int32_t trials, void* stream, int32_t* variant,
                      int32_t* min_active);

/*
 * Batches: several scenes rendered by one persistent launch whose warps share
 * one work list, so scenes of uneven size, spp and path length balance on
 * the GPU.  The scenes must share precision and integrator, live on the
 * current device and outlive the batch.  The launch (counter reset and
 * kernel) is recorded in a CUDA graph by the first rt_batch_render and
 * replayed by later calls; results equal those of rendering each scene alone.
 */
typedef struct rt_batch rt_batch;

/* rt_batch_create: copy the scene tables of scenes[0..n-1] to the device. */
int rt_batch_create(rt_scene* const* scenes, int32_t n, rt_batch** out);

/*
 * rt_batch_update: new scene parameters for the next renders of the batch (a
 * moving camera, another grating, another seed: one frame's inputs).  descs is
 * a host array of n descriptors (n equal to the batch's), each with the same
 * image size, samples per pixel, precision, integrator, background kind and
 * flags as the scene it replaces (the textures stay the scenes').  The scene
 * table is rebuilt on the host, staged in pinned host memory and copied to the
 * device on `stream` (asynchronous, ordered before the next rt_batch_render on
 * that stream; a second update waits for the first copy).  *h2d_bytes
 * (nullable) receives the bytes copied.  RT_EINVAL for a descriptor that does
 * not fit the batch.
 */
int rt_batch_update(rt_batch* batch, const rt_scene_desc* descs, int32_t n, void* stream, uint64_t* h2d_bytes);

/* rt_batch_destroy: free the batch (waits for its outstanding work). */
void rt_batch_destroy(rt_batch* batch);

/*
 * rt_batch_render: render every scene of the batch; d_rgb is a host array of
 * n device pointers, d_rgb[i] receiving scene i's height x width_out x 3
 * float image.  Asynchronous on `stream` (a change of output pointers
 * uploads the new table first, synchronously).
 */
int rt_batch_render(rt_batch* batch, float* const* d_rgb, void* stream);

/* rt_batch_stats: counters of the last batch render, summed over its scenes. */
int rt_batch_stats(rt_batch* batch, rt_stats* out);

/* rt_batch_set_launch / rt_batch_get_launch: min_active of the batch kernel
   (1..32), its grid and the total number of pixels. */
int rt_batch_set_launch(rt_batch* batch, int32_t min_active);
int rt_batch_get_launch(rt_batch* batch, int32_t* min_active, int32_t* grid, int64_t* total_pixels);

/* rt_batch_autotune: as rt_scene_autotune for the batch kernel (min_active). */
int rt_batch_autotune(rt_batch* batch, float* const* d_rgb, int32_t trials, void* stream, int32_t* min_active);

/* rt_validate_desc: check a descriptor on the host (no device needed);
   RT_OK or RT_EINVAL with the offending field in rt_last_error(). */
int rt_validate_desc(const rt_scene_desc* desc);

/*
 * Serving: rt_submit queues a render request; a worker thread admits queued
 * requests in arrival order while the sum of their ray-state footprints
 * (76 bytes per sample: 64 of ray state and a 12-byte colour slot; 16 bytes
 * per pixel: the float output image and a sample counter; see
 * rt_request_bytes) stays within the budget.  A request that fits may pass
 * queued requests that do not fit yet (so that a small request does not wait
 * behind a large one for the budget), but no request is passed more than 32
 * times; the worker looks 64 requests deep.  It publishes each admitted
 * request into a ring of request slots in device memory (one ring per
 * precision and integrator, 1024 requests in flight each).  A persistent
 * launch of the wavefront loop takes samples from the ring up to the
 * published count: requests published while it runs are taken up as its
 * lanes free up, so their work overlaps on the device with the requests
 * already running, and a small request does not wait for a large one to end.
 * A launch ends when no sample is left; at most max_inflight launches run at
 * once.  The last pixel of a request writes a completion record into
 * host-mapped memory.  Each result equals a render of the scene alone.
 * Scratch and textures of the requests in flight come from a device arena
 * allocated with the server (at most the budget, at most half of the free
 * device memory); nothing is allocated per request.  Scenes with options
 * (RT_FLAG_*) and the Gaussian bump are not served.
 */
typedef struct rt_server rt_server;

typedef struct rt_result {
    int32_t status;           /* RT_OK or the error of the request           */
    float latency_ms;         /* submission to completion                     */
    float queue_ms;           /* submission to publication on the device       */
    uint64_t rays;            /* camera samples of the request                */
} rt_result;

typedef struct rt_server_info {
    uint64_t queued, in_flight, completed, failed;
    uint64_t bytes_in_use, budget;
} rt_server_info;

/* rt_request_bytes: the ray-state footprint a request of `desc` holds in a
   server's budget while it is in flight (host only).  RT_EINVAL for an
   invalid descriptor. */
int rt_request_bytes(const rt_scene_desc* desc, uint64_t* bytes);

/* rt_server_create: server on the current device; max_inflight 1..16 launches
   of the server kernel per ring; RT_ENOMEM if the arena cannot be allocated. */
int rt_server_create(size_t ray_state_budget_bytes, int32_t max_inflight, rt_server** out);

/* rt_server_destroy: fails the requests not yet admitted (RT_ETIMEDOUT),
   finishes the requests in flight, stops the worker. */
void rt_server_destroy(rt_server* server);

/* rt_submit: queue a request rendering into d_out (caller-owned device image
   of height x width_out x 3 floats, untouched until the request completes).
   RT_EINVAL for an invalid descriptor, RT_EBUSY if the request alone exceeds
   the budget or the queue is full. */
int rt_submit(rt_server* server, const rt_scene_desc* desc, float* d_out, uint64_t* ticket);

/* rt_poll: RT_OK (result in *out, the ticket is then forgotten) or the
   request's error; RT_PENDING if not finished and timeout_us <= 0; waits up
   to timeout_us microseconds otherwise and returns RT_ETIMEDOUT if still
   pending. */
int rt_poll(rt_server* server, uint64_t ticket, int32_t timeout_us, rt_result* out);

/* rt_server_stats: queue and budget state. */
int rt_server_stats(rt_server* server, rt_server_info* out);

/*
 * rt_xcorr: image cross-correlation C(0,0) of Eqs. 14-15 (Sec. 5) between
 * the reference d_f and d_g (both height x width x channels float, device).
 * For each of the n_fov fields of view fov_deg[q] (host array, degrees) the
 * window is the columns whose pixel-centre horizontal angle is within
 * fov/2 of the image centre for a camera of horizontal field hfov_deg (a
 * width-1 centre-line image has its one column at angle 0).  Per window and
 * channel c: C_c = sum (f-<f>)(g-<g>) / sum (f-<f>)^2 with the means over the
 * window (Eq. 14); the last entry treats the channels as one stacked image.
 * Writes n_fov x (channels+1) doubles to d_out (device).  Empty windows give
 * NaN.  Asynchronous; uses scratch owned by the library.
 */
int rt_xcorr(const float* d_f, const float* d_g, int32_t height, int32_t width, int32_t channels,
             const double* fov_deg, int32_t n_fov, double hfov_deg, double* d_out, void* stream);

/*
 * rt_xcorr_noalloc: rt_xcorr without any device allocation, for callers that
 * cannot allocate -- hosts that give all device memory to their own pool and
 * forbid allocations behind its back, and latency-bound loops in which an
 * allocation call (which can synchronise the device or take a driver lock) is
 * not acceptable.  The paper has no counterpart: this is an interface
 * variant of rt_xcorr with the same arguments, arithmetic and results.
 * Its scratch is a fixed device array of 16 MiB and 129 KiB inside the
 * library, held by every GPU that loads the library until the process
 * exits; images with
 * min(ceil(height / 64), 64) * width * channels > 524288 are rejected with
 * RT_EINVAL.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  The address is kept for the life of the process, so do not call
 * this entry point on a device after cudaDeviceReset of that device.  Every call shares the one array, so calls that overlap on the GPU
 * (on different streams, or from different threads) race; each call
 * overwrites all scratch it reads, so nothing needs clearing.  Asynchronous.
 */
int rt_xcorr_noalloc(const float* d_f, const float* d_g, int32_t height, int32_t width, int32_t channels,
                     const double* fov_deg, int32_t n_fov, double hfov_deg, double* d_out, void* stream);

/*
 * rt_xcorr_map: the cross-correlation function C(di, dj) of Eq. 15 over pixel
 * shifts (Sec. 5), its peak and its mean over several reference pairs.
 * d_f[p], d_g[p] (host arrays of n_pairs device pointers, 1..64 pairs): the
 * reference and compared images, each height x width x channels float.  The
 * window is the columns within the field of view fov_deg (as in rt_xcorr) of
 * both images, which have no values outside it:
 *   f' = f - <f>, g' = g - <g> with the means over the window (Eq. 14),
 *   C_c(di, dj) = sum f'(i, j) g'(i + di, j + dj) / sum f'(i, j)^2,
 * the numerator over the pixels where both lie in the window, the denominator
 * over the whole window; di is a row shift, dj a column shift, |di| <=
 * max_di, |dj| <= max_dj (0..64).  Per channel and for the stacked channels
 * (sum of numerators over sum of denominators), averaged over the pairs.
 * d_map (device) receives (2 max_di + 1) x (2 max_dj + 1) x (channels + 1)
 * doubles, row-major in (di, dj, channel); d_peak (device, nullable) receives
 * the largest stacked value of the mean map and its (di, dj) as three
 * doubles, the first in row-major order among equal values.  RT_EINVAL for an
 * empty window or arguments out of range.  Asynchronous; its scratch is
 * allocated and freed in stream order on `stream`.
 */
int rt_xcorr_map(const float* const* d_f, const float* const* d_g, int32_t n_pairs, int32_t height, int32_t width,
                 int32_t channels, double fov_deg, double hfov_deg, int32_t max_di, int32_t max_dj, double* d_map,
                 double* d_peak, void* stream);

/*
 * rt_eval_medium: W0, n and the ray force grad(n^2)/2 at npoints points
 * (device d_xy: x0,y0,x1,y1,..., world units) for grating period Lambda and
 * amplitude A (Eqs. 1, 12, 13).  d_out gets per point
 * (Re W0, Im W0, n, F_x, F_y) in world units.  precision RT_FP32 | RT_FP64.
 */
int rt_eval_medium(int32_t precision, double Lambda, double A, const double* d_xy, int64_t npoints,
                   double* d_out, void* stream);

/* rt_last_error: message of the last failing call on this thread ("" if none). */
const char* rt_last_error(void);

/* rt_version: library version string. */
const char* rt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GRATINGRT_RT_H */
