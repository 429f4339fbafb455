// rt_api.cu -- host runtime behind the C ABI of include/rt.h: descriptor
// validation, scene tables on the device, launches, counters and errors.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "rt_internal.h"

namespace grt {

static thread_local char g_err[512];

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
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

struct rt_scene {
    rt_scene_desc desc;
    DevScene dev;
    int device;
    int nsm;
    int variant;              // launch variant of the render (per-lane loop or wavefront loop)
    int min_active;           // lanes inside the cloak that keep the integration loop going
    int grid;
    float* d_tex;
    unsigned long long* d_counters;
    float* d_host_rgb;        // buffers of rt_render_host
    uint8_t* d_host_rgb8;
    float* d_samp;            // wavefront loop: per-sample colours and per-pixel counters,
    int* d_pcnt;              // grown on demand (stream-ordered)
    int64_t samp_cap, pix_cap;
    void* d_branch;           // Fresnel branch queues of the wavefront loop (stream-ordered)
    size_t branch_cap;
    cudaEvent_t done;
    bool rendered;
    WaitLimit wait;           // bounds of the wavefront loop's waits (rt_scene_set_wait_limit)
};

static int current_device(int* dev)
{
    cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess) {
        set_error("no CUDA device: %s", cudaGetErrorString(e));
        return RT_ENODEV;
    }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, *dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, *dev);
    if (major != 10 || minor != 3) {
        set_error("device %d is sm_%d%d; this library is built for sm_103a only", *dev, major, minor);
        return RT_ENODEV;
    }
    return RT_OK;
}

static int validate(const rt_scene_desc* d)
{
    RT_REQ(d, "desc is NULL");
    RT_REQ(d->Lambda > 0.0 && std::isfinite(d->Lambda), "Lambda must be finite and > 0");
    RT_REQ(d->mirror == RT_MIRROR_FLAT || d->mirror == RT_MIRROR_TROCHOID || d->mirror == RT_MIRROR_GAUSS,
           "mirror must be RT_MIRROR_FLAT, RT_MIRROR_TROCHOID or RT_MIRROR_GAUSS");
    RT_REQ(d->cloak == 0 || d->cloak == 1, "cloak must be 0 or 1");
    RT_REQ(!d->cloak || d->mirror != RT_MIRROR_FLAT, "the cloak needs the trochoid (or Gaussian) mirror");
    if (d->mirror == RT_MIRROR_GAUSS) {
        RT_REQ(d->gauss_w > 0.0 && std::isfinite(d->gauss_w), "gauss_w must be finite and > 0");
        RT_REQ(d->A >= 0.0 && d->A < 0.8 * d->gauss_w, "the Gaussian bump needs 0 <= A < 0.8 gauss_w");
        RT_REQ(!d->cloak || (d->H > d->A && d->E > 0.0 && std::isfinite(d->H) && std::isfinite(d->E)),
               "cloak box needs H > A and E > 0 over the Gaussian bump");
        RT_REQ(d->flags == 0, "flags: the Gaussian bump takes no options");
        RT_REQ(d->integrator == RT_RK4 || d->integrator == RT_DP45, "the Gaussian bump needs RT_RK4 or RT_DP45");
    } else {
        const double kA = 2.0 * kPi * d->A / d->Lambda;
        RT_REQ(d->A >= 0.0 && kA < 1.0, "A must satisfy 0 <= 2 pi A / Lambda < 1 (curtate trochoid)");
        RT_REQ(!d->cloak || (d->H > 2.0 * d->A && d->E > 0.0 && std::isfinite(d->H) && std::isfinite(d->E)),
               "cloak box needs H > 2A and E > 0");
    }
    RT_REQ(d->width >= 1 && d->height >= 1 && d->spp >= 1, "width, height and spp must be >= 1");
    RT_REQ(d->centre_line == 0 || d->centre_line == 1, "centre_line must be 0 or 1");
    RT_REQ(d->hfov_deg > 0.0 && d->hfov_deg < 180.0, "hfov_deg must be in (0, 180)");
    RT_REQ(d->cam_dist > 0.0 && std::isfinite(d->cam_dist), "cam_dist must be > 0");
    RT_REQ(d->elev_deg >= -90.0 && d->elev_deg <= 90.0 && std::fabs(std::cos(d->elev_deg * kPi / 180.0)) > 1e-9,
           "elev_deg must be in (-90, 90)");
    RT_REQ(std::isfinite(d->azim_deg), "azim_deg must be finite");
    RT_REQ(d->integrator == RT_RK4 || d->integrator == RT_DP45 || d->integrator == RT_RK4T,
           "integrator must be RT_RK4, RT_DP45 or RT_RK4T");
    RT_REQ(d->precision == RT_FP32 || d->precision == RT_FP64, "precision must be RT_FP32 or RT_FP64");
    RT_REQ(d->h > 0.0 && std::isfinite(d->h), "h must be > 0");
    if (d->integrator == RT_DP45)
        RT_REQ(d->rtol > 0.0 && d->atol > 0.0 && d->h_max > 0.0, "DP45 needs rtol, atol, h_max > 0");
    RT_REQ(d->background == RT_BG_CHECKER || d->background == RT_BG_TEXTURE, "background must be RT_BG_*");
    if (d->background == RT_BG_CHECKER) RT_REQ(d->bg_cell > 0.0, "bg_cell must be > 0");
    else RT_REQ(d->tex && d->tex_size > 0 && d->tex_texel > 0.0, "texture background needs tex, tex_size, tex_texel");
    RT_REQ(d->max_bounces >= 0 && d->max_steps >= 1, "max_bounces >= 0 and max_steps >= 1");
    RT_REQ((d->flags & ~(RT_FLAG_REFERENCED | RT_FLAG_PLATE | RT_FLAG_FRESNEL)) == 0, "flags: unknown bits");
    RT_REQ(!(d->flags & RT_FLAG_PLATE) || (d->mirror == RT_MIRROR_FLAT && d->cloak == 0),
           "flags: the plate lies on the flat mirror (mirror = RT_MIRROR_FLAT, cloak = 0)");
    RT_REQ(!(d->flags & RT_FLAG_PLATE) || (d->H > d->A && d->E > 0.0 && std::isfinite(d->H) && std::isfinite(d->E)),
           "the plate needs H > A and E > 0");
    const double wout = d->centre_line ? 1.0 : (double)d->width;
    RT_REQ((double)d->height * wout * (double)d->spp < 4.0e18, "image too large");
    return RT_OK;
}

static void build_dev(const rt_scene_desc* d, DevScene* s)
{
    memset(s, 0, sizeof *s);
    const double L = d->Lambda;
    s->Lambda = L;
    s->A = d->A / L;
    s->kA = kTwoPi * s->A;
    s->H = d->H / L;
    s->E2 = 0.5 * d->E / L;
    // the box spans y = -A (the grating's troughs) or y = 0 (under the
    // Gaussian bump) to H above that
    const double ybox = d->mirror == RT_MIRROR_GAUSS ? 0.0 : -s->A;
    s->ytop = ybox + s->H;
    s->yrec = ybox + s->H + 1.0;
    const double te = d->elev_deg * kPi / 180.0, ph = d->azim_deg * kPi / 180.0, D = d->cam_dist / L;
    s->C[0] = -D * cos(te) * cos(ph);
    s->C[1] = D * sin(te);
    s->C[2] = -D * cos(te) * sin(ph);
    for (int a = 0; a < 3; ++a) s->f[a] = -s->C[a] / D;
    // r = f x y_hat normalised, u = r x f
    double r[3] = {-s->f[2], 0.0, s->f[0]};
    const double rl = sqrt(r[0] * r[0] + r[2] * r[2]);
    for (int a = 0; a < 3; ++a) s->r[a] = r[a] / rl;
    s->u[0] = s->r[1] * s->f[2] - s->r[2] * s->f[1];
    s->u[1] = s->r[2] * s->f[0] - s->r[0] * s->f[2];
    s->u[2] = s->r[0] * s->f[1] - s->r[1] * s->f[0];
    s->tx = tan(0.5 * d->hfov_deg * kPi / 180.0);
    s->ty = s->tx * (double)d->height / (double)d->width;
    s->fr[0] = s->f[0]; s->fr[1] = -s->f[1]; s->fr[2] = s->f[2];
    s->ur[0] = s->r[1] * s->fr[2] - s->r[2] * s->fr[1];
    s->ur[1] = s->r[2] * s->fr[0] - s->r[0] * s->fr[2];
    s->ur[2] = s->r[0] * s->fr[1] - s->r[1] * s->fr[0];
    for (int a = 0; a < 3; ++a) s->Pb[a] = D * s->fr[a];
    s->cell = d->bg_cell / L;
    s->texel = d->tex_texel / L;
    s->h = d->h / L;
    s->rtol = d->rtol;
    s->atol = d->atol / L;
    s->hmax = d->h_max / L;
    for (int a = 0; a < 3; ++a) { s->col0[a] = (float)d->colour0[a]; s->col1[a] = (float)d->colour1[a]; }
    s->seed = d->seed;
    s->scene_id = d->scene_id;
    s->max_steps = d->max_steps;
    s->mirror = d->mirror;
    s->cloak = d->cloak;
    s->width = d->width;
    s->height = d->height;
    s->wout = d->centre_line ? 1 : d->width;
    s->spp = d->spp;
    int m = (int)floor(sqrt((double)d->spp) + 0.5);
    s->m = (m * m == d->spp) ? m : 0;
    s->centre_line = d->centre_line;
    s->background = d->background;
    s->tex_size = d->tex_size;
    s->integrator = d->integrator;
    s->max_bounces = d->max_bounces;
    s->nwork = (int64_t)d->height * s->wout;
    s->cd.kA = s->kA; s->cd.A = s->A; s->cd.h = s->h; s->cd.ytop = s->ytop; s->cd.E2 = s->E2;
    s->cd.rtol = s->rtol; s->cd.atol = s->atol; s->cd.hmax = s->hmax;
    s->cf.kA = (float)s->kA; s->cf.A = (float)s->A; s->cf.h = (float)s->h; s->cf.ytop = (float)s->ytop;
    s->cf.E2 = (float)s->E2; s->cf.rtol = (float)s->rtol; s->cf.atol = (float)s->atol; s->cf.hmax = (float)s->hmax;
    // FP32 Newton stop on W0: absolute, scaled by kA (|W| < kA in the cloak)
    s->cf.w0tol = (float)(Mth<float>::kRel * s->kA);
    s->cd.w0tol = Mth<double>::kRel * s->kA;
    // index scale of the referenced cloak (n / n_min) and the plate's index
    s->flags = d->flags;
    s->idx_scale = (d->flags & RT_FLAG_REFERENCED) ? 1.0 + s->kA : 1.0;
    s->plate_n = 1.0 + s->kA;
    s->cd.fk = kTwoPi * s->idx_scale * s->idx_scale;
    s->cf.fk = (float)s->cd.fk;
    s->cd.is2 = 1.0 / (s->idx_scale * s->idx_scale);
    s->cf.is2 = (float)s->cd.is2;
    // RK4 moves a ray by |h p + h^2/6 (F1 + F2 + F3)| <= h |p|max + h^2 |F|max / 2 a step,
    // with |p| = n <= s / (1 - kA) (|1 + W0| >= 1 - |W0| > 1 - kA) and
    // |F| = k s^2 |W0| n^4 <= k s^2 kA / (1 - kA)^4; a thousandth of slack on |p|
    {
        const double sc2 = s->idx_scale, q = 1.0 - s->kA;
        const double pmax = 1.001 * sc2 / q, fmax = kTwoPi * sc2 * sc2 * s->kA / (q * q * q * q);
        s->cd.isafe = 1.0 / (s->h * pmax + 0.5 * s->h * s->h * fmax);
        s->cf.isafe = (float)(s->cd.isafe * (1.0 - 1e-6));
        // a full RK4 step's second stage lies h/2 |p| from its start and its
        // fourth at least h/2 |p| - 3/4 h^2 |F| from its third, with
        // |p| >= s / (1 + kA) and |1/(1 + W0)|^2 >= 1 / (1 + kA)^2: if even
        // the shortest of those distances is beyond the continuation's reach
        // (kPredTol, with a factor 4 of margin), those stages always solve
        const double nmin = 1.0 / (1.0 + s->kA), pmin = sc2 * nmin;
        const double d = std::min(0.5 * s->h * pmin, 0.5 * s->h * pmin - 0.75 * s->h * s->h * fmax);
        const double reach = d > 0.0 ? d * d * nmin * nmin : 0.0;
        s->cf.far24 = reach > 4.0 * (double)Mth<float>::kPredTol ? 1.0f : 0.0f;
        s->cd.far24 = reach > 4.0 * Mth<double>::kPredTol ? 1.0 : 0.0;
    }
    s->cd.ybot = ((d->flags & RT_FLAG_PLATE) || d->mirror == RT_MIRROR_GAUSS) ? 0.0 : -s->A;
    s->cf.ybot = (float)s->cd.ybot;
    // Gaussian bump: width, 1/width, k h, h/width, the Newton stop on W and
    // the largest Newton step (a quarter width in w)
    if (d->mirror == RT_MIRROR_GAUSS) {
        const double gw = d->gauss_w / L;
        s->cd.gw = gw; s->cd.igw = 1.0 / gw; s->cd.gkh = kTwoPi * s->A; s->cd.gq = s->A / gw;
        s->cd.gtol = 1.6e-29;
        s->cd.gcap2 = (0.25 * kTwoPi * gw) * (0.25 * kTwoPi * gw);
        s->cf.gw = (float)gw; s->cf.igw = (float)(1.0 / gw); s->cf.gkh = (float)s->cd.gkh;
        s->cf.gq = (float)s->cd.gq; s->cf.gtol = 1e-12f; s->cf.gcap2 = (float)s->cd.gcap2;
        // continuation over |dz| <= 6e-5 w_b (FP32) or 3e-9 w_b (FP64): the terms
        // it leaves out, of second order in |dz| / w_b, stay below the precision
        s->cf.gpred = 4e-9f;
        s->cd.gpred = 0.0;                    // FP64 solves at every point
    }
    for (int a = 0; a < 3; ++a) {
        s->ad.fr[a] = s->fr[a]; s->ad.ur[a] = s->ur[a]; s->ad.r[a] = s->r[a]; s->ad.Pb[a] = s->Pb[a];
        s->af.fr[a] = (float)s->fr[a]; s->af.ur[a] = (float)s->ur[a]; s->af.r[a] = (float)s->r[a];
        s->af.Pb[a] = (float)s->Pb[a];
    }
    s->ad.inv_cell = s->cell > 0.0 ? 1.0 / s->cell : 0.0;
    s->ad.inv_texel = s->texel > 0.0 ? 1.0 / s->texel : 0.0;
    s->af.inv_cell = (float)s->ad.inv_cell;
    s->af.inv_texel = (float)s->ad.inv_texel;
    s->ymirror = d->mirror != RT_MIRROR_FLAT ? s->A : 0.0;
    s->box_lo[0] = -s->E2; s->box_lo[1] = s->cd.ybot; s->box_lo[2] = -s->E2;
    s->box_hi[0] = s->E2; s->box_hi[1] = s->ytop; s->box_hi[2] = s->E2;
    for (int a = 0; a < 3; ++a) {
        s->cam_lo[a] = (float)(s->box_lo[a] - s->C[a]);
        s->cam_hi[a] = (float)(s->box_hi[a] - s->C[a]);
    }
    s->cam_ym = (float)(s->ymirror - s->C[1]);
    s->inv_m = s->m > 0 ? 1.0 / s->m : 0.0;
    s->two_over_w = 2.0 / (double)d->width;
    s->two_over_h = 2.0 / (double)d->height;
}

namespace grt {

void build_scene_table(const rt_scene_desc* d, DevScene* s) { build_dev(d, s); }

int scene_info(rt_scene* s, DevScene* dev, int* precision, int* integrator, int* device)
{
    if (!s) { set_error("scene is NULL"); return RT_EINVAL; }
    *dev = s->dev;
    *precision = s->desc.precision;
    *integrator = s->desc.integrator;
    *device = s->device;
    return RT_OK;
}

void counters_to_stats(const unsigned long long* c, rt_stats* out)
{
    out->rays = c[1];
    out->steps = c[2];
    out->evals = c[3];
    out->newton = c[4];
    out->events = c[5];
    out->fp64_refine = c[6];
    for (int q = 0; q < 5; ++q) out->status[q] = c[7 + q];
    for (int q = 0; q < 4; ++q) out->profile[q] = c[12 + q];
    out->sched_timeouts = c[16];
}

}  // namespace grt

extern "C" {

const char* rt_last_error(void) { return g_err; }

int rt_validate_desc(const rt_scene_desc* desc)
{
    g_err[0] = 0;
    return validate(desc);
}

const char* rt_version(void) { return "gratingrt 0.1 (sm_103a)"; }

int rt_create_scene(const rt_scene_desc* desc, rt_scene** out)
{
    g_err[0] = 0;
    RT_REQ(out, "out is NULL");
    *out = nullptr;
    int rc = validate(desc);
    if (rc) return rc;
    int dev;
    rc = current_device(&dev);
    if (rc) return rc;
    rt_scene* s = (rt_scene*)calloc(1, sizeof(rt_scene));
    if (!s) { set_error("host allocation failed"); return RT_ENOMEM; }
    s->desc = *desc;
    s->desc.tex = nullptr;
    s->device = dev;
    build_dev(desc, &s->dev);
    int bps = 0;
    s->variant = kDefaultVariant;
    s->min_active = default_min_active(desc->precision, render_mode(*desc));
    s->wait = WaitLimit{kDefaultWaitSpin, 0};
    cudaError_t e = desc->mirror == RT_MIRROR_GAUSS ? gauss_upload() : cudaSuccess;
    if (e == cudaSuccess) e = render_occupancy(desc->precision, render_mode(*desc), s->variant, desc->flags != 0, &bps);
    int nsm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    s->nsm = nsm;
    if (e == cudaSuccess && desc->background == RT_BG_TEXTURE) {
        const size_t bytes = (size_t)desc->tex_size * desc->tex_size * sizeof(float);
        e = cudaMalloc(&s->d_tex, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(s->d_tex, desc->tex, bytes, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->d_counters, kCounters * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(s->d_counters, 0, kCounters * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        set_error("rt_create_scene: %s", cudaGetErrorString(e));
        rt_destroy_scene(s);
        return e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA;
    }
    s->dev.tex = s->d_tex;
    s->grid = (bps > 0 ? bps : 1) * nsm;
    *out = s;
    return RT_OK;
}

void rt_destroy_scene(rt_scene* s)
{
    if (!s) return;
    if (s->done) cudaEventSynchronize(s->done);
    if (s->d_tex) cudaFree(s->d_tex);
    if (s->d_counters) cudaFree(s->d_counters);
    if (s->d_host_rgb) cudaFree(s->d_host_rgb);
    if (s->d_host_rgb8) cudaFree(s->d_host_rgb8);
    if (s->d_samp) cudaFree(s->d_samp);
    if (s->d_pcnt) cudaFree(s->d_pcnt);
    if (s->d_branch) cudaFree(s->d_branch);
    if (s->done) cudaEventDestroy(s->done);
    free(s);
}

static int render_common(rt_scene* s, const int64_t* d_pix, int64_t nwork, float* d_rgb, uint8_t* d_rgb8,
                         rt_ray_record* d_rec, void* stream)
{
    RT_REQ(s, "scene is NULL");
    RT_REQ(d_rgb || nwork == 0, "d_rgb is NULL");
    int dev;
    int rc = current_device(&dev);
    if (rc) return rc;
    RT_REQ(dev == s->device, "scene was created on device %d, current device is %d", s->device, dev);
    cudaStream_t st = (cudaStream_t)stream;
    DevScene sc = s->dev;
    sc.pix_list = d_pix;
    sc.nwork = nwork;
    RT_CK(cudaMemsetAsync(s->d_counters, 0, kCounters * sizeof(unsigned long long), st));
    RT_REQ(s->desc.flags == 0 || s->variant == kVariantWave,
           "scene options (RT_FLAG_*) are rendered by the wavefront loop (variant %d) only", kVariantWave);
    SampleScratch ss = {nullptr, nullptr, nullptr};
    if (nwork > 0 && (s->desc.flags & RT_FLAG_FRESNEL)) {
        const size_t bytes = branch_queue_bytes(s->desc.precision, s->desc.integrator, s->grid);
        if (bytes > s->branch_cap) {
            RT_CK(cudaStreamWaitEvent(st, s->done, 0));
            if (s->d_branch) RT_CK(cudaFreeAsync(s->d_branch, st));
            s->d_branch = nullptr;
            s->branch_cap = 0;
            RT_CK(cudaMallocAsync(&s->d_branch, bytes, st));
            s->branch_cap = bytes;
        }
        ss.br = s->d_branch;
    }
    if (nwork > 0 && s->variant == kVariantWave && sc.spp > 1) {
        // the wavefront loop traces the samples of a pixel at the same time
        const int64_t ns = nwork * sc.spp;
        if (ns > s->samp_cap || nwork > s->pix_cap) {
            RT_CK(cudaStreamWaitEvent(st, s->done, 0));      // the last render of this scene is done with them
            if (s->d_samp) RT_CK(cudaFreeAsync(s->d_samp, st));
            if (s->d_pcnt) RT_CK(cudaFreeAsync(s->d_pcnt, st));
            s->d_samp = nullptr;
            s->d_pcnt = nullptr;
            s->samp_cap = s->pix_cap = 0;
            RT_CK(cudaMallocAsync((void**)&s->d_samp, (size_t)nwork * (size_t)col_block_bytes(sc.spp), st));
            RT_CK(cudaMallocAsync((void**)&s->d_pcnt, (size_t)nwork * kScratchBytesPerPixel, st));
            s->samp_cap = ns;
            s->pix_cap = nwork;
        }
        RT_CK(cudaMemsetAsync(s->d_pcnt, 0, (size_t)nwork * kScratchBytesPerPixel, st));
        ss.col = s->d_samp;
        ss.cnt = s->d_pcnt;
    }
    if (nwork > 0)
        RT_CK(launch_render(sc, s->desc.precision, s->variant, s->min_active, d_rgb, d_rgb8, d_rec, s->d_counters,
                            s->grid, ss, s->wait, st));
    RT_CK(cudaEventRecord(s->done, st));
    s->rendered = true;
    return RT_OK;
}

int rt_render(rt_scene* s, float* d_rgb, uint8_t* d_rgb8, rt_ray_record* d_rec, void* stream)
{
    g_err[0] = 0;
    RT_REQ(s, "scene is NULL");
    return render_common(s, nullptr, s->dev.nwork, d_rgb, d_rgb8, d_rec, stream);
}

int rt_render_pixels(rt_scene* s, const int64_t* d_pix, int64_t npix, float* d_rgb, rt_ray_record* d_rec,
                     void* stream)
{
    g_err[0] = 0;
    RT_REQ(npix >= 0, "npix must be >= 0");
    RT_REQ(npix == 0 || d_pix, "d_pix is NULL");
    return render_common(s, d_pix, npix, d_rgb, nullptr, d_rec, stream);
}

int rt_render_host(rt_scene* s, float* h_rgb, uint8_t* h_rgb8, void* stream)
{
    g_err[0] = 0;
    RT_REQ(s && h_rgb, "scene and h_rgb must not be NULL");
    const size_t n = (size_t)s->dev.nwork * 3;
    if (!s->d_host_rgb) RT_CK(cudaMalloc(&s->d_host_rgb, n * sizeof(float)));
    if (h_rgb8 && !s->d_host_rgb8) RT_CK(cudaMalloc(&s->d_host_rgb8, n));
    cudaStream_t st = (cudaStream_t)stream;
    int rc = render_common(s, nullptr, s->dev.nwork, s->d_host_rgb, h_rgb8 ? s->d_host_rgb8 : nullptr, nullptr,
                           stream);
    if (rc) return rc;
    RT_CK(cudaMemcpyAsync(h_rgb, s->d_host_rgb, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (h_rgb8) RT_CK(cudaMemcpyAsync(h_rgb8, s->d_host_rgb8, n, cudaMemcpyDeviceToHost, st));
    RT_CK(cudaStreamSynchronize(st));
    return RT_OK;
}

int rt_scene_stats(rt_scene* s, rt_stats* out)
{
    g_err[0] = 0;
    RT_REQ(s && out, "scene and out must not be NULL");
    unsigned long long c[kCounters];
    RT_CK(cudaEventSynchronize(s->done));
    RT_CK(cudaMemcpy(c, s->d_counters, sizeof c, cudaMemcpyDeviceToHost));
    counters_to_stats(c, out);
    if (out->sched_timeouts) {
        set_error("the last render of this scene gave up %llu bounded waits of its work queues; its image is "
                  "incomplete", (unsigned long long)out->sched_timeouts);
        return RT_ETIMEDOUT;
    }
    return RT_OK;
}

int rt_scene_autotune(rt_scene* s, float* d_rgb, int32_t trials, void* stream, int32_t* variant_out,
                      int32_t* min_active_out)
{
    g_err[0] = 0;
    RT_REQ(s && d_rgb, "scene and d_rgb must not be NULL");
    RT_REQ(trials >= 1 && trials <= 64, "trials must be 1..64");
    const rt_scene_desc& d = s->desc;
    // scenes of one class share a configuration: precision, integrator,
    // cloak and the power of two of the number of samples
    const double samples = (double)s->dev.nwork * d.spp;
    char key[160];
    snprintf(key, sizeof key, "scene/p%d/i%d/c%d/m%d/f%d/log2n%d", d.precision, d.integrator, d.cloak, d.mirror, d.flags,
             (int)floor(log2(samples > 1.0 ? samples : 1.0)));
    int v = kDefaultVariant, m = default_min_active(d.precision, render_mode(d));
    if (!tune_lookup(key, &v, &m)) {
        const int cand[] = {12, 16, 20, 24, 28};
        cudaStream_t st = (cudaStream_t)stream;
        cudaEvent_t e0, e1;
        RT_CK(cudaEventCreate(&e0));
        RT_CK(cudaEventCreate(&e1));
        float best = 1e30f;
        int rc = RT_OK;
        for (int var = 0; var < kVariants && rc == RT_OK; ++var) {
            if (!variant_compiled(d.precision, render_mode(d), var)) continue;
            if (d.flags != 0 && var != kVariantWave) continue;
            for (int c : cand) {
                rc = rt_scene_set_launch(s, var, c);
                if (rc != RT_OK) break;
                rc = render_common(s, nullptr, s->dev.nwork, d_rgb, nullptr, nullptr, stream);   // warm-up
                float t[64];
                for (int k = 0; rc == RT_OK && k < trials; ++k) {
                    cudaEventRecord(e0, st);
                    rc = render_common(s, nullptr, s->dev.nwork, d_rgb, nullptr, nullptr, stream);
                    cudaEventRecord(e1, st);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&t[k], e0, e1);
                }
                if (rc != RT_OK) break;
                std::sort(t, t + trials);
                if (t[trials / 2] < best) { best = t[trials / 2]; v = var; m = c; }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc != RT_OK) return rc;
        tune_record(key, v, m);
    }
    const int rc = rt_scene_set_launch(s, v, m);
    if (rc != RT_OK) return rc;
    if (variant_out) *variant_out = v;
    if (min_active_out) *min_active_out = m;
    return RT_OK;
}

int rt_scene_set_launch(rt_scene* s, int32_t variant, int32_t min_active)
{
    g_err[0] = 0;
    RT_REQ(s, "scene is NULL");
    RT_REQ(variant >= -1 && variant < kVariants, "variant must be -1 (keep) or 0..%d", kVariants - 1);
    RT_REQ(variant < 0 || variant_compiled(s->desc.precision, render_mode(s->desc), variant),
           "variant %d is not compiled for this precision, integrator and mirror", variant);
    RT_REQ(variant < 0 || variant == kVariantWave || s->desc.flags == 0,
           "scene options (RT_FLAG_*) are rendered by the wavefront loop (variant %d) only", kVariantWave);
    RT_REQ(min_active == 0 || (min_active >= 1 && min_active <= 32), "min_active must be 0 (keep) or 1..32");
    if (variant >= 0 && variant != s->variant) {
        int bps = 0;
        RT_CK(render_occupancy(s->desc.precision, render_mode(s->desc), variant, s->desc.flags != 0, &bps));
        RT_REQ(bps > 0, "variant %d does not fit on this device", variant);
        s->variant = variant;
        s->grid = bps * s->nsm;
    }
    if (min_active > 0) s->min_active = min_active;
    return RT_OK;
}

int rt_scene_set_wait_limit(rt_scene* s, int32_t spin_limit, int32_t hold_lock)
{
    g_err[0] = 0;
    RT_REQ(s, "scene is NULL");
    RT_REQ(spin_limit >= 0 && spin_limit <= kDefaultWaitSpin, "spin_limit must be 0 (default) or 1..%d",
           kDefaultWaitSpin);
    s->wait.spin = spin_limit ? spin_limit : kDefaultWaitSpin;
    s->wait.hold = hold_lock ? 1 : 0;
    return RT_OK;
}

int rt_scene_get_launch(rt_scene* s, int32_t* variant, int32_t* min_active, int32_t* grid)
{
    g_err[0] = 0;
    RT_REQ(s, "scene is NULL");
    if (variant) *variant = s->variant;
    if (min_active) *min_active = s->min_active;
    if (grid) *grid = s->grid;
    return RT_OK;
}

int rt_xcorr(const float* d_f, const float* d_g, int32_t height, int32_t width, int32_t channels,
             const double* fov_deg, int32_t n_fov, double hfov_deg, double* d_out, void* stream)
{
    g_err[0] = 0;
    RT_REQ(d_f && d_g && d_out && fov_deg, "null pointer argument");
    RT_REQ(height >= 1 && width >= 1, "height and width must be >= 1");
    RT_REQ(channels >= 1 && channels <= 4, "channels must be 1..4");
    RT_REQ(n_fov >= 1 && n_fov <= kMaxWindows, "n_fov must be 1..%d", kMaxWindows);
    RT_REQ(hfov_deg > 0.0 && hfov_deg < 180.0, "hfov_deg must be in (0, 180)");
    for (int q = 0; q < n_fov; ++q) RT_REQ(fov_deg[q] >= 0.0, "fov_deg must be >= 0");
    int dev;
    int rc = current_device(&dev);
    if (rc) return rc;
    Windows win;
    fov_windows(width, hfov_deg, fov_deg, n_fov, &win);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = xcorr_scratch_bytes(height, width, channels);
    void* partial = nullptr;
    if (bytes) RT_CK(cudaMallocAsync(&partial, bytes, st));
    cudaError_t e = launch_xcorr(d_f, d_g, height, width, channels, win, partial, d_out, st);
    cudaError_t e2 = bytes ? cudaFreeAsync(partial, st) : cudaSuccess;
    RT_CK(e);
    RT_CK(e2);
    return RT_OK;
}

int rt_eval_medium(int32_t precision, double Lambda, double A, const double* d_xy, int64_t npoints,
                   double* d_out, void* stream)
{
    g_err[0] = 0;
    RT_REQ(precision == RT_FP32 || precision == RT_FP64, "precision must be RT_FP32 or RT_FP64");
    RT_REQ(Lambda > 0.0 && A >= 0.0 && 2.0 * kPi * A / Lambda < 1.0, "need Lambda > 0 and 0 <= kA < 1");
    RT_REQ(npoints >= 0 && (npoints == 0 || (d_xy && d_out)), "null pointer argument");
    int dev;
    int rc = current_device(&dev);
    if (rc) return rc;
    RT_CK(launch_medium(precision, kTwoPi * A / Lambda, Lambda, d_xy, npoints, d_out, (cudaStream_t)stream));
    return RT_OK;
}

}  // extern "C"
