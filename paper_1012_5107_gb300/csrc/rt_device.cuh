// rt_device.cuh -- device-side arithmetic of the grating-cloak ray tracer.
//
// Units: every length is divided by the grating period Lambda, so k = 2 pi.
// The abscissa x is carried as an integer cell plus a fraction X in
// [-1/2, 1/2): the index (Eq. 1) is periodic in x, so the W0 solve, the
// force and the trochoid see only X and keep full FP32 resolution however
// far the ray is from the origin.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace grt {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.28318530717958647692;
constexpr double kInvTwoPi = 0.15915494309189533577;
constexpr double kLog2e = 1.44269504088896340736;

// ------------------------------------------------------------------------
// Scene constants (normalised units) passed by value to every kernel.  The
// per-step constants are also stored in the precision of the path, so the
// inner loop reads them from the constant bank without conversions (a
// double-to-float conversion runs on the FP64 pipe).
// ------------------------------------------------------------------------
template <class R>
struct StepConst {
    R kA, A, h, ytop, E2;
    R rtol, atol, hmax;
    R w0tol;     // FP32: Newton on W0 stops when |dW|^2 <= w0tol
    R fk;        // force factor k s^2 (s: index scale of the cloak, 1 unless referenced)
    R ybot;      // bottom of the box: -A (cloak) or 0 (plate on the flat mirror)
    R is2;       // 1/s^2: the time form's acceleration F/n^2 with F scaled by s^2 and n^2 = s^2 |r|^2
    // Gaussian bump (RT_MIRROR_GAUSS): width w_b, 1/w_b, k h, h/w_b, Newton
    // stop |dW|^2 <= gtol, and the largest Newton step |dW|^2 <= gcap2
    R gw, igw, gkh, gq, gtol, gcap2;
    R gpred;     // Gaussian bump: a step continues the medium when |dz|^2 / w_b^2 <= gpred
    R isafe;     // RK4 in the grating cloak: 1 / (the largest move of one step), see box_step_into
    R far24;     // RK4 in the grating cloak: 1 if a full step's second and fourth stage points always lie too
                 // far from the previous point for W0 to be continued without a solve (see med_stage)
};

// Hot counters of a lane, kept in registers.
struct LaneStats {
    uint32_t steps, evals, newton, refine;
};

// Constants of the straight segments to the background, in the path's precision.
template <class R>
struct AirConst {
    R fr[3], ur[3], r[3], Pb[3];
    R inv_cell, inv_texel;
};

struct DevScene {
    StepConst<float> cf;
    StepConst<double> cd;
    AirConst<float> af;
    AirConst<double> ad;
    double ymirror;                         // the mirror cannot be met above this height
    double box_lo[3], box_hi[3];            // cloak box
    float cam_lo[3], cam_hi[3], cam_ym;     // box bounds and ymirror relative to the camera, FP32
    double inv_m, two_over_w, two_over_h;   // sampling constants
    double A, kA, H, E2, ytop, yrec;       // grating, cloak box (E2 = E/2), record plane
    double C[3], f[3], r[3], u[3];         // camera position and basis
    double tx, ty;                          // tangent of the half fields of view
    double fr[3], ur[3], Pb[3];             // background plane frame
    double cell, texel;                     // checkerboard cell, texel size
    double h, rtol, atol, hmax;             // integrator
    double Lambda;                          // world scale of outputs
    float col0[3], col1[3];
    const float* tex;
    const int64_t* pix_list;                // optional subset of pixels
    uint64_t seed, scene_id;
    int64_t max_steps;
    int64_t nwork;                          // pixels to render
    int64_t col_base;                       // first float of the scene's pixel colour blocks in the launch scratch
    int mirror, cloak, width, height, wout, spp, m, centre_line;
    int background, tex_size, integrator, max_bounces;
    int flags;                              // RT_FLAG_*
    double idx_scale;                       // index scale inside the cloak (1 + kA when referenced)
    double plate_n;                         // index of the dielectric plate (1 + kA)
};

// ------------------------------------------------------------------------
// Precision back ends.  FP32 uses the SFU (MUFU) approximations; FP64 the
// CUDA math library.
// ------------------------------------------------------------------------
template <class R> struct Mth;

template <> struct Mth<float> {
    static __device__ __forceinline__ float rcp(float x) {
        float y;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ float ex2(float x) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ float lg2(float x) {
        float y;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    // sin and cos of 2 pi a for |a| <= 1/2
    static __device__ __forceinline__ void sincos2pi(float a, float& s, float& c) {
        __sincosf(6.28318530717958647692f * a, &s, &c);
    }
    static __device__ __forceinline__ void sincos(float a, float& s, float& c) { __sincosf(a, &s, &c); }
    static __device__ __forceinline__ float rint_(float x) { return rintf(x); }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    // Newton on W0 stops when |dW|^2 <= kRel kA: the next step would change W
    // by about |dW|^2 |W| / 2, below the FP32 resolution of the force
    static constexpr float kRel = 3.6e-8f;
    // the first-order continuation of W0 over dz is kept without a Newton step
    // when its error k^2 |W| n^3 |dz|^2 / 2 is below 1e-8 |W|
    static constexpr float kPredTol = 5e-10f;
    static constexpr int kMaxIt = 16;
    static constexpr float kEventTol = 2e-9f;   // |g| at a located event (units of Lambda)
    static constexpr int kEventIt = 40;
    static constexpr float kRehit = 1e-5f;      // a ray leaving a surface cannot meet it again closer
    static constexpr float kEps = 1.1920929e-7f;
};

template <> struct Mth<double> {
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double ex2(double x) { return exp2(x); }
    static __device__ __forceinline__ void sincos2pi(double a, double& s, double& c) { sincospi(2.0 * a, &s, &c); }
    static __device__ __forceinline__ void sincos(double a, double& s, double& c) { ::sincos(a, &s, &c); }
    static __device__ __forceinline__ double rint_(double x) { return rint(x); }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static constexpr double kRel = 6e-17;
    static constexpr double kPredTol = 2.5e-18;
    static constexpr int kMaxIt = 40;
    static constexpr double kEventTol = 1e-14;
    static constexpr int kEventIt = 100;
    static constexpr double kRehit = 1e-9;
    static constexpr double kEps = 2.220446049250313e-16;
};

// FP64 reciprocal and reciprocal square root for the few FP64 steps of the
// FP32 path (interfaces, reflections): an FP32 seed from the SFU refined by
// two Newton-Raphson steps in FP64 -- y <- y (2 - x y) and
// y <- y (3 - x y^2) / 2, each squaring the relative error (2^-23 -> 2^-46
// -> below the FP64 rounding) -- instead of a full-precision FP64 division
// or square root, which take many more operations on the FP64 pipe.
// Arguments are positive and within the FP32 range.
__device__ __forceinline__ double recip_nr(double x)
{
    float s;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"((float)x));
    double y = (double)s;
    y = y * fma(-x, y, 2.0);
    y = y * fma(-x, y, 2.0);
    return y;
}

__device__ __forceinline__ double rsqrt_nr(double x)
{
    double y = (double)rsqrtf((float)x);
    y = y * fma(-0.5 * x * y, y, 1.5);
    y = y * fma(-0.5 * x * y, y, 1.5);
    return y;
}

// ------------------------------------------------------------------------
// Packed FP32 pairs: sm_100 and later issue two FP32 fused multiply-adds,
// adds or multiplies of a thread in one instruction (FFMA2, FADD2, FMUL2).
// The FP32 path keeps (x, y) components and real and imaginary parts as such
// pairs where its arithmetic pairs up; per component every result is the
// scalar operation's in round-to-nearest (a - b is taken as fma(b, -1, a),
// which is exact before its one rounding).
__device__ __forceinline__ float2 p2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 p2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
// compensated (Kahan) sum of both components
__device__ __forceinline__ void kahan2(float2& sum, float2& comp, float2 inc)
{
    const float2 yv = sub2(inc, comp);
    const float2 t = add2(sum, yv);
    comp = sub2(sub2(t, sum), yv);
    sum = t;
}

// Lambert W0 of zeta = -kA exp(i k z) (Eq. 1 with c = iA, Eq. 13).
//
// W e^W = zeta is solved in the equivalent form
//     g(W) = W + kA exp(-(W - i k z)) = 0,
// whose Newton constant g''/2g' = -W/(2(1+W)) is small for the cloak's
// |W| < kA < 1, by Newton steps with the derivative 1 + W of the current
// iterate (g'(W) = 1 + W at the root).  Each step costs one exp, one
// sin/cos pair and one reciprocal.
// Stop: FP32 when |dW|^2 <= tol (tol = 3.6e-8 kA: the next step would move W
// by about |dW|^2 |W|/2, below the FP32 resolution of the force); FP64 when
// |dW|^2 |1/(1+W)| <= 1e-16, so that the error left after the step, about
// |dW|^2 |W| |1/(1+W)| / 2 by the Newton constant, is below 5e-17 |W|.  On return (wr, wi) = W and (rr, ri) = 1/(1+W): a fresh
// reciprocal in FP32, the one of the last iterate corrected to second order
// in the last step in FP64 (where a division costs more than the correction).
// The result is the number of Newton steps.
// ------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void newton_w0(R kA, R X, R y, R& wr, R& wi, R& rr, R& ri, R& dr, R& di)
{
    const R L2E = R(kLog2e);
    const R KL2E = R(kTwoPi * kLog2e);
    const R I2PI = R(kInvTwoPi);
    const R ar = R(1) + wr, ai = wi;
    const R inv = Mth<R>::rcp(ar * ar + ai * ai);
    rr = ar * inv;
    ri = -ai * inv;
    // q = kA exp(-(Re W + k y)) (cos(k X - Im W) + i sin(k X - Im W))
    const R e = kA * Mth<R>::ex2(-(wr * L2E) - y * KL2E);
    R a = X - wi * I2PI;
    a -= Mth<R>::rint_(a);
    R s, c;
    Mth<R>::sincos2pi(a, s, c);
    const R nr = wr + e * c, ni = wi + e * s;           // g(W)
    dr = nr * rr - ni * ri;                              // dW = g(W)/(1+W)
    di = nr * ri + ni * rr;
    wr -= dr;
    wi -= di;
}

template <class R>
__device__ __forceinline__ bool w0_converged(R tol, R rr, R ri, R dr, R di)
{
    const R d2 = dr * dr + di * di;
    if constexpr (sizeof(R) == 4) return d2 <= tol;
    else return d2 * d2 * (rr * rr + ri * ri) <= R(1e-32);
}

template <class R>
__device__ __forceinline__ int w0_solve(R kA, R tol, R X, R y, R& wr, R& wi, R& rr, R& ri)
{
    R dr, di;
    int it = 0;
    for (;;) {
        newton_w0(kA, X, y, wr, wi, rr, ri, dr, di);
        ++it;
        if (w0_converged(tol, rr, ri, dr, di) || it >= Mth<R>::kMaxIt) break;
    }
    if constexpr (sizeof(R) == 4) {
        const R ar = R(1) + wr, ai = wi;
        const R inv = Mth<R>::rcp(ar * ar + ai * ai);
        rr = ar * inv;
        ri = -ai * inv;
    } else {
        const R tr = rr * dr - ri * di, ti = rr * di + ri * dr;   // r dW
        const R nrr = rr + (rr * tr - ri * ti), nri = ri + (rr * ti + ri * tr);
        rr = nrr;
        ri = nri;
    }
    return it;
}

// First-order continuation of W along a displacement (dx, dy):
// W' = dW/dz = i k W / (1 + W) = i k W r.
// Third-order continuation (the guess of an FP64 solve, which then takes one
// Newton step where the first-order guess needed two): with u = W r and
// t = i k r dz,  W(z + dz) = W (1 + t + r t^2/2 + r t^3 (1 - 3u)/6), from
// W' = i k u, W'' = -k^2 u r^2 and W''' = -i k^3 u r^3 (1 - 3u).
template <class R>
__device__ __forceinline__ void w0_predict3(R& wr, R& wi, R rr, R ri, R dx, R dy)
{
    const R k = R(kTwoPi);
    const R ar = -k * dy, ai = k * dx;                               // i k dz
    const R tr = rr * ar - ri * ai, ti = rr * ai + ri * ar;          // t
    const R t2r = tr * tr - ti * ti, t2i = R(2) * tr * ti;
    const R t3r = t2r * tr - t2i * ti, t3i = t2r * ti + t2i * tr;
    const R ur = wr * rr - wi * ri, ui = wr * ri + wi * rr;          // u = W r
    const R vr = R(1) - R(3) * ur, vi = R(-3) * ui;                  // 1 - 3u
    const R mr = t3r * vr - t3i * vi, mi = t3r * vi + t3i * vr;      // t^3 (1 - 3u)
    const R sr = R(0.5) * t2r + mr * R(1.0 / 6.0), si = R(0.5) * t2i + mi * R(1.0 / 6.0);
    const R qr = tr + (rr * sr - ri * si), qi = ti + (rr * si + ri * sr);   // t + r (t^2/2 + t^3 (1 - 3u)/6)
    const R dwr = wr * qr - wi * qi, dwi = wr * qi + wi * qr;
    wr += dwr;
    wi += dwi;
}

template <class R>
__device__ __forceinline__ void w0_predict(R& wr, R& wi, R rr, R ri, R dx, R dy)
{
    const R k = R(kTwoPi);
    const R pr = wr * rr - wi * ri, pi = wr * ri + wi * rr;   // W r
    wr += k * (-pi * dx - pr * dy);
    wi += k * (pr * dx - pi * dy);
}

// Ray force F = grad(n^2)/2 = n grad n (Eq. 12 times n) in the Hamiltonian
// parameter: F = k n^2 (Im(W r^2), Re(W r^2)) with r = 1/(1+W), n^2 = |r|^2;
// an index scaled by s inside the cloak (the referenced cloak, n / n_min)
// scales the force by s^2: fk = k s^2.
template <class R>
__device__ __forceinline__ void ray_force(R wr, R wi, R rr, R ri, R fk, R& Fx, R& Fy)
{
    const R n2 = rr * rr + ri * ri;
    const R r2r = rr * rr - ri * ri, r2i = R(2) * rr * ri;
    const R gr = wr * r2r - wi * r2i, gi = wr * r2i + wi * r2r;
    const R s = fk * n2;
    Fx = s * gi;
    Fy = s * gr;
}

// ------------------------------------------------------------------------
// Trochoid grating (Eq. 2): x = xi - A sin(k xi), y = A cos(k xi).
// ------------------------------------------------------------------------
// Kepler's equation E - e sin E = M for the phase E = k xi given M = k x,
// e = kA < 1, by Newton's method from E = M + e sin M.  M is reduced to
// [-pi, pi] by the caller.
template <class R>
__device__ __forceinline__ R kepler(R M, R e)
{
    R s, c;
    Mth<R>::sincos(M, s, c);
    R E = M + e * s;
    for (int it = 0; it < (sizeof(R) == 4 ? 6 : 12); ++it) {
        Mth<R>::sincos(E, s, c);
        const R f = E - e * s - M;
        const R dE = f / (R(1) - e * c);
        E -= dE;
        if (fabs(dE) <= R(4) * Mth<R>::kEps * (R(1) + fabs(E))) break;
    }
    return E;
}

// Phase E and surface height y_s at cell-local abscissa X.
template <class R>
__device__ __forceinline__ R trochoid_phase(R X, R kA)
{
    R a = X - Mth<R>::rint_(X);
    return kepler(R(kTwoPi) * a, kA);
}

// ------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): output m of the generator seeded
// with `seed` is mix(seed + m * golden).
// ------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t m)
{
    uint64_t z = seed + m * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform24(uint64_t seed, uint64_t m)
{
    return (double)(splitmix64(seed, m) >> 40) * (1.0 / 16777216.0);
}

template <class R> __device__ __forceinline__ const AirConst<R>& air_const(const DevScene& s);
template <> __device__ __forceinline__ const AirConst<float>& air_const<float>(const DevScene& s) { return s.af; }
template <> __device__ __forceinline__ const AirConst<double>& air_const<double>(const DevScene& s) { return s.ad; }

// Illinois (modified regula falsi) on [a, b] with fa > 0 >= fb; returns the
// last point evaluated.
template <class R, class F>
__device__ __forceinline__ R illinois_root(F& f, R a, R fa, R b, R fb)
{
    int side = 0;
    R c = b;
    for (int it = 0; it < Mth<R>::kEventIt; ++it) {
        c = b - fb * (b - a) / (fb - fa);
        if (!(c > a && c < b)) c = R(0.5) * (a + b);
        const R fc = f(c);
        if (fabs(fc) <= Mth<R>::kEventTol) return c;
        if (fc < R(0)) {
            b = c; fb = fc;
            if (side == -1) fa *= R(0.5);
            side = -1;
        } else {
            a = c; fa = fc;
            if (side == 1) fb *= R(0.5);
            side = 1;
        }
        if (b - a <= R(4) * Mth<R>::kEps * (R(1) + fabs(b))) return c;
    }
    return c;
}

template <class R> __device__ __forceinline__ const StepConst<R>& step_const(const DevScene& s);
template <> __device__ __forceinline__ const StepConst<float>& step_const<float>(const DevScene& s) { return s.cf; }
template <> __device__ __forceinline__ const StepConst<double>& step_const<double>(const DevScene& s) { return s.cd; }

}  // namespace grt
