// rt_trace.cuh -- the render kernel of the grating-cloak ray tracer,
// templated on the arithmetic type R (float or double).
//
// Structure.  One lane owns one pixel at a time and traces its samples one
// after the other, so the per-pixel sum has a fixed order.  The kernel is
// persistent and alternates two phases per warp:
//   * the integration loop advances every lane whose ray is inside the cloak
//     by one RK4 step per iteration, as long as enough lanes of the warp are
//     inside; a step that crosses a surface, hits the step cap or goes
//     non-finite only marks the lane;
//   * the service pass lets every other lane catch up: locate and act on the
//     marked events, take new pixels (one atomic per group of lanes), start
//     samples, trace straight segments in air and finish samples.
// The integration loop touches only the ray state in registers; everything
// else a lane owns lives in shared memory.
//
// Paper: index Eq. 1, its gradient Eq. 12 and W0 (Eq. 13) in Sec. 2-3; the
// Newtonian ray equation Eq. 11 (Sec. 3), integrated in the Hamiltonian
// parameter tau (dr/dtau = p, dp/dtau = grad(n^2)/2, |p| = n), which traces
// the same curves; Snell's law at the cloak boundary (Sec. 3); the trochoid
// grating of Eq. 2 (Sec. 2); the camera of Sec. 4.
//
// Precision.  FP32 keeps the abscissa as cell + fraction and sums the state
// with compensation; the camera ray is set up in FP64 (a few operations per
// sample) because its lever arm from the camera to the scene would otherwise
// dominate the error.  Nothing else in the FP32 kernel uses the FP64 pipe,
// whose rate on this GPU is 1/64 of FP32.
#pragma once

#include <cfloat>
#include <cmath>
#include <cstdint>

#include "rt.h"
#include "rt_device.cuh"
#include "rt_gauss.cuh"
#include "rt_internal.h"

// Texel loads of the background.  A launch whose textures stay put reads
// them through the read-only data cache; the render server, whose running
// launches meet textures copied in while they run, loads them from L2.
#ifndef RT_TEX_LOAD
#define RT_TEX_LOAD __ldg
#endif

namespace grt {

// The integrator template argument INTEG of the tracer also carries the
// medium of the box: kModeGauss (rt_internal.h) set selects the Gaussian
// conformal cloak (rt_gauss.cuh) in place of the grating cloak of Eq. 1.
__host__ __device__ constexpr int integ_of(int mode) { return mode & 7; }
__host__ __device__ constexpr bool gauss_of(int mode) { return (mode & kModeGauss) != 0; }

enum : int { PH_IDLE = 0, PH_AIR = 1, PH_BOX = 2, PH_DONE = 3, PH_EXIT = 4, PH_EVENT = 5, PH_GUARD = 6 };
enum : int { EV_NONE = -1, EV_GRATING = 0, EV_TOP = 1, EV_XP = 2, EV_XM = 3, EV_ZP = 4, EV_ZM = 5, EV_COUNT = 6 };


template <class R> struct Branch;

// Ray inside the cloak, local coordinates: x = cx + X, |X| <= 1/2.
template <class R>
struct Box {
    R cx, X, y, z, px, py, pz;
    R cX, cy, cz, cpx, cpy;   // compensation terms of the FP32 sums
    R wr, wi, rr, ri;         // W0 and 1/(1+W0) at (X, y) (a prediction until solved)
    R Fx, Fy;                 // force at (X, y)
    R hc;                     // Dormand-Prince: size of the next step
};

// What a lane owns outside the integration loop (shared memory).
template <class R>
struct Cold {
    R cx, X, y, z;            // air: position, x = cx + X
    R dx, dy, dz;             // air: unit direction
    float dl[3];              // FP32 path: the rounding residual of a direction formed in FP64 (else 0)
    R g1[EV_COUNT];           // event functions at the end of a step that crossed a surface
    R hs;                     // size of that step
    int64_t work;             // output slot of the pixel in its scene's arrays
    int64_t pix;              // pixel index i*wout + j
    int scene;                // scene of the pixel (batched renders)
    float acc[3], col[3];
    int sample, bounces, events, status;
    uint32_t rays, nevents, stat[5];
    int phase, surf, steps;   // the wavefront loop (rt_wave.cuh): state of a pixel between tasks
    // Fresnel weights (RT_FLAG_FRESNEL): weight of the current path, which path
    // of the sample it is (0: the camera's, k: the k-th branch), branches
    // queued and taken, and whether the path starts inside the plate
    R w;
    int path, nbr, ibr, in_plate;
    Branch<R>* br;            // this sample's branch queue (kMaxBranches records)
};

enum : int { MED_AIR = 0, MED_BOX = 1, MED_PLATE = 2 };

// The air direction in FP64.  Directions formed in FP64 (the camera ray, a
// reflection or refraction) keep their FP32 rounding residual in dl, so that
// the next FP64 step -- Snell's law at a box face, a mirror reflection --
// starts from the direction as it was formed: Snell's law at a shallow entry
// multiplies a direction error by |p_t| / |p_n|, and the rays that leave the
// cloak and meet the bare grating again amplify it further.
template <class R>
__device__ __forceinline__ void air_dir(const Cold<R>& C, double d[3])
{
    d[0] = (double)C.dx + (double)C.dl[0];
    d[1] = (double)C.dy + (double)C.dl[1];
    d[2] = (double)C.dz + (double)C.dl[2];
}

template <class R>
__device__ __forceinline__ void set_air_dir(Cold<R>& C, double x, double y, double z)
{
    C.dx = (R)x;
    C.dy = (R)y;
    C.dz = (R)z;
    C.dl[0] = (float)(x - (double)C.dx);
    C.dl[1] = (float)(y - (double)C.dy);
    C.dl[2] = (float)(z - (double)C.dz);
}

// The residual matters only where a box face lies ahead (Snell's law); scenes
// without a cloak box or plate skip its FP64 work.
template <class R>
__device__ __forceinline__ void set_air_dir_if(Cold<R>& C, bool keep, double x, double y, double z)
{
    if (keep) {
        set_air_dir(C, x, y, z);
    } else {
        C.dx = (R)x;
        C.dy = (R)y;
        C.dz = (R)z;
        C.dl[0] = C.dl[1] = C.dl[2] = 0.0f;
    }
}

// A direction known only in the path's precision (no residual).
template <class R>
__device__ __forceinline__ void set_air_dir_r(Cold<R>& C, R x, R y, R z)
{
    C.dx = x;
    C.dy = y;
    C.dz = z;
    C.dl[0] = C.dl[1] = C.dl[2] = 0.0f;
}
constexpr int kMaxBranches = 8;      // Fresnel branches followed per camera sample

// A Fresnel branch waiting to be traced: where it starts, its momentum (unit
// direction in air, |p| = n in the box or the plate), its weight and the
// counters of the path it split from.
template <class R>
struct Branch {
    R cx, X, y, z;
    R p[3];
    R w;
    int medium, surf, bounces, events, steps;
};

// Unpolarised Fresnel reflectance R = (rs^2 + rp^2)/2 going from index n1 into
// n2, from the normal components of the momentum on both sides (|p| = n):
//   rs = (|pn1| - |pn2|) / (|pn1| + |pn2|),
//   rp = (n2^2 |pn1| - n1^2 |pn2|) / (n2^2 |pn1| + n1^2 |pn2|).
// Written with explicit roundings (__dmul_rn, __dadd_rn: never contracted
// into FMAs) so that every kernel computes the same weights.
__device__ __forceinline__ double fresnel_R(double n1, double n2, double pn1, double pn2)
{
    const double a = fabs(pn1), b = fabs(pn2);
    const double rs = (a - b) / (a + b);
    const double u = __dmul_rn(__dmul_rn(n2, n2), a), v = __dmul_rn(__dmul_rn(n1, n1), b);
    const double rp = __dadd_rn(u, -v) / __dadd_rn(u, v);
    return 0.5 * __dadd_rn(__dmul_rn(rs, rs), __dmul_rn(rp, rp));
}

// At a Fresnel crossing: the camera's path queues the reflected branch (if
// there is room) and every path keeps the transmitted share of its weight.
template <class R>
__device__ __forceinline__ void fresnel_split(Cold<R>& C, double Rf, int medium, R cx, R X, R y, R z, double pr0,
                                              double pr1, double pr2, int surf, int steps)
{
    if (C.path == 0 && C.br && C.nbr < kMaxBranches) {
        Branch<R>& q = C.br[C.nbr++];
        q.cx = cx; q.X = X; q.y = y; q.z = z;
        q.p[0] = (R)pr0; q.p[1] = (R)pr1; q.p[2] = (R)pr2;
        q.w = (R)((double)C.w * Rf);
        q.medium = medium;
        q.surf = surf;
        q.bounces = C.bounces;
        q.events = C.events;
        q.steps = steps;
    }
    C.w = (R)((double)C.w * (1.0 - Rf));
}

// Scene options (RT_FLAG_*) as one build of the kernels sees them: the plain
// build (OPT = false) compiles every option out, so scenes without options
// pay nothing for them; the options build reads them from the scene.
template <bool OPT>
__device__ __forceinline__ int opt_flags(const DevScene& sc)
{
    if constexpr (OPT) return sc.flags;
    else return 0;
}

// ------------------------------------------------------------------------
// W0 near the branch point in FP64 (FP32 path only).
// ------------------------------------------------------------------------
// Halley's iteration on W e^W = zeta from the branch-point series in
// p = sqrt(2 (e zeta + 1)) (Corless et al. 1996), for |zeta + 1/e| < 1e-3.
static __device__ __noinline__ void w0_branch_fp64(double kA, double X, double y, double& wr, double& wi,
                                                   int& iters)
{
    const double e = kA * exp(-kTwoPi * y);
    double s, c;
    sincospi(2.0 * X, &s, &c);
    const double zr = -e * c, zi = -e * s;
    const double qr = 2.0 * (M_E * zr + 1.0), qi = 2.0 * M_E * zi;
    const double m = sqrt(qr * qr + qi * qi);
    double pr = sqrt(0.5 * (m + qr));
    double pi = (pr > 0.0) ? 0.5 * qi / pr : sqrt(0.5 * (m - qr));
    if (pr == 0.0 && qi < 0.0) pi = -pi;
    const double p2r = pr * pr - pi * pi, p2i = 2.0 * pr * pi;
    const double p3r = p2r * pr - p2i * pi, p3i = p2r * pi + p2i * pr;
    wr = -1.0 + pr - p2r / 3.0 + (11.0 / 72.0) * p3r;
    wi = pi - p2i / 3.0 + (11.0 / 72.0) * p3i;
    iters = 0;
    for (int it = 0; it < 60; ++it) {
        const double ex = exp(wr);
        double sw, cw;
        sincos(wi, &sw, &cw);
        const double er = ex * cw, ei = ex * sw;
        const double fr = wr * er - wi * ei - zr, fi = wr * ei + wi * er - zi;
        const double ar = wr + 1.0, ai = wi;
        const double nr = (wr + 2.0) * fr - wi * fi, ni = (wr + 2.0) * fi + wi * fr;
        const double den = 2.0 * (ar * ar + ai * ai);
        const double tr = (nr * ar + ni * ai) / den, ti = (ni * ar - nr * ai) / den;
        const double Dr = er * ar - ei * ai - tr, Di = er * ai + ei * ar - ti;
        const double dd = Dr * Dr + Di * Di;
        const double dwr = (fr * Dr + fi * Di) / dd, dwi = (fi * Dr - fr * Di) / dd;
        wr -= dwr;
        wi -= dwi;
        ++iters;
        if (!(dwr * dwr + dwi * dwi > 1e-30 * (wr * wr + wi * wi))) break;
    }
}

template <class R>
__device__ __forceinline__ void w0_eval(const StepConst<R>& k, R X, R y, R& wr, R& wi, R& rr, R& ri, LaneStats& st)
{
    const R kA = k.kA;
    st.newton += w0_solve(kA, k.w0tol, X, y, wr, wi, rr, ri);
    st.evals += 1;
    if constexpr (sizeof(R) == 4) {
        // |zeta + 1/e| < 1e-3 corresponds to |1 + W0|^2 < 2e * 1e-3
        if (rr * rr + ri * ri > R(1.0 / (2.0 * M_E * 1e-3))) {
            double dwr, dwi;
            int it;
            w0_branch_fp64((double)kA, (double)X, (double)y, dwr, dwi, it);
            const double ar = 1.0 + dwr, ai = dwi, inv = 1.0 / (ar * ar + ai * ai);
            wr = (R)dwr;
            wi = (R)dwi;
            rr = (R)(ar * inv);
            ri = (R)(-ai * inv);
            st.refine += 1;
            st.newton += it;
        }
    }
}

// W0 at (X, y) from its value at a point (dx, dy) away: first-order
// continuation, then Newton steps unless the continuation is already exact to
// the working precision (its error is about k^2 |W| n^3 |dz|^2 / 2); in that
// case 1/(1+W) is continued to first order as well.  Returns whether it
// solved (took Newton steps).
template <class R>
__device__ __forceinline__ bool w0_continue(const StepConst<R>& k, R X, R y, R dx, R dy, R& wr, R& wi, R& rr, R& ri,
                                            LaneStats& st)
{
    const R n2 = rr * rr + ri * ri;
    const R dz2 = dx * dx + dy * dy;
    const R ow = wr, owi = wi;
    const bool cont = dz2 * n2 * (n2 > R(1) ? n2 : R(1)) <= Mth<R>::kPredTol;
    // FP32 predicts to first order either way; FP64 guesses a solve's start
    // to third order (w0_predict3)
    if (sizeof(R) == 4 || cont) w0_predict(wr, wi, rr, ri, dx, dy);
    if (cont) {
        const R ddr = wr - ow, ddi = wi - owi;            // dW
        const R tr = rr * ddr - ri * ddi, ti = rr * ddi + ri * ddr;   // r dW
        const R nrr = rr - (rr * tr - ri * ti), nri = ri - (rr * ti + ri * tr);   // r (1 - r dW)
        rr = nrr;
        ri = nri;
        st.evals += 1;
        return false;
    }
    if constexpr (sizeof(R) == 8) w0_predict3(wr, wi, rr, ri, dx, dy);
    w0_eval(k, X, y, wr, wi, rr, ri, st);
    return true;
}

// ------------------------------------------------------------------------
// Medium of the box, by the kind of cloak.  The Box fields (wr, wi) hold W0
// (grating) or W = -i k (w - z) (Gaussian), (rr, ri) hold dw/dz, (Fx, Fy)
// the force.
// ------------------------------------------------------------------------
// Solve at (X, y) from the guess in (wr, wi); the force too.
template <class R, int INTEG>
__device__ __forceinline__ void med_eval(const StepConst<R>& k, R X, R y, R& wr, R& wi, R& rr, R& ri, R& Fx, R& Fy,
                                         LaneStats& st)
{
    if constexpr (gauss_of(INTEG)) {
        gauss_solve(k, X, y, wr, wi, rr, ri, Fx, Fy, st);
    } else {
        w0_eval(k, X, y, wr, wi, rr, ri, st);
        ray_force(wr, wi, rr, ri, k.fk, Fx, Fy);
    }
}

// Solve only: the grating leaves the force to med_force (which it computes
// from W0 and 1/(1+W0) alone); the Gaussian solve yields it anyway.
template <class R, int INTEG>
__device__ __forceinline__ void med_solve(const StepConst<R>& k, R X, R y, R& wr, R& wi, R& rr, R& ri, R& Fx,
                                          R& Fy, LaneStats& st)
{
    if constexpr (gauss_of(INTEG)) gauss_solve(k, X, y, wr, wi, rr, ri, Fx, Fy, st);
    else w0_eval(k, X, y, wr, wi, rr, ri, st);
}

template <class R, int INTEG>
__device__ __forceinline__ void med_force(const StepConst<R>& k, Box<R>& b)
{
    if constexpr (!gauss_of(INTEG)) ray_force(b.wr, b.wi, b.rr, b.ri, k.fk, b.Fx, b.Fy);
}

// A stage point (X, y) reached by (dx, dy) from the previous point, whose
// values are in (wr, wi, rr, ri) and (Fpx, Fpy): continuation and solve; the
// force at the new point goes to (Fx, Fy).
// (gpr, gpi): the Gaussian medium's second derivative of dw/dz at the
// previous point in, at the new one out (zero when unknown).
// `far`: the point is known to lie beyond the continuation's reach (the
// second and fourth stages of a full RK4 step, StepConst::far24), so W0 is
// predicted and solved without testing the distance: the same arithmetic as
// w0_continue's solving branch.
template <class R, int INTEG>
__device__ __forceinline__ bool med_stage(const StepConst<R>& k, R X, R y, R dx, R dy, R& wr, R& wi, R& rr, R& ri,
                                          R Fpx, R Fpy, R& Fx, R& Fy, R& gpr, R& gpi, LaneStats& st,
                                          bool far = false)
{
    if constexpr (gauss_of(INTEG)) {
        Fx = Fpx;
        Fy = Fpy;
        return gauss_continue(k, X, y, dx, dy, wr, wi, rr, ri, Fx, Fy, gpr, gpi, st);
    } else {
        bool solved;
        if (far) {
            if constexpr (sizeof(R) == 4) w0_predict(wr, wi, rr, ri, dx, dy);
            else w0_predict3(wr, wi, rr, ri, dx, dy);
            w0_eval(k, X, y, wr, wi, rr, ri, st);
            solved = true;
        } else {
            solved = w0_continue(k, X, y, dx, dy, wr, wi, rr, ri, st);
        }
        ray_force(wr, wi, rr, ri, k.fk, Fx, Fy);
        return solved;
    }
}

// The end point of an RK4 step, (dx, dy) from its fourth stage point.  The
// grating continues W0 from the stages' solves, with a Newton step only when
// the continuation is not exact to the working precision (it is for the
// distance between the two points, O(h^2) times the change of the force);
// a step whose stages were all continued (a very small h) solves here, so
// that every step solves W0 at least once and continuation errors cannot
// add up from step to step.  The Gaussian medium continues or solves for its
// force as well, which it returns in (Fx, Fy); the grating's force is left to
// the caller.
template <class R, int INTEG>
__device__ __forceinline__ void med_end(const StepConst<R>& k, R X, R y, R dx, R dy, R& wr, R& wi, R& rr, R& ri,
                                        R& Fx, R& Fy, R& gpr, R& gpi, bool solved, LaneStats& st)
{
    if constexpr (gauss_of(INTEG)) {
        if (solved) {
            gauss_continue(k, X, y, dx, dy, wr, wi, rr, ri, Fx, Fy, gpr, gpi, st);
        } else {
            gauss_predict(wr, wi, rr, ri, Fx, Fy, dx, dy);
            gauss_solve(k, X, y, wr, wi, rr, ri, Fx, Fy, gpr, gpi, st);
        }
    } else if (solved) {
        w0_continue(k, X, y, dx, dy, wr, wi, rr, ri, st);
    } else {
        w0_predict(wr, wi, rr, ri, dx, dy);
        w0_eval(k, X, y, wr, wi, rr, ri, st);
    }
}

// Keep the grating's abscissa as cell + fraction; the Gaussian box works
// with the absolute abscissa (cx = 0).
template <class R, int INTEG>
__device__ __forceinline__ void wrap_cell(Box<R>& o)
{
    if constexpr (!gauss_of(INTEG)) {
        if (o.X >= R(0.5)) { o.X -= R(1); o.cx += R(1); }
        else if (o.X < R(-0.5)) { o.X += R(1); o.cx -= R(1); }
    }
}

// ------------------------------------------------------------------------
// RK4 in the cloak.
// ------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void kahan_add(R& s, R& c, R inc)
{
    if constexpr (sizeof(R) == 4) {
        const R yv = inc - c;
        const R t = s + yv;
        c = (t - s) - yv;
        s = t;
    } else {
        s += inc;
    }
}

// One RK4 step of size h from s (W0 solved and force known at s) into o;
// o's W0 is continued to the end point but not solved.
template <class R, int INTEG>
__device__ __forceinline__ void rk4_step(const StepConst<R>& k, const Box<R>& s, R h, Box<R>& o, LaneStats& st)
{
    if constexpr (sizeof(R) == 4) {
        // the same step with the (x, y) arithmetic in packed pairs
        const float h2 = 0.5f * h;
        // a full step's second and fourth stages always solve (StepConst::far24)
        const bool far = (k.far24 != 0.0f) & (h == k.h);
        float wr = s.wr, wi = s.wi, rr = s.rr, ri = s.ri;
        const float2 P = p2(s.X, s.y), M = p2(s.px, s.py), F1 = p2(s.Fx, s.Fy);
        const float2 H2 = p2s(h2), H = p2s(h);
        // stage 2 at r + h/2 p
        const float2 D2 = mul2(H2, M);
        const float2 P2 = fma2(H2, M, P);
        float F2x, F2y, gpr = 0.0f, gpi = 0.0f;
        bool solved = med_stage<R, INTEG>(k, P2.x, P2.y, D2.x, D2.y, wr, wi, rr, ri, s.Fx, s.Fy, F2x, F2y, gpr,
                                          gpi, st, far);
        // stage 3 at r + h/2 (p + h/2 F1)
        const float2 P3 = fma2(H2, fma2(H2, F1, M), P);
        const float2 D3 = sub2(P3, P2);
        float F3x, F3y;
        solved |= med_stage<R, INTEG>(k, P3.x, P3.y, D3.x, D3.y, wr, wi, rr, ri, F2x, F2y, F3x, F3y, gpr, gpi, st);
        // stage 4 at r + h (p + h/2 F2)
        const float2 Fs2 = p2(F2x, F2y);
        const float2 P4 = fma2(H, fma2(H2, Fs2, M), P);
        const float2 D4 = sub2(P4, P3);
        float F4x, F4y;
        solved |= med_stage<R, INTEG>(k, P4.x, P4.y, D4.x, D4.y, wr, wi, rr, ri, F3x, F3y, F4x, F4y, gpr, gpi, st,
                                      far);
        // position increment h p + h^2/6 (F1 + F2 + F3), momentum h/6 (F1 + 2F2 + 2F3 + F4)
        const float h6 = h * (1.0f / 6.0f), hh6 = h * h6;
        const float2 Fs3 = p2(F3x, F3y), Fs4 = p2(F4x, F4y);
        const float2 S23 = add2(Fs2, Fs3);
        const float2 dP = fma2(p2s(hh6), add2(F1, S23), mul2(H, M));
        const float2 dM = mul2(p2s(h6), add2(fma2(p2s(2.0f), S23, F1), Fs4));
        float2 Pn = P, Pc = p2(s.cX, s.cy), Mn = M, Mc = p2(s.cpx, s.cpy);
        kahan2(Pn, Pc, dP);
        kahan2(Mn, Mc, dM);
        o = s;
        o.X = Pn.x; o.y = Pn.y; o.cX = Pc.x; o.cy = Pc.y;
        o.px = Mn.x; o.py = Mn.y; o.cpx = Mc.x; o.cpy = Mc.y;
        kahan_add(o.z, o.cz, h * s.pz);
        const float2 De = sub2(Pn, P4);
        float Fex = F4x, Fey = F4y;
        med_end<R, INTEG>(k, o.X, o.y, De.x, De.y, wr, wi, rr, ri, Fex, Fey, gpr, gpi, solved, st);
        o.wr = wr; o.wi = wi; o.rr = rr; o.ri = ri;
        if constexpr (gauss_of(INTEG)) { o.Fx = Fex; o.Fy = Fey; }
        wrap_cell<R, INTEG>(o);
        return;
    }
    const R h2 = R(0.5) * h;
    const bool far = (k.far24 != R(0)) & (h == k.h);
    R wr = s.wr, wi = s.wi, rr = s.rr, ri = s.ri;
    // stage 2 at r + h/2 p
    const R X2 = s.X + h2 * s.px, y2 = s.y + h2 * s.py;
    R F2x, F2y, gpr = R(0), gpi = R(0);
    bool solved = med_stage<R, INTEG>(k, X2, y2, h2 * s.px, h2 * s.py, wr, wi, rr, ri, s.Fx, s.Fy, F2x, F2y, gpr, gpi,
                                      st, far);
    // stage 3 at r + h/2 (p + h/2 F1), (h/2)^2 F1 away from stage 2
    const R X3 = s.X + h2 * (s.px + h2 * s.Fx), y3 = s.y + h2 * (s.py + h2 * s.Fy);
    R F3x, F3y;
    solved |= med_stage<R, INTEG>(k, X3, y3, X3 - X2, y3 - y2, wr, wi, rr, ri, F2x, F2y, F3x, F3y, gpr, gpi, st);
    // stage 4 at r + h (p + h/2 F2)
    const R X4 = s.X + h * (s.px + h2 * F2x), y4 = s.y + h * (s.py + h2 * F2y);
    R F4x, F4y;
    solved |= med_stage<R, INTEG>(k, X4, y4, X4 - X3, y4 - y3, wr, wi, rr, ri, F3x, F3y, F4x, F4y, gpr, gpi, st, far);
    // position increment h p + h^2/6 (F1 + F2 + F3), momentum h/6 (F1 + 2F2 + 2F3 + F4)
    const R h6 = h * R(1.0 / 6.0), hh6 = h * h6;
    const R dX = h * s.px + hh6 * (s.Fx + F2x + F3x);
    const R dY = h * s.py + hh6 * (s.Fy + F2y + F3y);
    const R dZ = h * s.pz;
    const R dPx = h6 * (s.Fx + R(2) * (F2x + F3x) + F4x);
    const R dPy = h6 * (s.Fy + R(2) * (F2y + F3y) + F4y);
    o = s;
    kahan_add(o.X, o.cX, dX);
    kahan_add(o.y, o.cy, dY);
    kahan_add(o.z, o.cz, dZ);
    kahan_add(o.px, o.cpx, dPx);
    kahan_add(o.py, o.cpy, dPy);
    R Fex = F4x, Fey = F4y;
    med_end<R, INTEG>(k, o.X, o.y, o.X - X4, o.y - y4, wr, wi, rr, ri, Fex, Fey, gpr, gpi, solved, st);
    o.wr = wr; o.wi = wi; o.rr = rr; o.ri = ri;
    if constexpr (gauss_of(INTEG)) { o.Fx = Fex; o.Fy = Fey; }
    wrap_cell<R, INTEG>(o);
}

// ------------------------------------------------------------------------
// RK4 on Eq. 11 in physical time t (RT_RK4T).
// ------------------------------------------------------------------------
// The box state carries the velocity v (|v| = c0/n, c0 = 1) in px, py, pz.
// With F = n grad n, the force of the tau form (scaled by s^2 like it), the
// acceleration of Eq. 11 is dv/dt = (|v|^2 grad n - 2 (grad n . v) v) / n
// = (|v|^2 F - 2 (F . v) v) / n^2, n^2 = s^2 |r|^2; F has no z component.
template <class R>
__device__ __forceinline__ void accel_t(const StepConst<R>& k, R Fx, R Fy, R vx, R vy, R vz, R rr, R ri, R& ax,
                                        R& ay, R& az)
{
    const R in2 = k.is2 * Mth<R>::rcp(rr * rr + ri * ri);
    const R v2 = vx * vx + vy * vy + vz * vz;
    const R g2 = R(2) * (Fx * vx + Fy * vy);
    ax = (v2 * Fx - g2 * vx) * in2;
    ay = (v2 * Fy - g2 * vy) * in2;
    az = -(g2 * vz) * in2;
}

// One classical RK4 step of size h (in t) on the first-order system
// (r, v)' = (v, a(r, v)) from s (W0 solved and F known at s) into o; o's W0
// is continued to the end point but not solved.  v_z changes along the ray
// (n^2 v_z is the conserved momentum) and is summed without compensation.
template <class R, int INTEG>
__device__ __forceinline__ void rk4t_step(const StepConst<R>& k, const Box<R>& s, R h, Box<R>& o, LaneStats& st)
{
    const R h2 = R(0.5) * h;
    R wr = s.wr, wi = s.wi, rr = s.rr, ri = s.ri;
    R a1x, a1y, a1z;
    accel_t(k, s.Fx, s.Fy, s.px, s.py, s.pz, rr, ri, a1x, a1y, a1z);
    R Fx, Fy;
    // stage 2 at (r + h/2 v, v + h/2 a1)
    const R v2x = s.px + h2 * a1x, v2y = s.py + h2 * a1y, v2z = s.pz + h2 * a1z;
    const R X2 = s.X + h2 * s.px, y2 = s.y + h2 * s.py;
    R gpr = R(0), gpi = R(0);
    bool solved = med_stage<R, INTEG>(k, X2, y2, h2 * s.px, h2 * s.py, wr, wi, rr, ri, s.Fx, s.Fy, Fx, Fy, gpr, gpi,
                                      st);
    R a2x, a2y, a2z;
    accel_t(k, Fx, Fy, v2x, v2y, v2z, rr, ri, a2x, a2y, a2z);
    // stage 3 at (r + h/2 v2, v + h/2 a2)
    const R v3x = s.px + h2 * a2x, v3y = s.py + h2 * a2y, v3z = s.pz + h2 * a2z;
    const R X3 = s.X + h2 * v2x, y3 = s.y + h2 * v2y;
    solved |= med_stage<R, INTEG>(k, X3, y3, X3 - X2, y3 - y2, wr, wi, rr, ri, Fx, Fy, Fx, Fy, gpr, gpi, st);
    R a3x, a3y, a3z;
    accel_t(k, Fx, Fy, v3x, v3y, v3z, rr, ri, a3x, a3y, a3z);
    // stage 4 at (r + h v3, v + h a3)
    const R v4x = s.px + h * a3x, v4y = s.py + h * a3y, v4z = s.pz + h * a3z;
    const R X4 = s.X + h * v3x, y4 = s.y + h * v3y;
    solved |= med_stage<R, INTEG>(k, X4, y4, X4 - X3, y4 - y3, wr, wi, rr, ri, Fx, Fy, Fx, Fy, gpr, gpi, st);
    R a4x, a4y, a4z;
    accel_t(k, Fx, Fy, v4x, v4y, v4z, rr, ri, a4x, a4y, a4z);
    // increments h/6 (k1 + 2 k2 + 2 k3 + k4) of both halves of the state
    const R h6 = h * R(1.0 / 6.0);
    const R dX = h6 * (s.px + R(2) * (v2x + v3x) + v4x);
    const R dY = h6 * (s.py + R(2) * (v2y + v3y) + v4y);
    const R dZ = h6 * (s.pz + R(2) * (v2z + v3z) + v4z);
    const R dVx = h6 * (a1x + R(2) * (a2x + a3x) + a4x);
    const R dVy = h6 * (a1y + R(2) * (a2y + a3y) + a4y);
    const R dVz = h6 * (a1z + R(2) * (a2z + a3z) + a4z);
    o = s;
    kahan_add(o.X, o.cX, dX);
    kahan_add(o.y, o.cy, dY);
    kahan_add(o.z, o.cz, dZ);
    kahan_add(o.px, o.cpx, dVx);
    kahan_add(o.py, o.cpy, dVy);
    o.pz += dVz;
    med_end<R, INTEG>(k, o.X, o.y, o.X - X4, o.y - y4, wr, wi, rr, ri, Fx, Fy, gpr, gpi, solved, st);
    o.wr = wr; o.wi = wi; o.rr = rr; o.ri = ri;
    wrap_cell<R, INTEG>(o);
}

// Dormand & Prince (1980) RK5(4)7M: nodes, coefficients, fifth-order weights
// and the differences between the fifth- and fourth-order weights.
struct DPT {
    static constexpr double a21 = 1.0 / 5;
    static constexpr double a31 = 3.0 / 40, a32 = 9.0 / 40;
    static constexpr double a41 = 44.0 / 45, a42 = -56.0 / 15, a43 = 32.0 / 9;
    static constexpr double a51 = 19372.0 / 6561, a52 = -25360.0 / 2187, a53 = 64448.0 / 6561, a54 = -212.0 / 729;
    static constexpr double a61 = 9017.0 / 3168, a62 = -355.0 / 33, a63 = 46732.0 / 5247, a64 = 49.0 / 176,
                            a65 = -5103.0 / 18656;
    static constexpr double b1 = 35.0 / 384, b3 = 500.0 / 1113, b4 = 125.0 / 192, b5 = -2187.0 / 6784, b6 = 11.0 / 84;
    static constexpr double e1 = 35.0 / 384 - 5179.0 / 57600, e3 = 500.0 / 1113 - 7571.0 / 16695,
                            e4 = 125.0 / 192 - 393.0 / 640, e5 = -2187.0 / 6784 + 92097.0 / 339200,
                            e6 = 11.0 / 84 - 187.0 / 2100, e7 = -1.0 / 40;
};

// The tableau as a function: a(j, k) for stages j, k = 1..7, row 7 holding
// the fifth-order weights b (first same as last), and e(j) = b_j - b*_j.
__host__ __device__ constexpr double dp_a(int j, int k)
{
    return j == 2 ? (k == 1 ? DPT::a21 : 0.0)
         : j == 3 ? (k == 1 ? DPT::a31 : k == 2 ? DPT::a32 : 0.0)
         : j == 4 ? (k == 1 ? DPT::a41 : k == 2 ? DPT::a42 : k == 3 ? DPT::a43 : 0.0)
         : j == 5 ? (k == 1 ? DPT::a51 : k == 2 ? DPT::a52 : k == 3 ? DPT::a53 : k == 4 ? DPT::a54 : 0.0)
         : j == 6 ? (k == 1 ? DPT::a61 : k == 2 ? DPT::a62 : k == 3 ? DPT::a63 : k == 4 ? DPT::a64
                     : k == 5 ? DPT::a65 : 0.0)
         : j == 7 ? (k == 1 ? DPT::b1 : k == 3 ? DPT::b3 : k == 4 ? DPT::b4 : k == 5 ? DPT::b5
                     : k == 6 ? DPT::b6 : 0.0)
         : 0.0;
}
__host__ __device__ constexpr double dp_e(int j)
{
    return j == 1 ? DPT::e1 : j == 3 ? DPT::e3 : j == 4 ? DPT::e4 : j == 5 ? DPT::e5 : j == 6 ? DPT::e6
         : j == 7 ? DPT::e7 : 0.0;
}
// Nystrom form for r'' = F(r): node c_j = sum_k a_jk, position weights
// (A A)_jl = sum_k a_jk a_kl of the forces, and (e A)_l = sum_j e_j a_jl.
__host__ __device__ constexpr double dp_c(int j)
{
    double c = 0.0;
    for (int k = 1; k < j; ++k) c += dp_a(j, k);
    return c;
}
__host__ __device__ constexpr double dp_aa(int j, int l)
{
    double v = 0.0;
    for (int k = l + 1; k < j; ++k) v += dp_a(j, k) * dp_a(k, l);
    return v;
}
__host__ __device__ constexpr double dp_ea(int l)
{
    double v = 0.0;
    for (int j = l + 1; j <= 7; ++j) v += dp_e(j) * dp_a(j, l);
    return v;
}

// Coefficients of the Nystrom form for the FP64 stage loop: row j - 2 of
// kDpAA holds (A A)_jl for stages j = 2..6 and (b A)_l for the solution
// (j = 7); kDpC the nodes c_j.  The loop over the stages is kept rolled, with
// one evaluation of W0 and the force in its body: unrolled, the seven inlined
// evaluations overflow the instruction cache (most issue slots were lost to
// instruction fetch).
#define RT_DPAA_ROWD(j) {dp_aa(j, 1), dp_aa(j, 2), dp_aa(j, 3), dp_aa(j, 4), dp_aa(j, 5), dp_aa(j, 6)}
static __constant__ double kDpAAd[6][6] = {RT_DPAA_ROWD(2), RT_DPAA_ROWD(3), RT_DPAA_ROWD(4),
                                           RT_DPAA_ROWD(5), RT_DPAA_ROWD(6), RT_DPAA_ROWD(7)};
#undef RT_DPAA_ROWD
static __constant__ double kDpCd[6] = {dp_c(2), dp_c(3), dp_c(4), dp_c(5), dp_c(6), 1.0};
template <class R> __device__ __forceinline__ R dp_tab_aa(int r, int c);
template <> __device__ __forceinline__ double dp_tab_aa<double>(int r, int c) { return kDpAAd[r][c]; }
// The same coefficients for the running sums of the FP32 step, each value
// twice (a packed pair for FFMA2): row r of kDpP2 holds (A A)_{r+2, q+1} for
// q = 0..6 (zero past the tableau, so that rows up to 10 may be read); kDpB2,
// kDpEA2 and kDpE2 hold b_{q+1}, (e A)_{q+1} and e_{q+1}; kDpC2 c_{q+2}.
__host__ __device__ constexpr double dp_aap(int r, int q) { return (r + 2 <= 7 && q + 1 <= 6) ? dp_aa(r + 2, q + 1) : 0.0; }
__host__ __device__ constexpr double dp_b(int l) { return dp_a(7, l); }
#define RT_F2(v) {(float)(v), (float)(v)}
#define RT_DPP_ROW(r) {RT_F2(dp_aap(r, 0)), RT_F2(dp_aap(r, 1)), RT_F2(dp_aap(r, 2)), RT_F2(dp_aap(r, 3)), \
                       RT_F2(dp_aap(r, 4)), RT_F2(dp_aap(r, 5)), RT_F2(dp_aap(r, 6))}
#define RT_DPV(f) {RT_F2(f(1)), RT_F2(f(2)), RT_F2(f(3)), RT_F2(f(4)), RT_F2(f(5)), RT_F2(f(6)), RT_F2(f(7))}
static __constant__ float2 kDpP2[11][7] = {RT_DPP_ROW(0), RT_DPP_ROW(1), RT_DPP_ROW(2), RT_DPP_ROW(3), RT_DPP_ROW(4),
                                           RT_DPP_ROW(5), RT_DPP_ROW(6), RT_DPP_ROW(7), RT_DPP_ROW(8), RT_DPP_ROW(9),
                                           RT_DPP_ROW(10)};
static __constant__ float2 kDpB2[7] = RT_DPV(dp_b);
static __constant__ float2 kDpEA2[7] = RT_DPV(dp_ea);
static __constant__ float2 kDpE2[7] = RT_DPV(dp_e);
static __constant__ float2 kDpC2[6] = {RT_F2(dp_c(2)), RT_F2(dp_c(3)), RT_F2(dp_c(4)), RT_F2(dp_c(5)), RT_F2(dp_c(6)),
                                       RT_F2(dp_c(7))};
#undef RT_DPP_ROW
#undef RT_DPV
#undef RT_F2
template <class R> __device__ __forceinline__ R dp_tab_c(int r);
template <> __device__ __forceinline__ double dp_tab_c<double>(int r) { return kDpCd[r]; }

// One Dormand-Prince step of size h from s (W0 solved and force known at s)
// into o: the fifth-order solution, W0 solved and the force at it (the first
// stage of the next step).  e[4] receives the error estimate of
// (x, y, p_x, p_y).  The ODE is r' = p, p' = F(r) with F a function of r
// alone, so the method is taken in its Nystrom form: stage momenta
// p + h sum_k a_jk F_k are never needed, stage positions are
// r + c_j h p + h^2 sum_l (A A)_jl F_l, the solution
// r + h p + h^2 sum_l (b A)_l F_l and p + h sum_j b_j F_j, and the position
// error h^2 sum_l (e A)_l F_l -- the same method with only the forces kept.
template <class R, int INTEG>
__device__ __forceinline__ void dp45_step_table(const StepConst<R>& k, const Box<R>& s, R h, Box<R>& o, R e[4],
                                                LaneStats& st)
{
    R wr = s.wr, wi = s.wi, rr = s.rr, ri = s.ri;
    R Xp = s.X, yp = s.y;
    R gpr = R(0), gpi = R(0);
    const R hpx = h * s.px, hpy = h * s.py, hh = h * h;
    R Fx[7], Fy[7];
    Fx[0] = s.Fx;
    Fy[0] = s.Fy;
#pragma unroll 1
    for (int j = 2; j <= 7; ++j) {
        R ax = R(0), ay = R(0);
        const int nl = (j < 7) ? j - 2 : 6;
#pragma unroll 1
        for (int l = 0; l < nl; ++l) {
            const R a = dp_tab_aa<R>(j - 2, l);
            ax += a * Fx[l];
            ay += a * Fy[l];
        }
        R Xs, Ys;
        if (j < 7) {
            Xs = s.X + (dp_tab_c<R>(j - 2) * hpx + hh * ax);
            Ys = s.y + (dp_tab_c<R>(j - 2) * hpy + hh * ay);
        } else {
            R fx = R(0), fy = R(0);
#pragma unroll
            for (int l = 1; l <= 6; ++l) {
                fx += R(dp_a(7, l)) * Fx[l - 1];
                fy += R(dp_a(7, l)) * Fy[l - 1];
            }
            o = s;
            kahan_add(o.X, o.cX, hpx + hh * ax);
            kahan_add(o.y, o.cy, hpy + hh * ay);
            kahan_add(o.z, o.cz, h * s.pz);
            kahan_add(o.px, o.cpx, h * fx);
            kahan_add(o.py, o.cpy, h * fy);
            Xs = o.X;
            Ys = o.y;
        }
        med_stage<R, INTEG>(k, Xs, Ys, Xs - Xp, Ys - yp, wr, wi, rr, ri, Fx[j - 2], Fy[j - 2], Fx[j - 1], Fy[j - 1],
                            gpr, gpi, st);
        Xp = Xs;
        yp = Ys;
    }
    o.wr = wr; o.wi = wi; o.rr = rr; o.ri = ri;
    o.Fx = Fx[6];
    o.Fy = Fy[6];
    R ex = R(0), ey = R(0), gx = R(0), gy = R(0);
#pragma unroll
    for (int l = 1; l <= 7; ++l) {
        if (l <= 6) {
            ex += R(dp_ea(l)) * Fx[l - 1];
            ey += R(dp_ea(l)) * Fy[l - 1];
        }
        gx += R(dp_e(l)) * Fx[l - 1];
        gy += R(dp_e(l)) * Fy[l - 1];
    }
    e[0] = hh * ex;
    e[1] = hh * ey;
    e[2] = h * gx;
    e[3] = h * gy;
    wrap_cell<R, INTEG>(o);
}

// The same step with running sums in place of the table of stage forces,
// which the rolled stage loop indexes and so keeps in local memory; FP32
// only, with the sums' (x, y) components in packed pairs.
template <class R, int INTEG>
__device__ __forceinline__ void dp45_step_sums(const StepConst<R>& k, const Box<R>& s, R h, Box<R>& o, R e[4],
                                               LaneStats& st)
{
    static_assert(sizeof(R) == 4, "the running-sum step is the FP32 one");
    float wr = s.wr, wi = s.wi, rr = s.rr, ri = s.ri;
    float gpr = 0.0f, gpi = 0.0f;
    const float2 P0 = p2(s.X, s.y), H = p2s(h), HH = p2s(h * h);
    const float2 HP = mul2(H, p2(s.px, s.py));
    // slot m holds the position sum sum_l (A A)_{j+m, l} F_l of stage j + m
    // over the forces known so far; Mv, EAv and Ev the momentum sum b.F and
    // the error sums (e A).F and e.F
    float2 S[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) S[m] = p2s(0.0f);
    float2 Mv = p2s(0.0f), EAv = p2s(0.0f), Ev = p2s(0.0f);
    float2 Fc = p2(s.Fx, s.Fy);                        // the newest force (stage j - 1)
    float2 Pp = P0;                                    // the previous stage point
#pragma unroll 1
    for (int j = 2; j <= 7; ++j) {
        const int q = j - 2;                           // the newest force's index
        Mv = fma2(kDpB2[q], Fc, Mv);
        EAv = fma2(kDpEA2[q], Fc, EAv);
        Ev = fma2(kDpE2[q], Fc, Ev);
#pragma unroll
        for (int m = 0; m < 6; ++m) S[m] = fma2(kDpP2[q + m][q], Fc, S[m]);
        float2 Ps;
        if (j < 7) {
            Ps = add2(P0, fma2(kDpC2[q], HP, mul2(HH, S[0])));
        } else {
            o = s;
            float2 Pn = P0, Pc = p2(s.cX, s.cy), Mn = p2(s.px, s.py), Mc = p2(s.cpx, s.cpy);
            kahan2(Pn, Pc, fma2(HH, S[0], HP));
            kahan2(Mn, Mc, mul2(H, Mv));
            kahan_add(o.z, o.cz, h * s.pz);
            o.X = Pn.x; o.y = Pn.y; o.cX = Pc.x; o.cy = Pc.y;
            o.px = Mn.x; o.py = Mn.y; o.cpx = Mc.x; o.cpy = Mc.y;
            Ps = Pn;
        }
        const float2 D = sub2(Ps, Pp);
        float Fnx, Fny;
        med_stage<R, INTEG>(k, Ps.x, Ps.y, D.x, D.y, wr, wi, rr, ri, Fc.x, Fc.y, Fnx, Fny, gpr, gpi, st);
        Fc = p2(Fnx, Fny);
        Pp = Ps;
#pragma unroll
        for (int m = 0; m < 5; ++m) S[m] = S[m + 1];
        S[5] = p2s(0.0f);
    }
    // the force at the solution (stage 7) enters the momentum error only
    Ev = fma2(kDpE2[6], Fc, Ev);
    o.wr = wr; o.wi = wi; o.rr = rr; o.ri = ri;
    o.Fx = Fc.x;
    o.Fy = Fc.y;
    const float2 EA = mul2(HH, EAv), E = mul2(H, Ev);
    e[0] = EA.x;
    e[1] = EA.y;
    e[2] = E.x;
    e[3] = E.y;
    wrap_cell<R, INTEG>(o);
}

// FP32 takes the running sums (13 % faster on the 1920 x 1080 workload);
// FP64 the table, since the sums' 24 more registers cost it occupancy (4 %
// slower).
template <class R, int INTEG>
__device__ __forceinline__ void dp45_step(const StepConst<R>& k, const Box<R>& s, R h, Box<R>& o, R e[4],
                                          LaneStats& st)
{
    if constexpr (sizeof(R) == 4)
        dp45_step_sums<R, INTEG>(k, s, h, o, e, st);
    else
        dp45_step_table<R, INTEG>(k, s, h, o, e, st);
}

// One step of the scene's integrator of size h from s into o (for event
// location: Phi_{theta h}(s) is one step of size theta h).
template <class R, int INTEG>
__device__ __forceinline__ void integ_step(const StepConst<R>& k, const Box<R>& s, R h, Box<R>& o, LaneStats& st)
{
    if constexpr (integ_of(INTEG) == RT_DP45) {
        R e[4];
        dp45_step<R, INTEG>(k, s, h, o, e, st);
    } else if constexpr (integ_of(INTEG) == RT_RK4T) {
        rk4t_step<R, INTEG>(k, s, h, o, st);
    } else {
        rk4_step<R, INTEG>(k, s, h, o, st);
    }
}

// ------------------------------------------------------------------------
// Events inside the cloak: positive while the ray is inside, negative once it
// crossed the grating (v = Im w = y + Re W0/k < 0) or a face of the box.
// ------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R event_g(const StepConst<R>& k, int ev, const Box<R>& s)
{
    switch (ev) {
        case EV_GRATING: return s.y + s.wr * R(kInvTwoPi);
        case EV_TOP: return k.ytop - s.y;
        case EV_XP: return (k.E2 - s.cx) - s.X;
        case EV_XM: return (k.E2 + s.cx) + s.X;
        case EV_ZP: return k.E2 - s.z;
        default: return k.E2 + s.z;
    }
}

// h grad g . p: the derivative of g(Phi_{theta h}(s)) in theta at the state s.
template <class R>
__device__ __forceinline__ R event_slope(int ev, const Box<R>& s, R h)
{
    switch (ev) {
        case EV_GRATING: return h * (s.ri * s.px + s.rr * s.py);   // grad v = (Im r, Re r)
        case EV_TOP: return -h * s.py;
        case EV_XP: return -h * s.px;
        case EV_XM: return h * s.px;
        case EV_ZP: return -h * s.pz;
        default: return h * s.pz;
    }
}

template <class R>
__device__ __forceinline__ void face_normal(int ev, R N[3])
{
    N[0] = N[1] = N[2] = R(0);
    if (ev == EV_TOP) N[1] = R(1);
    else if (ev == EV_XP) N[0] = R(1);
    else if (ev == EV_XM) N[0] = R(-1);
    else if (ev == EV_ZP) N[2] = R(1);
    else if (ev == EV_ZM) N[2] = R(-1);
    else N[1] = R(-1);
}

// Whether a trial step's end point needs a W0 solve: RK4 only continues W0
// to its end point; the FP32 Dormand-Prince step has already solved it there
// (or continued it exactly to FP32), as its last stage.  The FP64 path solves
// again, as it always did, to keep its rays on the oracle's to 1e-12.
template <class R, int INTEG>
__host__ __device__ constexpr bool resolve_end()
{
    return !(sizeof(R) == 4 && integ_of(INTEG) == RT_DP45);
}

// Root theta in (0, 1] of g_ev(Phi_{theta h}(b)) given its value g1 < 0 at
// theta = 1 (the zero at theta = 0 divided out when the step starts on that
// surface).  First guess from the quadratic through g(0), g'(0) and g(1);
// then Newton steps with the slope at the current point, kept inside the
// bracket (regula falsi otherwise).  On return t = Phi_{theta h}(b) with W0
// solved.
template <class R, int INTEG>
__device__ R locate_event(const StepConst<R>& k, const Box<R>& b, R h, int ev, bool on_surface, R g1, Box<R>& t,
                          LaneStats& st)
{
    const R s0 = event_slope(ev, b, h);
    R lo = R(0), hi = R(1), glo, ghi = g1;
    R th;
    if (on_surface) {
        glo = s0 > R(0) ? s0 : R(1e-30);
        const R c = g1 - glo;                        // g/theta ~ s0 + c theta
        th = (c < R(0)) ? -glo / c : R(0.5);
    } else {
        glo = event_g(k, ev, b);
        if (!(glo > R(0))) {
            t = b;
            return R(0);
        }
        const R c = g1 - glo - s0;                   // g ~ g0 + s0 theta + c theta^2
        th = (glo / (glo - g1));                     // secant
        if (fabs(c) > R(1e-6) * (fabs(s0) + fabs(glo))) {
            const R disc = s0 * s0 - R(4) * c * glo;
            if (disc >= R(0)) {
                const R sq = Mth<R>::sqrt_(disc);
                const R q = R(-0.5) * (s0 + (s0 >= R(0) ? sq : -sq));
                R r1 = q / c, r2 = glo / q;
                if (r1 > R(0) && r1 <= R(1)) th = r1;
                if (r2 > R(0) && r2 <= R(1) && (!(th > R(0) && th <= R(1)) || r2 < th)) th = r2;
            }
        }
    }
    if (!(th > lo && th < hi)) th = R(0.5) * (lo + hi);
    int side = 0;
    for (int it = 0; it < Mth<R>::kEventIt; ++it) {
        integ_step<R, INTEG>(k, b, th * h, t, st);
        if constexpr (resolve_end<R, INTEG>())
            med_solve<R, INTEG>(k, t.X, t.y, t.wr, t.wi, t.rr, t.ri, t.Fx, t.Fy, st);
        const R g = event_g(k, ev, t);
        if (fabs(g) <= Mth<R>::kEventTol) return th;
        const R gd = on_surface ? g / th : g;
        if (gd > R(0)) { lo = th; glo = gd; if (side == 1) ghi *= R(0.5); side = 1; }
        else { hi = th; ghi = gd; if (side == -1) glo *= R(0.5); side = -1; }
        if (hi - lo <= R(4) * Mth<R>::kEps) return th;
        if (it + 1 == Mth<R>::kEventIt) break;       // keep t at the last theta evaluated
        const R dg = event_slope(ev, t, h);
        const R dgd = on_surface ? (dg * th - g) / (th * th) : dg;
        R nt = th - gd / dgd;
        if (!(nt > lo && nt < hi)) nt = (lo * ghi - hi * glo) / (ghi - glo);
        if (!(nt > lo && nt < hi)) nt = R(0.5) * (lo + hi);
        th = nt;
    }
    return th;
}

// ------------------------------------------------------------------------
// Air: local-coordinate helpers, camera, mirror, box, background.
// ------------------------------------------------------------------------
// Move the air ray by t along its direction.  t * dx is split exactly into a
// rounded product and its remainder, so the cell fraction keeps full
// resolution however long the move.
template <class R>
__device__ __forceinline__ void advance(Cold<R>& C, R t)
{
    const R a = t * C.dx;
    const R e = fma(t, C.dx, -a);
    const R n = Mth<R>::rint_(a);
    C.cx += n;
    C.X = (C.X + (a - n)) + e;
    const R m = Mth<R>::rint_(C.X);
    C.cx += m;
    C.X -= m;
    C.y += t * C.dy;
    C.z += t * C.dz;
}

// Camera ray of sample s of pixel pix (Sec. 4), set up in FP64 and advanced
// to 2^-10 periods before the first surface it can meet (the cloak box, the
// grating band y = A or the flat mirror), then stored in local coordinates:
// the lever arm of the FP32 rounding of the direction is that short, and the
// remaining distance is far above the box-entry threshold of the FP32 path.  Reciprocals and the norm use FP32 seeds refined by one
// Newton step in FP64.
template <class R, bool OPT>
__device__ __forceinline__ void camera_start(const DevScene& sc, Cold<R>& C)
{
    const int i = (int)(C.pix / sc.wout), j = (int)(C.pix % sc.wout);
    double ox = 0.5, oy = 0.5;
    if (sc.spp > 1) {
        const uint64_t c = (((uint64_t)sc.scene_id * (uint64_t)sc.height + (uint64_t)i) * (uint64_t)sc.wout +
                            (uint64_t)j) * (uint64_t)sc.spp + (uint64_t)C.sample;
        const double u1 = uniform24(sc.seed, 2 * c + 1), u2 = uniform24(sc.seed, 2 * c + 2);
        if (sc.m > 0) {
            ox = ((double)(C.sample % sc.m) + u1) * sc.inv_m;
            oy = ((double)(C.sample / sc.m) + u2) * sc.inv_m;
        } else {
            ox = u1;
            oy = u2;
        }
    }
    const double px = sc.centre_line ? 0.0 : ((double)j + ox) * sc.two_over_w - 1.0;
    const double py = 1.0 - ((double)i + oy) * sc.two_over_h;
    const double ptx = px * sc.tx, pty = py * sc.ty;
    double d[3], n2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        d[a] = sc.f[a] + ptx * sc.r[a] + pty * sc.u[a];
        n2 += d[a] * d[a];
    }
    double is = (double)rsqrtf((float)n2);
    is = is * (1.5 - 0.5 * n2 * is * is);
    for (int a = 0; a < 3; ++a) d[a] *= is;
    // How far to advance: only a distance, found in FP32 (the FP64 pipe runs
    // at 1/64 of the FP32 rate); the point reached is then formed in FP64
    // along the FP64 direction.  2^-10 short of the first surface, with
    // 1e-5 relative slack for the FP32 distances.
    float t = 0.0f;
    if (d[1] < 0.0) {
        const float df[3] = {(float)d[0], (float)d[1], (float)d[2]};
        float inv[3];
        for (int a = 0; a < 3; ++a) inv[a] = (df[a] != 0.0f) ? Mth<float>::rcp(df[a]) : 0.0f;
        float tf = sc.cam_ym * inv[1];                              // the mirror cannot be met earlier
        if (sc.cloak || (opt_flags<OPT>(sc) & RT_FLAG_PLATE)) {
            float tn = -INFINITY, tx = INFINITY;
            bool miss = false;
            for (int a = 0; a < 3; ++a) {
                if (df[a] == 0.0f) {
                    if (sc.cam_lo[a] > 0.0f || sc.cam_hi[a] < 0.0f) miss = true;
                    continue;
                }
                const float t1 = sc.cam_lo[a] * inv[a], t2 = sc.cam_hi[a] * inv[a];
                tn = fmaxf(tn, fminf(t1, t2));
                tx = fminf(tx, fmaxf(t1, t2));
            }
            if (!miss && tn <= tx && tn > 0.0f && tn < tf) tf = tn;
        }
        tf = tf * (1.0f - 1e-5f) - 0.0009765625f;
        if (tf > 0.0f) t = tf;
    }
    const double Px = sc.C[0] + t * d[0];
    const double cxd = rint(Px);
    C.cx = (R)cxd;
    C.X = (R)(Px - cxd);
    C.y = (R)(sc.C[1] + t * d[1]);
    C.z = (R)(sc.C[2] + t * d[2]);
    set_air_dir_if(C, sc.cloak || (opt_flags<OPT>(sc) & RT_FLAG_PLATE), d[0], d[1], d[2]);
}

// Straight line against the flat mirror y = 0.
template <class R>
__device__ __forceinline__ R flat_line_hit(const Cold<R>& C)
{
    if (C.dy < R(0) && C.y > R(0)) return -C.y / C.dy;
    return R(INFINITY);
}

// First hit of the line with the trochoid of Eq. 2, or infinity.  From where
// the line enters the band |y| <= A it is marched in increments that move the
// point by at most 1/(8 pi) in the xy-plane, each increment taken from the
// end of the previous one (so the local coordinates stay small); the first
// increment ending at or below the surface brackets the hit, refined by
// Illinois.  On a hit, the hit point is returned in (hcx, hX, hy).
template <class R>
__device__ R trochoid_line_hit(const StepConst<R>& k, const Cold<R>& C, bool on_surface, R& hcx, R& hX, R& hy)
{
    const R A = k.A, kA = k.kA;
    const R dx = C.dx, dy = C.dy;
    const R dxy = Mth<R>::sqrt_(dx * dx + dy * dy);
    if (!(dxy > R(1e-30))) return R(INFINITY);
    if (dy >= R(0) && C.y >= A) return R(INFINITY);
    Cold<R> Q = C;
    R t0 = R(0);
    if (C.y > A) {
        t0 = (A - C.y) / dy;
        advance(Q, t0);
    }
    R L;
    if (dy < R(0)) L = (-A - Q.y) / dy;
    else if (dy > R(0)) L = (A - Q.y) / dy;
    else L = R(2) / fabs(dx);
    if (!(L >= R(0))) L = R(0);
    const R ds = R(0.25 * kInvTwoPi) / dxy;
    auto height = [&](R X, R y) -> R {
        const R E = trochoid_phase(X, kA);
        R sn, cs;
        Mth<R>::sincos(E, sn, cs);
        return y - A * cs;
    };
    // frame at the start of the current increment
    R fcx = Q.cx, fX = Q.X, fy = Q.y, s_a = R(0);
    bool first = on_surface && t0 == R(0);
    R ha;
    if (first) {
        const R E = trochoid_phase(fX, kA);
        R sn, cs;
        Mth<R>::sincos(E, sn, cs);
        const R slope = -kA * sn / (R(1) - kA * cs);
        ha = dy - slope * dx;
        if (!(ha > R(0))) ha = R(1e-30);
    } else {
        ha = height(fX, fy);
        if (ha <= R(0)) { hcx = fcx; hX = fX; hy = fy; return t0; }
    }
    for (int guard = 0; guard < (1 << 20); ++guard) {
        R u_b = fmin(ds, L - s_a);
        if (first && u_b <= Mth<R>::kRehit) {
            if (s_a + u_b >= L) return R(INFINITY);
            u_b = fmin(Mth<R>::kRehit, L - s_a);
        }
        if (!(u_b >= R(0))) return R(INFINITY);
        const bool last = !(s_a + u_b < L);
        R hb = height(fX + u_b * dx, fy + u_b * dy);
        if (last && dy < R(0) && hb > R(0)) hb = R(0);   // a descending line meets the surface by y = -A
        if (hb <= R(0)) {
            R u;
            if (first) {
                auto defl = [&](R v) -> R { return height(fX + v * dx, fy + v * dy) / v; };
                u = (u_b > R(0)) ? illinois_root(defl, R(0), ha, u_b, hb / u_b) : R(0);
            } else {
                auto hf = [&](R v) -> R { return height(fX + v * dx, fy + v * dy); };
                u = (u_b > R(0)) ? illinois_root(hf, R(0), ha, u_b, hb) : R(0);
            }
            R a = u * dx;
            const R n = Mth<R>::rint_(fX + a);
            hcx = fcx + n;
            hX = (fX - n) + a;
            hy = fy + u * dy;
            return t0 + s_a + u;
        }
        if (last) break;
        first = false;
        s_a += u_b;
        fX += u_b * dx;
        const R m = Mth<R>::rint_(fX);
        fcx += m;
        fX -= m;
        fy += u_b * dy;
        ha = hb;
    }
    return R(INFINITY);
}

// First hit of the line with the Gaussian bump, or infinity.  As for the
// trochoid, the part of the line in the band 0 <= y <= h is marched, in
// increments of w_b/8 in the xy-plane, and the first increment ending at or
// below the surface is refined by Illinois; the abscissa is absolute.  Only
// the core |x| <= 10 w_b + h is marched: beyond it the bump lies below
// h exp(-100), and a descending line meets the surface where it reaches
// y = 0.  On a hit the hit point is returned in (hcx, hX, hy).
template <class R>
__device__ R bump_line_hit(const StepConst<R>& k, const Cold<R>& C, bool on_surface, R& hcx, R& hX, R& hy)
{
    const R A = k.A;
    const R dx = C.dx, dy = C.dy;
    const R dxy = Mth<R>::sqrt_(dx * dx + dy * dy);
    if (!(dxy > R(1e-30))) return R(INFINITY);
    if (dy >= R(0) && C.y >= A) return R(INFINITY);
    R t0 = R(0), x0 = C.cx + C.X, y0 = C.y;
    if (C.y > A) {
        t0 = (A - C.y) / dy;
        x0 += t0 * dx;
        y0 = A;
    }
    const R xc = R(10) * k.gw + A;
    R L;
    if (dy < R(0)) L = -y0 / dy;
    else if (dy > R(0)) L = (A - y0) / dy;
    else L = (fabs(x0) + xc) / fabs(dx);
    if (!(L >= R(0))) L = R(0);
    // the part [va, vb] of [0, L] over the core
    R va = R(0), vb = L;
    if (dx != R(0)) {
        const R v1 = (-xc - x0) / dx, v2 = (xc - x0) / dx;
        va = fmax(va, fmin(v1, v2));
        vb = fmin(vb, fmax(v1, v2));
    } else if (fabs(x0) > xc) {
        vb = R(-1);
    }
    auto set_hit = [&](R v) {
        const R x = x0 + v * dx;
        const R m = Mth<R>::rint_(x);
        hcx = m;
        hX = x - m;
        hy = y0 + v * dy;
        return t0 + v;
    };
    auto height = [&](R v) -> R { return bump_height(k, x0 + v * dx, y0 + v * dy); };
    if (va < vb) {
        const R ds = R(0.125) * k.gw / dxy;
        bool first = on_surface && t0 == R(0) && va == R(0);
        R s_a = va, ha;
        if (first) {
            R tx, ty;
            bump_tangent(k, bump_u(k, x0), tx, ty);
            ha = dy - (ty / tx) * dx;
            if (!(ha > R(0))) ha = R(1e-30);
        } else {
            ha = height(s_a);
            if (ha <= R(0)) return set_hit(s_a);
        }
        for (int guard = 0; guard < (1 << 20); ++guard) {
            R u_b = fmin(ds, vb - s_a);
            if (first && u_b <= Mth<R>::kRehit) {
                if (s_a + u_b >= vb) break;
                u_b = fmin(Mth<R>::kRehit, vb - s_a);
            }
            if (!(u_b >= R(0))) break;
            const bool last = !(s_a + u_b < vb);
            R hb = height(s_a + u_b);
            if (last && vb == L && dy < R(0) && hb > R(0)) hb = R(0);   // the line reaches y = 0 here
            if (hb <= R(0)) {
                R u;
                if (first) {
                    auto defl = [&](R v) -> R { return height(s_a + v) / v; };
                    u = (u_b > R(0)) ? illinois_root(defl, R(0), ha, u_b, hb / u_b) : R(0);
                } else {
                    auto hf = [&](R v) -> R { return height(s_a + v); };
                    u = (u_b > R(0)) ? illinois_root(hf, R(0), ha, u_b, hb) : R(0);
                }
                return set_hit(s_a + u);
            }
            if (last) break;
            first = false;
            s_a += u_b;
            ha = hb;
        }
    }
    // no hit over the core: a descending line meets the flat part at y = 0
    if (dy < R(0) && !(on_surface && t0 == R(0) && L <= Mth<R>::kRehit)) return set_hit(L);
    return R(INFINITY);
}

// Entry of the line into the cloak box (slab method), infinity if it misses.
template <class R>
__device__ __forceinline__ R box_entry(const StepConst<R>& k, const Cold<R>& C, int& face)
{
    const R pos[3] = {C.X, C.y, C.z};
    const R dir[3] = {C.dx, C.dy, C.dz};
    const R lo[3] = {-k.E2 - C.cx, k.ybot, -k.E2}, hi[3] = {k.E2 - C.cx, k.ytop, k.E2};
    const int flo[3] = {EV_XM, EV_NONE, EV_ZM}, fhi[3] = {EV_XP, EV_TOP, EV_ZP};
    R tn = R(-INFINITY), tf = R(INFINITY);
    int fn = EV_NONE;
    for (int a = 0; a < 3; ++a) {
        if (dir[a] == R(0)) {
            if (pos[a] < lo[a] || pos[a] > hi[a]) return R(INFINITY);
            continue;
        }
        const R inv = R(1) / dir[a];
        const R t1 = (lo[a] - pos[a]) * inv, t2 = (hi[a] - pos[a]) * inv;
        R tmin = t1, tmax = t2;
        int f = flo[a];
        if (t1 > t2) { tmin = t2; tmax = t1; f = fhi[a]; }
        if (tmin > tn) { tn = tmin; fn = f; }
        if (tmax < tf) tf = tmax;
    }
    if (!(tn <= tf) || !(tn > R(64) * Mth<R>::kEps)) return R(INFINITY);
    face = fn;
    return tn;
}

// Background plane standing in for the photograph (Sec. 4, Fig. 2a).
template <class R>
__device__ __forceinline__ int background(const DevScene& sc, const AirConst<R>& a, const Cold<R>& C, float col[3])
{
    col[0] = col[1] = col[2] = 0.0f;
    const R d[3] = {C.dx, C.dy, C.dz};
    const R X[3] = {C.cx + C.X, C.y, C.z};
    const R dn = d[0] * a.fr[0] + d[1] * a.fr[1] + d[2] * a.fr[2];
    if (!(dn > R(0))) return RT_RAY_SKY;
    const R t = ((a.Pb[0] - X[0]) * a.fr[0] + (a.Pb[1] - X[1]) * a.fr[1] + (a.Pb[2] - X[2]) * a.fr[2]) / dn;
    R Y[3];
    for (int q = 0; q < 3; ++q) Y[q] = X[q] + t * d[q] - a.Pb[q];
    const R s = Y[0] * a.r[0] + Y[1] * a.r[1] + Y[2] * a.r[2];
    const R tt = Y[0] * a.ur[0] + Y[1] * a.ur[1] + Y[2] * a.ur[2];
    if (sc.background == RT_BG_CHECKER) {
        const long long u = (long long)floor(s * a.inv_cell), v = (long long)floor(tt * a.inv_cell);
        const float* c = (((u + v) & 1LL) == 0) ? sc.col0 : sc.col1;
        col[0] = c[0]; col[1] = c[1]; col[2] = c[2];
    } else {
        const int N = sc.tex_size;
        const R U = s * a.inv_texel - R(0.5), V = tt * a.inv_texel - R(0.5);
        const R fu0 = floor(U), fv0 = floor(V);
        const float fu = (float)(U - fu0), fv = (float)(V - fv0);
        long long u0 = (long long)fu0 % N, v0 = (long long)fv0 % N;
        if (u0 < 0) u0 += N;
        if (v0 < 0) v0 += N;
        const long long u1 = (u0 + 1 == N) ? 0 : u0 + 1, v1 = (v0 + 1 == N) ? 0 : v0 + 1;
        const float t00 = RT_TEX_LOAD(sc.tex + v0 * N + u0), t01 = RT_TEX_LOAD(sc.tex + v0 * N + u1);
        const float t10 = RT_TEX_LOAD(sc.tex + v1 * N + u0), t11 = RT_TEX_LOAD(sc.tex + v1 * N + u1);
        const float val = (1.0f - fu) * (1.0f - fv) * t00 + fu * (1.0f - fv) * t01 + (1.0f - fu) * fv * t10 +
                          fu * fv * t11;
        col[0] = col[1] = col[2] = val;
    }
    return RT_RAY_OK;
}

template <class R, bool OPT>
__device__ __forceinline__ void finish_sample(const DevScene& sc, Cold<R>& C, int steps, int status, int& phase,
                                              rt_ray_record* rec)
{
    if (status != RT_RAY_OK && status != RT_RAY_SKY) C.col[0] = C.col[1] = C.col[2] = 0.0f;
    if (opt_flags<OPT>(sc) & RT_FLAG_FRESNEL) {
        // an explicit FMA: the same rounding in every kernel that inlines this
        const float w = (float)C.w;
        C.acc[0] = fmaf(w, C.col[0], C.acc[0]);
        C.acc[1] = fmaf(w, C.col[1], C.acc[1]);
        C.acc[2] = fmaf(w, C.col[2], C.acc[2]);
    } else {
        C.acc[0] += C.col[0];
        C.acc[1] += C.col[1];
        C.acc[2] += C.col[2];
    }
    phase = PH_DONE;
    if (OPT && C.path != 0) return;                 // a Fresnel branch: no record, no ray of its own
    C.status = status;
    C.rays += 1;
    C.stat[status < 5 ? status : 4] += 1;
    if (rec) {
        rt_ray_record* o = rec + C.work * sc.spp + C.sample;
        const double pos[3] = {(double)C.cx + (double)C.X, (double)C.y, (double)C.z};
        double d[3];
        air_dir(C, d);
        const double l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int a = 0; a < 3; ++a) {
            o->pos[a] = pos[a] * sc.Lambda;
            o->dir[a] = d[a] / l;
            o->rgb[a] = C.col[a];
        }
        o->status = status;
        o->bounces = C.bounces;
        o->events = C.events;
        o->steps = steps;
    }
    phase = PH_DONE;
}

// Copy a ray in the cloak to the air state (position and unit direction).
template <class R>
__device__ __forceinline__ void box_to_air(Cold<R>& C, const Box<R>& b, const R d[3])
{
    C.cx = b.cx;
    C.X = b.X;
    C.y = b.y;
    C.z = b.z;
    const R il = R(1) / Mth<R>::sqrt_(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    set_air_dir_r(C, d[0] * il, d[1] * il, d[2] * il);
}

// Inside the homogeneous plate of RT_FLAG_PLATE (index 1 + kA on the flat
// mirror, filling the box from y = 0 to its top): straight segments in FP64
// from P with momentum q (|q| = n_plate) to the mirror (reflection), the top
// or a side face (refraction into air, or total internal reflection).  On the
// way out the air state of C is set and true returned; false when the path
// ended inside (bounce guard), with phase = PH_DONE.
template <class R, bool OPT>
__device__ bool plate_traverse(const DevScene& sc, Cold<R>& C, double P[3], double q[3], int steps, int& phase,
                               rt_ray_record* rec)
{
    const double lo[3] = {-sc.E2, 0.0, -sc.E2}, hi[3] = {sc.E2, sc.ytop, sc.E2};
    for (;;) {
        int hit = EV_NONE;
        double tmin = INFINITY;
        if (C.bounces <= sc.max_bounces) {
            for (int a = 0; a < 3; ++a) {
                if (q[a] == 0.0) continue;
                const double t = ((q[a] > 0.0 ? hi[a] : lo[a]) - P[a]) / q[a];
                if (t < tmin) {
                    tmin = t;
                    hit = (a == 0) ? (q[a] > 0.0 ? EV_XP : EV_XM)
                                   : (a == 1 ? (q[a] > 0.0 ? EV_TOP : EV_GRATING) : (q[a] > 0.0 ? EV_ZP : EV_ZM));
                }
            }
        }
        if (hit == EV_NONE) {                  // bounce guard (or no direction): report where it is
            const double cxd = rint(P[0]);
            const double ql = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
            C.cx = (R)cxd; C.X = (R)(P[0] - cxd); C.y = (R)P[1]; C.z = (R)P[2];
            set_air_dir(C, q[0] / ql, q[1] / ql, q[2] / ql);
            finish_sample<R, OPT>(sc, C, steps, C.bounces > sc.max_bounces ? RT_RAY_MAX_BOUNCES : RT_RAY_NAN, phase, rec);
            return false;
        }
        if (tmin < 0.0) tmin = 0.0;
        for (int a = 0; a < 3; ++a) P[a] += tmin * q[a];
        if (hit == EV_GRATING) {               // the mirror under the plate
            P[1] = 0.0;
            q[1] = -q[1];
            C.bounces++;
            continue;
        }
        R Nf[3];
        face_normal(hit, Nf);
        const double N[3] = {(double)Nf[0], (double)Nf[1], (double)Nf[2]};
        const double pn = q[0] * N[0] + q[1] * N[1] + q[2] * N[2];
        double pt[3];
        for (int a = 0; a < 3; ++a) pt[a] = q[a] - pn * N[a];
        const double pt2 = pt[0] * pt[0] + pt[1] * pt[1] + pt[2] * pt[2];
        if (pt2 >= 1.0) {                      // total internal reflection
            for (int a = 0; a < 3; ++a) q[a] -= 2.0 * pn * N[a];
            C.bounces++;
            continue;
        }
        const double pout = sqrt(1.0 - pt2);
        const double cxd = rint(P[0]);
        C.cx = (R)cxd; C.X = (R)(P[0] - cxd); C.y = (R)P[1]; C.z = (R)P[2];
        if (opt_flags<OPT>(sc) & RT_FLAG_FRESNEL)
            fresnel_split(C, fresnel_R(sc.plate_n, 1.0, pn, pout), MED_PLATE, C.cx, C.X, C.y, C.z,
                          q[0] - 2.0 * pn * N[0], q[1] - 2.0 * pn * N[1], q[2] - 2.0 * pn * N[2], hit, steps);
        set_air_dir(C, pt[0] + pout * N[0], pt[1] + pout * N[1], pt[2] + pout * N[2]);
        return true;
    }
}

template <class R, int INTEG, bool OPT>
__device__ void air_segment(const DevScene& sc, Cold<R>& C, Box<R>& b, int& phase, int& surf, int steps,
                            rt_ray_record* rec, LaneStats& st)
{
    const StepConst<R>& k = step_const<R>(sc);
    const bool plate = (opt_flags<OPT>(sc) & RT_FLAG_PLATE) != 0;
    if (OPT && C.in_plate) {
        // a Fresnel branch that starts inside the plate: C holds its position and momentum
        C.in_plate = 0;
        double P[3] = {(double)C.cx + (double)C.X, (double)C.y, (double)C.z};
        double q[3];
        air_dir(C, q);
        if (!plate_traverse<R, OPT>(sc, C, P, q, steps, phase, rec)) return;
        surf = EV_NONE;
    }
    for (;;) {
        if (C.bounces > sc.max_bounces) { finish_sample<R, OPT>(sc, C, steps, RT_RAY_MAX_BOUNCES, phase, rec); return; }
        R hcx = R(0), hX = R(0), hy = R(0);
        R tm;
        if constexpr (gauss_of(INTEG))
            tm = sc.mirror ? bump_line_hit(k, C, surf == EV_GRATING, hcx, hX, hy) : flat_line_hit(C);
        else
            tm = sc.mirror ? trochoid_line_hit(k, C, surf == EV_GRATING, hcx, hX, hy) : flat_line_hit(C);
        int face = EV_NONE;
        const R tb = (sc.cloak || plate) ? box_entry(k, C, face) : R(INFINITY);
        if (tb < tm) {
            advance(C, tb);
            R Nf[3];
            face_normal(face, Nf);
            double d[3];
            air_dir(C, d);
            const double N[3] = {(double)Nf[0], (double)Nf[1], (double)Nf[2]};
            const double pn = d[0] * N[0] + d[1] * N[1] + d[2] * N[2];
            double pt[3];
            for (int a = 0; a < 3; ++a) pt[a] = d[a] - pn * N[a];
            const double pt2 = pt[0] * pt[0] + pt[1] * pt[1] + pt[2] * pt[2];
            if (plate) {
                // into the denser plate (no total reflection), then straight through it
                const double npl = sc.plate_n;
                const double pin = sqrt(npl * npl - pt2);
                if (opt_flags<OPT>(sc) & RT_FLAG_FRESNEL)
                    fresnel_split(C, fresnel_R(1.0, npl, pn, pin), MED_AIR, C.cx, C.X, C.y, C.z,
                                  d[0] - 2.0 * pn * N[0], d[1] - 2.0 * pn * N[1], d[2] - 2.0 * pn * N[2], EV_NONE,
                                  steps);
                double P[3] = {(double)C.cx + (double)C.X, (double)C.y, (double)C.z};
                double q[3] = {pt[0] - pin * N[0], pt[1] - pin * N[1], pt[2] - pin * N[2]};
                if (!plate_traverse<R, OPT>(sc, C, P, q, steps, phase, rec)) return;
                surf = EV_NONE;
                continue;
            }
            b.cx = C.cx;
            b.X = C.X;
            if constexpr (gauss_of(INTEG)) {  // the Gaussian box works with the absolute abscissa
                b.cx = R(0);
                b.X = C.cx + C.X;
            }
            b.y = C.y;
            b.z = C.z;
            b.wr = b.wi = R(0);
            med_solve<R, INTEG>(k, b.X, b.y, b.wr, b.wi, b.rr, b.ri, b.Fx, b.Fy, st);
            // Snell's law in FP64 (a few operations per entry): sqrt(n^2 - |p_t|^2)
            // is ill-conditioned near grazing incidence; the index is scaled
            // by idx_scale in the referenced cloak.  The grating's n^2 =
            // 1/|1 + W0|^2 is formed in FP64 from W0: near the top of the box
            // |W0| is ~1e-6, and 1 + W0 rounded to FP32 would leave n with a
            // relative error of 6e-8, which the shallow entries of the
            // camera rays turn into 2e-7 of momentum
            double n2;
            if constexpr (gauss_of(INTEG)) {
                n2 = (double)b.rr * (double)b.rr + (double)b.ri * (double)b.ri;
            } else {
                const double ar = 1.0 + (double)b.wr, ai = (double)b.wi;
                n2 = recip_nr(ar * ar + ai * ai);
            }
            if (opt_flags<OPT>(sc) & RT_FLAG_REFERENCED) n2 *= sc.idx_scale * sc.idx_scale;
            if (n2 < pt2) {      // total reflection off the outside of the box
                set_air_dir(C, d[0] - 2.0 * pn * N[0], d[1] - 2.0 * pn * N[1], d[2] - 2.0 * pn * N[2]);
                C.bounces++;
                surf = EV_NONE;
                continue;
            }
            const double pin = sqrt(n2 - pt2);
            if (opt_flags<OPT>(sc) & RT_FLAG_FRESNEL)
                fresnel_split(C, fresnel_R(1.0, sqrt(n2), pn, pin), MED_AIR, C.cx, C.X, C.y, C.z,
                              d[0] - 2.0 * pn * N[0], d[1] - 2.0 * pn * N[1], d[2] - 2.0 * pn * N[2], EV_NONE, steps);
            // the momentum |p| = n inside; the time form carries v = p / n^2
            // (the FP32 path keeps the rounding of p_x, p_y in their
            // compensation terms, which hold p - exact)
            const double iv = (integ_of(INTEG) == RT_RK4T) ? 1.0 / n2 : 1.0;
            const double qx = (pt[0] - pin * N[0]) * iv, qy = (pt[1] - pin * N[1]) * iv;
            b.px = (R)qx;
            b.py = (R)qy;
            b.pz = (R)((pt[2] - pin * N[2]) * iv);
            b.cX = b.cy = b.cz = R(0);
            b.cpx = (R)((double)b.px - qx);
            b.cpy = (R)((double)b.py - qy);
            b.hc = k.h;
            med_force<R, INTEG>(k, b);
            surf = face;
            phase = PH_BOX;
            return;
        }
        if (tm < R(INFINITY)) {
            if (sc.mirror) {
                C.z += tm * C.dz;
                C.cx = hcx;
                C.X = hX;
                C.y = hy;
                // upward normal from the tangent of Eq. 2 at the phase of the
                // hit (of the bump's parametric form for the Gaussian bump)
                double nx, ny;
                if constexpr (gauss_of(INTEG)) {
                    R tx, ty;
                    bump_tangent(k, bump_u(k, C.cx + C.X), tx, ty);
                    nx = -(double)ty;
                    ny = (double)tx;
                } else {
                    const R E = trochoid_phase(C.X, k.kA);
                    R sn, cs;
                    Mth<R>::sincos(E, sn, cs);
                    nx = (double)k.kA * (double)sn;
                    ny = 1.0 - (double)k.kA * (double)cs;
                }
                const double il = rsqrt_nr(nx * nx + ny * ny);
                double d[3];
                air_dir(C, d);
                const double pn = (d[0] * nx + d[1] * ny) * il;
                set_air_dir_if(C, sc.cloak || plate, d[0] - 2.0 * pn * nx * il, d[1] - 2.0 * pn * ny * il, d[2]);
            } else {
                advance(C, tm);
                C.y = R(0);
                C.dy = -C.dy;
                C.dl[1] = -C.dl[1];
            }
            C.bounces++;
            surf = EV_GRATING;
            continue;
        }
        const int status = background(sc, air_const<R>(sc), C, C.col);
        finish_sample<R, OPT>(sc, C, steps, status, phase, rec);
        return;
    }
}

// ------------------------------------------------------------------------
// Service of a lane whose step crossed a surface (or hit a guard).
// ------------------------------------------------------------------------
// The FP32 RK4 steps in the grating cloak (in tau or, for Eq. 11, in t) are
// committed in place, also when they crossed a surface: the event service
// then rebuilds the step's start as one step of -h from its end
// (rebuild_start).  Keeping the start live through
// every step, for the one step in hundreds that crosses, costs a conditional
// copy of the whole state per step.  The rebuilt start differs from the true
// one by the integrator's local error, O(h^5): at h = Lambda/200 in the
// benchmark cloak (kA = 3/8), a forward and a backward step of the FP64
// oracle return within 7e-10 Lambda in position and 4e-8 in momentum, about
// one FP32 rounding of the momentum.  FP64 keeps the start (its rays match
// the oracle's to 1e-12), and so does the Gaussian medium, whose rebuilt
// start put the FP32 render's well-conditioned rays below the parity bar
// (99.75 % against 99.9 %).
template <class R, int INTEG>
__host__ __device__ constexpr bool back_start()
{
    return sizeof(R) == 4 && (integ_of(INTEG) == RT_RK4 || integ_of(INTEG) == RT_RK4T) && !gauss_of(INTEG);
}

// The start of the step that ended at b (back_start): one step of -h, the
// grating's force formed as at the end of a step (the Gaussian step returns
// its own).
template <class R, int INTEG>
__device__ __forceinline__ void rebuild_start(const StepConst<R>& k, Box<R>& b, R h, LaneStats& st)
{
    Box<R> s0;
    integ_step<R, INTEG>(k, b, -h, s0, st);
    if constexpr (!gauss_of(INTEG)) ray_force(s0.wr, s0.wi, s0.rr, s0.ri, k.fk, s0.Fx, s0.Fy);
    b = s0;
}

template <class R, int INTEG, bool OPT>
__device__ void service_event(const DevScene& sc, Cold<R>& C, Box<R>& b, int& phase, int& surf, int steps,
                              rt_ray_record* rec, LaneStats& st)
{
    const StepConst<R>& k = step_const<R>(sc);
    const R p0[3] = {b.px, b.py, b.pz};
    if (phase == PH_GUARD) {
        box_to_air(C, b, p0);
        finish_sample<R, OPT>(sc, C, steps, RT_RAY_MAX_STEPS, phase, rec);
        return;
    }
    bool finite = true;
    for (int ev = 0; ev < EV_COUNT; ++ev) finite = finite && isfinite(C.g1[ev]);
    if (!finite || !(isfinite(b.X) && isfinite(b.y) && isfinite(b.px) && isfinite(b.py))) {
        box_to_air(C, b, p0);
        finish_sample<R, OPT>(sc, C, steps, RT_RAY_NAN, phase, rec);
        return;
    }
    if constexpr (back_start<R, INTEG>()) rebuild_start<R, INTEG>(k, b, C.hs, st);   // b held the step's end
    int ev_best = EV_NONE, last = EV_NONE;
    R th_best = R(2);
    Box<R> t;
    for (int ev = 0; ev < EV_COUNT; ++ev) {
        if (C.g1[ev] < R(0)) {
            const R th = locate_event<R, INTEG>(k, b, C.hs, ev, surf == ev, C.g1[ev], t, st);
            last = ev;
            if (th < th_best) { th_best = th; ev_best = ev; }
        }
    }
    if (last != ev_best) {
        integ_step<R, INTEG>(k, b, th_best * C.hs, t, st);
        if constexpr (resolve_end<R, INTEG>())
            med_solve<R, INTEG>(k, t.X, t.y, t.wr, t.wi, t.rr, t.ri, t.Fx, t.Fy, st);
    }
    const R hc = b.hc;
    b = t;
    b.hc = hc;
    med_force<R, INTEG>(k, b);
    C.events++;
    C.nevents++;
    if (ev_best == EV_GRATING) {
        // mirror reflection about grad v / |grad v| = (Im r, Re r) / |r|, in
        // FP64 on the compensated momentum; for the grating r = 1/(1 + W0),
        // so the normal is along (-Im W0, 1 + Re W0), formed from W0 itself
        double nx, ny;
        if constexpr (gauss_of(INTEG)) {
            nx = (double)b.ri;
            ny = (double)b.rr;
        } else {
            nx = -(double)b.wi;
            ny = 1.0 + (double)b.wr;
        }
        const double il = rsqrt_nr(nx * nx + ny * ny);
        nx *= il;
        ny *= il;
        const double vx = (double)b.px - (double)b.cpx, vy = (double)b.py - (double)b.cpy;
        const double pn = vx * nx + vy * ny;
        const double ox = vx - 2.0 * pn * nx, oy = vy - 2.0 * pn * ny;
        b.px = (R)ox;
        b.py = (R)oy;
        b.cpx = (R)((double)b.px - ox);
        b.cpy = (R)((double)b.py - oy);
        C.bounces++;
        surf = EV_GRATING;
        phase = PH_BOX;
        if (C.bounces > sc.max_bounces) {
            const R p[3] = {b.px, b.py, b.pz};
            box_to_air(C, b, p);
            finish_sample<R, OPT>(sc, C, steps, RT_RAY_MAX_BOUNCES, phase, rec);
        }
        return;
    }
    // a face: refract into air (n = 1) or reflect totally; Snell's law in
    // FP64 since sqrt(1 - |p_t|^2) is ill-conditioned near grazing exit
    // (the time form converts its velocity to the momentum p = n^2 v first)
    R Nf[3];
    face_normal(ev_best, Nf);
    // The momentum with its compensation term (the compensated sum carries
    // the rounding of the FP32 sum: the exact sum is p - c); the time form's
    // n^2 from W0 in FP64, as at the entry
    double n2f = 1.0;
    if constexpr (integ_of(INTEG) == RT_RK4T) {
        if constexpr (gauss_of(INTEG)) {
            n2f = ((double)b.rr * (double)b.rr + (double)b.ri * (double)b.ri) / (double)k.is2;
        } else {
            const double ar = 1.0 + (double)b.wr, ai = (double)b.wi;
            n2f = 1.0 / ((ar * ar + ai * ai) * (double)k.is2);
        }
    }
    const double v[3] = {(double)b.px - (double)b.cpx, (double)b.py - (double)b.cpy, (double)b.pz};
    const double p[3] = {v[0] * n2f, v[1] * n2f, v[2] * n2f};
    const double N[3] = {(double)Nf[0], (double)Nf[1], (double)Nf[2]};
    const double pn = p[0] * N[0] + p[1] * N[1] + p[2] * N[2];
    double pt[3];
    for (int a = 0; a < 3; ++a) pt[a] = p[a] - pn * N[a];
    const double pt2 = pt[0] * pt[0] + pt[1] * pt[1] + pt[2] * pt[2];
    if (pt2 >= 1.0) {
        const double vn = pn / n2f;
        const double vx = v[0] - 2.0 * vn * N[0], vy = v[1] - 2.0 * vn * N[1];
        b.px = (R)vx;
        b.py = (R)vy;
        b.pz = (R)(v[2] - 2.0 * vn * N[2]);
        b.cpx = (R)((double)b.px - vx);
        b.cpy = (R)((double)b.py - vy);
        C.bounces++;
        surf = ev_best;
        phase = PH_BOX;
        if (C.bounces > sc.max_bounces) {
            const R q[3] = {b.px, b.py, b.pz};
            box_to_air(C, b, q);
            finish_sample<R, OPT>(sc, C, steps, RT_RAY_MAX_BOUNCES, phase, rec);
        }
        return;
    }
    const double pout = sqrt(1.0 - pt2);
    if (opt_flags<OPT>(sc) & RT_FLAG_FRESNEL) {
        // the reflected branch stays in the cloak, starting on this face
        const double n1 = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);   // |p| = n
        fresnel_split(C, fresnel_R(n1, 1.0, pn, pout), MED_BOX, b.cx, b.X, b.y, b.z, p[0] - 2.0 * pn * N[0],
                      p[1] - 2.0 * pn * N[1], p[2] - 2.0 * pn * N[2], ev_best, steps);
    }
    double d[3], l2 = 0.0;
    for (int a = 0; a < 3; ++a) { d[a] = pt[a] + pout * N[a]; l2 += d[a] * d[a]; }
    const double il = rsqrt_nr(l2);
    C.cx = b.cx;
    C.X = b.X;
    if constexpr (gauss_of(INTEG)) {          // back to cell + fraction in air
        const R m = Mth<R>::rint_(b.X);
        C.cx = m;
        C.X = b.X - m;
    }
    C.y = b.y;
    C.z = b.z;
    set_air_dir(C, d[0] * il, d[1] * il, d[2] * il);
    surf = EV_NONE;
    phase = PH_AIR;
}

// ------------------------------------------------------------------------
// The integration step of the hot loop.
// ------------------------------------------------------------------------
// One step from s into o.  Accepted (phase stays PH_BOX): the new state is in
// o.  A rejected Dormand-Prince attempt also leaves phase at PH_BOX, with o a
// copy of s and a smaller next step.  A step that crosses a surface or goes
// non-finite (PH_EVENT) leaves the step's end in o: box_step keeps s for the
// event service, except on the back_start paths, which keep o and rebuild s
// from it.  A step cap reached (PH_GUARD) leaves o undefined.
// RK4 in the grating cloak skips the box faces' tests while the ray is
// farther from every face than `safe` steps can move it (isafe: one over the
// largest move of a step); the grating's test runs every step.
template <int INTEG>
__host__ __device__ constexpr bool face_skip() { return integ_of(INTEG) == RT_RK4 && !gauss_of(INTEG); }

template <class R>
__device__ __forceinline__ int safe_steps(const StepConst<R>& k, const Box<R>& o)
{
    const R dx = k.E2 - fabs(o.cx + o.X), dz = k.E2 - fabs(o.z), dy = k.ytop - o.y;
    const R d = fmin(dy, fmin(dx, dz));
    return (int)(d * k.isafe) - 1;
}

template <class R, int INTEG>
__device__ __forceinline__ void box_step_into(const StepConst<R>& k, int64_t max_steps, Cold<R>& C, Box<R>& s,
                                              Box<R>& o, int& phase, int& surf, int& steps, LaneStats& st,
                                              int& safe)
{
    if (steps >= max_steps) {
        phase = PH_GUARD;
        return;
    }
    R hs;
    if constexpr (integ_of(INTEG) == RT_DP45) {
        // one attempt of an adaptive Dormand-Prince step; a rejected attempt
        // only shrinks the step
        hs = s.hc;
        R e[4];
        dp45_step<R, INTEG>(k, s, hs, o, e, st);
        ++steps;
        st.steps++;
        const R scp = k.atol + k.rtol;                                    // positions (units of Lambda)
        const R s2 = k.atol + k.rtol * fmax(fabs(s.px), fabs(o.px));
        const R s3 = k.atol + k.rtol * fmax(fabs(s.py), fabs(o.py));
        R err, fac;
        if constexpr (sizeof(R) == 4) {
            // FP32: reciprocals and err^-1/5 = (err^2)^-1/10 on the MUFU pipe
            // (the step factor is a heuristic; a few ulp do not matter)
            const R iscp = Mth<R>::rcp(scp);
            const R q0 = e[0] * iscp, q1 = e[1] * iscp, q2 = e[2] * Mth<R>::rcp(s2), q3 = e[3] * Mth<R>::rcp(s3);
            const R err2 = R(0.25) * (q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
            err = err2;                                                   // err <= 1 iff err^2 <= 1
            fac = (err2 > R(0)) ? R(0.9) * Mth<R>::ex2(R(-0.1) * Mth<R>::lg2(err2)) : R(5);
        } else {
            const R q0 = e[0] / scp, q1 = e[1] / scp, q2 = e[2] / s2, q3 = e[3] / s3;
            err = Mth<R>::sqrt_(R(0.25) * (q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3));
            fac = (err > R(0)) ? R(0.9) * pow(err, R(-0.2)) : R(5);
        }
        fac = fmin(R(5), fmax(R(0.2), fac));
        if (!(err <= R(1))) {
            if (!isfinite(err)) {
                for (int q = 0; q < EV_COUNT; ++q) C.g1[q] = R(NAN);
                C.hs = hs;
                phase = PH_EVENT;
                return;
            }
            o = s;
            o.hc = fmin(hs * fmin(fac, R(1)), k.hmax);
            return;
        }
        o.hc = fmin(hs * fac, k.hmax);
    } else {
        hs = k.h;
        if constexpr (integ_of(INTEG) == RT_RK4T) rk4t_step<R, INTEG>(k, s, hs, o, st);
        else rk4_step<R, INTEG>(k, s, hs, o, st);
        // W (and the Gaussian medium's force) at the end point come from the
        // step; the grating's force is formed here
        if constexpr (!gauss_of(INTEG)) ray_force(o.wr, o.wi, o.rr, o.ri, k.fk, o.Fx, o.Fy);
        ++steps;
        st.steps++;
    }
    const R gG = o.y + o.wr * R(kInvTwoPi);
    if constexpr (face_skip<INTEG>()) {
        if (safe > 0 && gG >= R(0)) {
            --safe;
            surf = EV_NONE;
            return;
        }
    }
    const R gT = k.ytop - o.y;
    const R gXp = (k.E2 - o.cx) - o.X, gXm = (k.E2 + o.cx) + o.X;
    const R gZp = k.E2 - o.z, gZm = k.E2 + o.z;
    if (gG >= R(0) && gT >= R(0) && gXp >= R(0) && gXm >= R(0) && gZp >= R(0) && gZm >= R(0)) {
        surf = EV_NONE;
        if constexpr (face_skip<INTEG>()) safe = safe_steps(k, o);
        return;
    }
    // crossed a surface (or went non-finite): the service pass locates it from s
    C.g1[EV_GRATING] = gG;
    C.g1[EV_TOP] = gT;
    C.g1[EV_XP] = gXp;
    C.g1[EV_XM] = gXm;
    C.g1[EV_ZP] = gZp;
    C.g1[EV_ZM] = gZm;
    C.hs = hs;
    if constexpr (integ_of(INTEG) == RT_DP45) s.hc = o.hc;
    phase = PH_EVENT;
}

// One step of b in place.
template <class R, int INTEG>
__device__ __forceinline__ void box_step(const StepConst<R>& k, int64_t max_steps, Cold<R>& C, Box<R>& b, int& phase,
                                         int& surf, int& steps, LaneStats& st, int& safe)
{
    if constexpr (back_start<R, INTEG>()) {
        if (steps >= max_steps) {
            phase = PH_GUARD;
            return;
        }
        Box<R> o;
        box_step_into<R, INTEG>(k, max_steps, C, b, o, phase, surf, steps, st, safe);
        b = o;
    } else {
        Box<R> o;
        box_step_into<R, INTEG>(k, max_steps, C, b, o, phase, surf, steps, st, safe);
        if (phase == PH_BOX) b = o;
    }
}

// ------------------------------------------------------------------------
// Work distribution and the persistent loop.
// ------------------------------------------------------------------------
// Warp-aggregated grab of one work item per calling lane: one atomic for the
// lanes that arrive together.
__device__ __forceinline__ int64_t grab_work(unsigned long long* counter, unsigned lane)
{
    const unsigned m = __activemask();
    const int leader = __ffs(m) - 1;
    const unsigned rank = __popc(m & ((1u << lane) - 1u));
    unsigned long long base = 0;
    if ((int)lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
    base = __shfl_sync(m, base, leader);
    return (int64_t)(base + rank);
}

template <class R, bool OPT>
__device__ __forceinline__ void start_sample(const DevScene& sc, Cold<R>& C, int& phase, int& surf, int& steps)
{
    camera_start<R, OPT>(sc, C);
    C.bounces = 0;
    C.events = 0;
    C.w = R(1);
    C.path = 0;
    C.nbr = 0;
    C.ibr = 0;
    C.in_plate = 0;
    C.col[0] = C.col[1] = C.col[2] = 0.0f;
    surf = EV_NONE;
    steps = 0;
    phase = PH_AIR;
}

// Start the next queued Fresnel branch of the sample in place of the path
// that just ended (phase becomes PH_AIR or PH_BOX).
template <class R, int INTEG>
__device__ void start_branch(const DevScene& sc, Cold<R>& C, Box<R>& b, int& phase, int& surf, int& steps,
                             LaneStats& st)
{
    const Branch<R> q = C.br[C.ibr++];
    C.path = C.ibr;
    C.w = q.w;
    C.bounces = q.bounces;
    C.events = q.events;
    C.col[0] = C.col[1] = C.col[2] = 0.0f;
    steps = q.steps;
    surf = q.surf;
    if (q.medium == MED_BOX) {
        const StepConst<R>& k = step_const<R>(sc);
        b.cx = q.cx;
        b.X = q.X;
        b.y = q.y;
        b.z = q.z;
        b.px = q.p[0];
        b.py = q.p[1];
        b.pz = q.p[2];
        b.cX = b.cy = b.cz = b.cpx = b.cpy = R(0);
        b.wr = b.wi = R(0);
        med_solve<R, INTEG>(k, b.X, b.y, b.wr, b.wi, b.rr, b.ri, b.Fx, b.Fy, st);
        med_force<R, INTEG>(k, b);
        if constexpr (integ_of(INTEG) == RT_RK4T) {
            // the branch holds the momentum; the time form carries v = p / n^2
            const double iv = (double)k.is2 / ((double)b.rr * (double)b.rr + (double)b.ri * (double)b.ri);
            b.px = (R)((double)q.p[0] * iv);
            b.py = (R)((double)q.p[1] * iv);
            b.pz = (R)((double)q.p[2] * iv);
        }
        b.hc = k.h;
        phase = PH_BOX;
    } else {
        C.cx = q.cx;
        C.X = q.X;
        C.y = q.y;
        C.z = q.z;
        set_air_dir_r(C, q.p[0], q.p[1], q.p[2]);
        C.in_plate = (q.medium == MED_PLATE);
        phase = PH_AIR;
    }
}

__device__ __forceinline__ uint8_t quantize8(float c)
{
    float v = c > 0.0f ? c : 0.0f;
    v = v < 1.0f ? v : 1.0f;
    return (uint8_t)floorf(v * 255.0f + 0.5f);
}

// Where the work of a launch comes from: one scene (constants in the kernel
// parameters) or a table of scenes whose pixels are numbered one after the
// other (constants in device memory).
// Pixels are numbered by work item (w), samples by w * spp + sample; the
// wavefront loop takes samples as its work items, the per-lane loop pixels.
// Samples of one pixel traced by different lanes leave their colours in the
// pixel's block of samp_col (col_block_bytes, from the scene's col_base on)
// and count themselves in pix_cnt (one int per pixel, zero at launch); the
// last one sums them in sample order.
struct OneScene {
    static constexpr bool kParamScene = true;    // the scene lives in the kernel parameters
    const DevScene& sc;
    float* rgb;
    uint8_t* rgb8;
    rt_ray_record* rec;
    float* samp_col;
    int* pix_cnt;
    void* branches;              // Fresnel branch queues, kMaxBranches per pool entry (or null)
    __device__ __forceinline__ const DevScene& scene(int) const { return sc; }
    __device__ __forceinline__ int64_t nwork() const { return sc.nwork; }
    __device__ __forceinline__ int64_t nsamples() const { return sc.nwork * sc.spp; }
    __device__ __forceinline__ void map(int64_t w, int& s, int64_t& pix, int64_t& out) const
    {
        s = 0;
        out = w;
        pix = sc.pix_list ? sc.pix_list[w] : w;
    }
    __device__ __forceinline__ void map_sample(int64_t ws, int& s, int64_t& pix, int64_t& out, int& sample) const
    {
        const int64_t w = ws / sc.spp;
        sample = (int)(ws - w * sc.spp);
        map(w, s, pix, out);
    }
    __device__ __forceinline__ int64_t sample_slot(int, int64_t out, int sample) const { return out * sc.spp + sample; }
    __device__ __forceinline__ int64_t pixel_slot(int, int64_t out) const { return out; }
    // colour slot of sample `sample` of output pixel `out`, and the pixel's counter
    __device__ __forceinline__ float* sample_col(int s, int64_t out, int sample) const
    {
        return samp_col + scene(s).col_base + (col_block_bytes(scene(s).spp) >> 2) * out + 4 * sample;
    }
    __device__ __forceinline__ int* pixel_count(int s, int64_t out) const { return pix_cnt + pixel_slot(s, out); }
    // the next work items of the calling lanes (warp-aggregated); -1 when none is left
    __device__ __forceinline__ int64_t grab(unsigned long long* counters, unsigned lane) const
    {
        const int64_t ws = grab_work(&counters[0], lane);
        return ws < nsamples() ? ws : -1;
    }
    __device__ __forceinline__ void pixel_done(int) const {}
    // the launch's counters are cleared before it starts: nothing to do
    __device__ __forceinline__ void release_count(int, int64_t) const {}
    __device__ __forceinline__ float* rgb_of(int) const { return rgb; }
    __device__ __forceinline__ uint8_t* rgb8_of(int) const { return rgb8; }
    __device__ __forceinline__ rt_ray_record* rec_of(int) const { return rec; }
};

struct ManyScenes {
    static constexpr bool kParamScene = false;   // scenes in a device table
    const DevScene* scenes;
    const int64_t* offsets;          // n + 1 entries: first pixel of each scene
    const int64_t* soffsets;         // n + 1 entries: first sample of each scene
    float* const* rgbs;              // per-scene output images
    int n;
    int64_t total, total_samples;
    float* samp_col;
    int* pix_cnt;
    void* branches;
    __device__ __forceinline__ const DevScene& scene(int s) const { return scenes[s]; }
    __device__ __forceinline__ int64_t nwork() const { return total; }
    __device__ __forceinline__ int64_t nsamples() const { return total_samples; }
    // last scene whose first entry in `table` is <= w
    __device__ __forceinline__ int find(const int64_t* table, int64_t w) const
    {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(table + mid) <= w) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    }
    __device__ __forceinline__ void map(int64_t w, int& s, int64_t& pix, int64_t& out) const
    {
        s = find(offsets, w);
        out = pix = w - __ldg(offsets + s);
    }
    __device__ __forceinline__ void map_sample(int64_t ws, int& s, int64_t& pix, int64_t& out, int& sample) const
    {
        s = find(soffsets, ws);
        const int64_t l = ws - __ldg(soffsets + s);
        const int spp = scenes[s].spp;
        const int64_t w = l / spp;
        sample = (int)(l - w * spp);
        out = pix = w;
    }
    __device__ __forceinline__ int64_t sample_slot(int s, int64_t out, int sample) const
    {
        return __ldg(soffsets + s) + out * scenes[s].spp + sample;
    }
    __device__ __forceinline__ int64_t pixel_slot(int s, int64_t out) const { return __ldg(offsets + s) + out; }
    __device__ __forceinline__ float* sample_col(int s, int64_t out, int sample) const
    {
        return samp_col + scene(s).col_base + (col_block_bytes(scene(s).spp) >> 2) * out + 4 * sample;
    }
    __device__ __forceinline__ int* pixel_count(int s, int64_t out) const { return pix_cnt + pixel_slot(s, out); }
    __device__ __forceinline__ int64_t grab(unsigned long long* counters, unsigned lane) const
    {
        const int64_t ws = grab_work(&counters[0], lane);
        return ws < nsamples() ? ws : -1;
    }
    __device__ __forceinline__ void pixel_done(int) const {}
    __device__ __forceinline__ void release_count(int, int64_t) const {}
    __device__ __forceinline__ float* rgb_of(int s) const { return rgbs[s]; }
    __device__ __forceinline__ uint8_t* rgb8_of(int) const { return nullptr; }
    __device__ __forceinline__ rt_ray_record* rec_of(int) const { return nullptr; }
};

// The persistent render loop of one thread (see the top of this file).
template <class R, int INTEG, class Src>
__device__ __forceinline__ void render_loop(const Src& src, unsigned long long* counters, int min_active)
{
    __shared__ Cold<R> cold_all[kRenderBlock];
    Cold<R>& C = cold_all[threadIdx.x];
    C.rays = 0;
    C.nevents = 0;
    C.scene = 0;
    for (int q = 0; q < 5; ++q) C.stat[q] = 0;
    Box<R> b;
    int phase = PH_IDLE, surf = EV_NONE, steps = 0;
    LaneStats st = {0u, 0u, 0u, 0u};
    const unsigned lane = threadIdx.x & 31u;
    const int64_t nwork = src.nwork();
#if RT_PROFILE
    // per-warp cycle split (lane 0): service pass, integration loop, loop
    // iterations and lanes inside the cloak summed over those iterations
    unsigned long long prof_service = 0, prof_hot = 0, prof_iters = 0, prof_lanes = 0;
#endif
    for (;;) {
#if RT_PROFILE
        const long long t_service = clock64();
#endif
        // lanes outside the integration catch up until their ray is inside
        // the cloak again or the work is exhausted
        while (phase != PH_BOX && phase != PH_EXIT) {
            if (phase == PH_EVENT || phase == PH_GUARD)
                service_event<R, INTEG, false>(src.scene(C.scene), C, b, phase, surf, steps, src.rec_of(C.scene), st);
            if (phase == PH_IDLE) {
                const int64_t w = grab_work(&counters[0], lane);
                if (w >= nwork) { phase = PH_EXIT; break; }
                int s;
                int64_t pix, out;
                src.map(w, s, pix, out);
                C.scene = s;
                C.work = out;
                C.pix = pix;
                C.sample = 0;
                C.acc[0] = C.acc[1] = C.acc[2] = 0.0f;
                start_sample<R, false>(src.scene(s), C, phase, surf, steps);
            }
            const DevScene& sc = src.scene(C.scene);
            if (phase == PH_AIR) air_segment<R, INTEG, false>(sc, C, b, phase, surf, steps, src.rec_of(C.scene), st);
            if (phase == PH_DONE) {
                if (++C.sample < sc.spp) {
                    start_sample<R, false>(sc, C, phase, surf, steps);
                } else {
                    const float inv = 1.0f / (float)sc.spp;
                    float c[3];
                    for (int a = 0; a < 3; ++a) c[a] = C.acc[a] * inv;
                    float* o = src.rgb_of(C.scene) + 3 * C.work;
                    o[0] = c[0]; o[1] = c[1]; o[2] = c[2];
                    uint8_t* q8 = src.rgb8_of(C.scene);
                    if (q8) {
                        uint8_t* q = q8 + 3 * C.work;
                        q[0] = quantize8(c[0]); q[1] = quantize8(c[1]); q[2] = quantize8(c[2]);
                    }
                    phase = PH_IDLE;
                }
            }
        }
        if (__ballot_sync(0xffffffffu, phase == PH_BOX) == 0u) break;   // every lane is out of work
#if RT_PROFILE
        const long long t_hot = clock64();
        prof_service += (unsigned long long)(t_hot - t_service);
#endif
        // once the work is exhausted, refills are pointless: step while any lane is inside
        const int need = __any_sync(0xffffffffu, phase == PH_EXIT) ? 1 : min_active;
        int safe = 0;                              // steps without the faces' tests (box_step_into)
        for (;;) {
#if RT_PROFILE
            prof_iters += 1;
            prof_lanes += __popc(__ballot_sync(0xffffffffu, phase == PH_BOX));
#endif
            if (phase == PH_BOX) {
                const DevScene& sc = src.scene(C.scene);
                box_step<R, INTEG>(step_const<R>(sc), sc.max_steps, C, b, phase, surf, steps, st, safe);
            }
            if (__popc(__ballot_sync(0xffffffffu, phase == PH_BOX)) < need) break;
        }
#if RT_PROFILE
        prof_hot += (unsigned long long)(clock64() - t_hot);
#endif
    }
#if RT_PROFILE
    if (lane == 0) {
        atomicAdd(&counters[12], prof_service);
        atomicAdd(&counters[13], prof_hot);
        atomicAdd(&counters[14], prof_iters);
        atomicAdd(&counters[15], prof_lanes);
    }
#endif
    // warp-reduce the counters, one atomic per warp and counter
    const uint32_t v[11] = {C.rays, st.steps, st.evals, st.newton, C.nevents, st.refine,
                            C.stat[0], C.stat[1], C.stat[2], C.stat[3], C.stat[4]};
#pragma unroll
    for (int q = 0; q < 11; ++q) {
        unsigned long long x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0 && x) atomicAdd(&counters[1 + q], x);
    }
}

template <class R, int MINB, int INTEG>
__global__ void __launch_bounds__(kRenderBlock, MINB) render_kernel(const __grid_constant__ DevScene sc,
                                                                    float* __restrict__ rgb,
                                                                    uint8_t* __restrict__ rgb8, rt_ray_record* rec,
                                                                    unsigned long long* counters, int min_active)
{
    const OneScene src{sc, rgb, rgb8, rec, nullptr, nullptr, nullptr};
    render_loop<R, INTEG>(src, counters, min_active);
}

// W0, n and the force at arbitrary points.
template <class R>
__global__ void medium_kernel(double kA, double Lambda, const double* __restrict__ xy, int64_t n,
                              double* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = xy[2 * i] / Lambda, y = xy[2 * i + 1] / Lambda;
    const double cxd = rint(x);
    const R X = (R)(x - cxd), yy = (R)y;
    R wr = R(0), wi = R(0), rr, ri;
    LaneStats st = {0u, 0u, 0u, 0u};
    StepConst<R> k = {};
    k.kA = (R)kA;
    k.w0tol = (R)(Mth<R>::kRel * kA);
    w0_eval(k, X, yy, wr, wi, rr, ri, st);
    R Fx, Fy;
    ray_force(wr, wi, rr, ri, R(kTwoPi), Fx, Fy);
    out[5 * i + 0] = (double)wr;
    out[5 * i + 1] = (double)wi;
    out[5 * i + 2] = sqrt((double)(rr * rr + ri * ri));
    out[5 * i + 3] = (double)Fx / Lambda;
    out[5 * i + 4] = (double)Fy / Lambda;
}

}  // namespace grt
