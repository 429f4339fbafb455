// rt_render.cu -- persistent render kernel of the grating-cloak ray tracer.
//
// One lane owns one pixel at a time and traces its samples one after the
// other (so the per-pixel sum has a fixed order).  The kernel is persistent:
// each loop iteration advances every lane by one unit of work -- one RK4 step
// inside the cloak, or a whole straight segment in air -- and lanes whose
// pixel is finished are refilled from a global work counter by one atomic per
// warp (ballot of the idle lanes, prefix rank by popc).
//
// Paper: ray ODE Sec. 3 (Eqs. 9-12), index Eq. 1, grating Eq. 2, camera and
// scene Sec. 4.  Inside the cloak the ray is integrated in the Hamiltonian
// parameter tau: dr/dtau = p, dp/dtau = grad(n^2)/2, |p| = n, which traces the
// curves of Eq. 11.
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "rt.h"
#include "rt_device.cuh"
#include "rt_internal.h"

namespace grt {

enum : int { PH_IDLE = 0, PH_AIR = 1, PH_BOX = 2, PH_DONE = 3, PH_EXIT = 4 };
enum : int { EV_NONE = -1, EV_GRATING = 0, EV_TOP = 1, EV_XP = 2, EV_XM = 3, EV_ZP = 4, EV_ZM = 5, EV_COUNT = 6 };

struct LaneStats {
    uint32_t rays, steps, evals, newton, events, refine;
    uint32_t status[5];
};

// Ray state inside the cloak, in local coordinates: x = cx + X.
template <class R>
struct Box {
    int cx;
    R X, y, z, px, py, pz;
    R cX, cy, cz, cpx, cpy;   // compensation terms of the FP32 sums
    R wr, wi, rr, ri;         // W0 and 1/(1+W0) at (X, y) (a prediction until solved)
    R Fx, Fy;                 // force at (X, y)
};

template <class R>
struct Lane {
    int64_t work;             // work item (pixel slot)
    int64_t pix;              // pixel index i*wout + j
    int sample, phase, surf, bounces, events, status;
    int64_t steps;
    float acc[3], col[3];
    double P[3], d[3];        // air: position and unit direction (normalised units)
    Box<R> b, prev;           // cloak: current state and the state at the start of the last step
    bool stepped;             // a step was taken since the last event
};

// ------------------------------------------------------------------------
// W0 with the FP64 branch-point refinement for the FP32 path.
// ------------------------------------------------------------------------
__device__ __noinline__ void w0_branch_fp64(double kA, double X, double y, double& wr, double& wi, int& iters)
{
    const double e = kA * exp(-kTwoPi * y);
    double s, c;
    sincospi(2.0 * X, &s, &c);
    const double zr = -e * c, zi = -e * s;                 // zeta = -kA e^{-ky} e^{ikx}
    // p = sqrt(2 (e zeta + 1)), principal root
    const double qr = 2.0 * (M_E * zr + 1.0), qi = 2.0 * M_E * zi;
    const double m = sqrt(qr * qr + qi * qi);
    double pr = sqrt(0.5 * (m + qr));
    double pi = (pr > 0.0) ? 0.5 * qi / pr : sqrt(0.5 * (m - qr));
    if (pr == 0.0 && qi < 0.0) pi = -pi;
    // w = -1 + p - p^2/3 + 11/72 p^3
    const double p2r = pr * pr - pi * pi, p2i = 2.0 * pr * pi;
    const double p3r = p2r * pr - p2i * pi, p3i = p2r * pi + p2i * pr;
    wr = -1.0 + pr - p2r / 3.0 + (11.0 / 72.0) * p3r;
    wi = pi - p2i / 3.0 + (11.0 / 72.0) * p3i;
    iters = 0;
    for (int it = 0; it < 60; ++it) {
        const double ex = exp(wr);
        double sw, cw;
        sincos(wi, &sw, &cw);
        const double er = ex * cw, ei = ex * sw;                       // e^w
        const double fr = wr * er - wi * ei - zr, fi = wr * ei + wi * er - zi;   // w e^w - zeta
        const double ar = wr + 1.0, ai = wi;                            // w + 1
        // t = (w+2) f / (2 (w+1))
        const double nr = (wr + 2.0) * fr - wi * fi, ni = (wr + 2.0) * fi + wi * fr;
        const double den = 2.0 * (ar * ar + ai * ai);
        const double tr = (nr * ar + ni * ai) / den, ti = (ni * ar - nr * ai) / den;
        // D = e^w (w+1) - t
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
__device__ __forceinline__ void w0_eval(R kA, R X, R y, R& wr, R& wi, R& rr, R& ri, LaneStats& st)
{
    st.newton += w0_solve(kA, X, y, wr, wi, rr, ri);
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

// ------------------------------------------------------------------------
// One RK4 step of size h from s (whose W and force are solved) into o.
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

template <class R>
__device__ __forceinline__ void rk4_step(R kA, const Box<R>& s, R h, Box<R>& o, LaneStats& st)
{
    const R h2 = R(0.5) * h;
    R wr = s.wr, wi = s.wi, rr = s.rr, ri = s.ri;
    // stage 2 at r + h/2 p
    const R X2 = s.X + h2 * s.px, y2 = s.y + h2 * s.py;
    w0_predict(wr, wi, rr, ri, h2 * s.px, h2 * s.py);
    w0_eval(kA, X2, y2, wr, wi, rr, ri, st);
    R F2x, F2y;
    ray_force(wr, wi, rr, ri, F2x, F2y);
    // stage 3 at r + h/2 (p + h/2 F1)
    const R X3 = s.X + h2 * (s.px + h2 * s.Fx), y3 = s.y + h2 * (s.py + h2 * s.Fy);
    w0_predict(wr, wi, rr, ri, X3 - X2, y3 - y2);
    w0_eval(kA, X3, y3, wr, wi, rr, ri, st);
    R F3x, F3y;
    ray_force(wr, wi, rr, ri, F3x, F3y);
    // stage 4 at r + h (p + h/2 F2)
    const R X4 = s.X + h * (s.px + h2 * F2x), y4 = s.y + h * (s.py + h2 * F2y);
    w0_predict(wr, wi, rr, ri, X4 - X3, y4 - y3);
    w0_eval(kA, X4, y4, wr, wi, rr, ri, st);
    R F4x, F4y;
    ray_force(wr, wi, rr, ri, F4x, F4y);
    // position increment h p + h^2/6 (F1 + F2 + F3), momentum h/6 (F1 + 2F2 + 2F3 + F4)
    const R h6 = h * R(1.0 / 6.0), hh6 = h * h6;
    const R dX = h * s.px + hh6 * (s.Fx + F2x + F3x);
    const R dY = h * s.py + hh6 * (s.Fy + F2y + F3y);
    const R dZ = h * s.pz;
    const R dPx = h6 * (s.Fx + R(2) * (F2x + F3x) + F4x);
    const R dPy = h6 * (s.Fy + R(2) * (F2y + F3y) + F4y);
    o.cx = s.cx;
    o.X = s.X; o.y = s.y; o.z = s.z; o.px = s.px; o.py = s.py; o.pz = s.pz;
    o.cX = s.cX; o.cy = s.cy; o.cz = s.cz; o.cpx = s.cpx; o.cpy = s.cpy;
    kahan_add(o.X, o.cX, dX);
    kahan_add(o.y, o.cy, dY);
    kahan_add(o.z, o.cz, dZ);
    kahan_add(o.px, o.cpx, dPx);
    kahan_add(o.py, o.cpy, dPy);
    // continue W to the end point
    w0_predict(wr, wi, rr, ri, o.X - X4, o.y - y4);
    o.wr = wr; o.wi = wi; o.rr = rr; o.ri = ri;
    if (o.X >= R(0.5)) { o.X -= R(1); o.cx += 1; }
    else if (o.X < R(-0.5)) { o.X += R(1); o.cx -= 1; }
    o.Fx = F4x; o.Fy = F4y;   // not the force at the end point; recomputed before use
}

// ------------------------------------------------------------------------
// Events inside the cloak: positive while the ray is inside, negative after
// it crossed the grating (v = Im w = y + Re W0/k < 0) or a face of the box.
// ------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R event_g(const DevScene& sc, int ev, const Box<R>& s)
{
    switch (ev) {
        case EV_GRATING: return s.y + s.wr * R(kInvTwoPi);
        case EV_TOP: return R(sc.ytop) - s.y;
        case EV_XP: return (R(sc.E2) - R(s.cx)) - s.X;
        case EV_XM: return (R(sc.E2) + R(s.cx)) + s.X;
        case EV_ZP: return R(sc.E2) - s.z;
        default: return R(sc.E2) + s.z;
    }
}

__device__ __forceinline__ void face_normal(int ev, double N[3])
{
    N[0] = N[1] = N[2] = 0.0;
    if (ev == EV_TOP) N[1] = 1.0;
    else if (ev == EV_XP) N[0] = 1.0;
    else if (ev == EV_XM) N[0] = -1.0;
    else if (ev == EV_ZP) N[2] = 1.0;
    else if (ev == EV_ZM) N[2] = -1.0;
    else N[1] = -1.0;
}

// d/dtheta of g(Phi_{theta h}(s)) at theta = 0, i.e. h grad g . p.
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

// Illinois (modified regula falsi) on [a, b] with fa > 0 >= fb.  Returns the
// last point evaluated, so the caller's functor holds the state there.
template <class R, class F>
__device__ __forceinline__ R illinois(F& f, R a, R fa, R b, R fb, R ftol, int maxit)
{
    int side = 0;
    R c = b;
    bool evaluated = false;
    for (int it = 0; it < maxit; ++it) {
        c = b - fb * (b - a) / (fb - fa);
        if (!(c > a && c < b)) c = R(0.5) * (a + b);
        const R fc = f(c);
        evaluated = true;
        if (fabs(fc) <= ftol) return c;
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
    if (!evaluated) f(c);
    return c;
}

// Locate theta in (0, 1] with g_ev(Phi_{theta h}(s0)) = 0 given g_ev(s1) = g1 < 0.
// When the step starts on that surface the zero at theta = 0 is divided out.
template <class R>
__device__ R locate_event(const DevScene& sc, const Box<R>& s0, R h, int ev, bool on_surface, R g1,
                          LaneStats& st)
{
    const R kA = R(sc.kA);
    R ga;
    if (on_surface) {
        ga = event_slope(ev, s0, h);
        if (!(ga > R(0))) ga = R(1e-30);
    } else {
        ga = event_g(sc, ev, s0);
        if (!(ga > R(0))) return R(0);
    }
    Box<R> t;
    auto fn = [&](R th) -> R {
        rk4_step(kA, s0, th * h, t, st);
        if (ev == EV_GRATING) w0_eval(kA, t.X, t.y, t.wr, t.wi, t.rr, t.ri, st);
        const R g = event_g(sc, ev, t);
        return on_surface ? g / th : g;
    };
    return illinois(fn, R(0), ga, R(1), g1, Mth<R>::kEventTol, Mth<R>::kEventIt);
}

// ------------------------------------------------------------------------
// Camera, background and finishing a sample.
// ------------------------------------------------------------------------
__device__ __forceinline__ void camera_ray(const DevScene& sc, int64_t pix, int s, double d[3])
{
    const int i = (int)(pix / sc.wout), j = (int)(pix % sc.wout);
    double ox = 0.5, oy = 0.5;
    if (sc.spp > 1) {
        const uint64_t c = (((uint64_t)sc.scene_id * (uint64_t)sc.height + (uint64_t)i) * (uint64_t)sc.wout +
                            (uint64_t)j) * (uint64_t)sc.spp + (uint64_t)s;
        const double u1 = uniform24(sc.seed, 2 * c + 1), u2 = uniform24(sc.seed, 2 * c + 2);
        if (sc.m > 0) {
            ox = ((double)(s % sc.m) + u1) / sc.m;
            oy = ((double)(s / sc.m) + u2) / sc.m;
        } else {
            ox = u1;
            oy = u2;
        }
    }
    const double px = sc.centre_line ? 0.0 : 2.0 * ((double)j + ox) / sc.width - 1.0;
    const double py = 1.0 - 2.0 * ((double)i + oy) / sc.height;
    double l = 0.0;
    for (int a = 0; a < 3; ++a) {
        d[a] = sc.f[a] + px * sc.tx * sc.r[a] + py * sc.ty * sc.u[a];
        l += d[a] * d[a];
    }
    l = sqrt(l);
    for (int a = 0; a < 3; ++a) d[a] /= l;
}

__device__ __forceinline__ int background(const DevScene& sc, const double X[3], const double d[3], float col[3])
{
    col[0] = col[1] = col[2] = 0.0f;
    const double dn = d[0] * sc.fr[0] + d[1] * sc.fr[1] + d[2] * sc.fr[2];
    if (!(dn > 0.0)) return RT_RAY_SKY;
    const double t = ((sc.Pb[0] - X[0]) * sc.fr[0] + (sc.Pb[1] - X[1]) * sc.fr[1] + (sc.Pb[2] - X[2]) * sc.fr[2]) / dn;
    double Y[3];
    for (int a = 0; a < 3; ++a) Y[a] = X[a] + t * d[a] - sc.Pb[a];
    const double s = Y[0] * sc.r[0] + Y[1] * sc.r[1] + Y[2] * sc.r[2];
    const double tt = Y[0] * sc.ur[0] + Y[1] * sc.ur[1] + Y[2] * sc.ur[2];
    if (sc.background == RT_BG_CHECKER) {
        const long long a = (long long)floor(s / sc.cell), b = (long long)floor(tt / sc.cell);
        const float* c = (((a + b) & 1LL) == 0) ? sc.col0 : sc.col1;
        col[0] = c[0]; col[1] = c[1]; col[2] = c[2];
    } else {
        const int N = sc.tex_size;
        const double U = s / sc.texel - 0.5, V = tt / sc.texel - 0.5;
        const double fu0 = floor(U), fv0 = floor(V);
        const float fu = (float)(U - fu0), fv = (float)(V - fv0);
        long long u0 = (long long)fu0 % N, v0 = (long long)fv0 % N;
        if (u0 < 0) u0 += N;
        if (v0 < 0) v0 += N;
        const long long u1 = (u0 + 1 == N) ? 0 : u0 + 1, v1 = (v0 + 1 == N) ? 0 : v0 + 1;
        const float t00 = __ldg(sc.tex + v0 * N + u0), t01 = __ldg(sc.tex + v0 * N + u1);
        const float t10 = __ldg(sc.tex + v1 * N + u0), t11 = __ldg(sc.tex + v1 * N + u1);
        const float val = (1.0f - fu) * (1.0f - fv) * t00 + fu * (1.0f - fv) * t01 + (1.0f - fu) * fv * t10 + fu * fv * t11;
        col[0] = col[1] = col[2] = val;
    }
    return RT_RAY_OK;
}

template <class R>
__device__ void finish_sample(const DevScene& sc, Lane<R>& L, int status, rt_ray_record* rec, LaneStats& st)
{
    if (status != RT_RAY_OK && status != RT_RAY_SKY) L.col[0] = L.col[1] = L.col[2] = 0.0f;
    L.status = status;
    L.acc[0] += L.col[0];
    L.acc[1] += L.col[1];
    L.acc[2] += L.col[2];
    st.rays += 1;
    st.status[status < 5 ? status : 4] += 1;
    if (rec) {
        double pos[3] = {L.P[0], L.P[1], L.P[2]};
        if (L.phase == PH_AIR && L.d[1] > 0.0 && L.P[1] < sc.yrec) {
            const double t = (sc.yrec - L.P[1]) / L.d[1];
            for (int a = 0; a < 3; ++a) pos[a] = L.P[a] + t * L.d[a];
        }
        rt_ray_record* o = rec + L.work * sc.spp + L.sample;
        for (int a = 0; a < 3; ++a) {
            o->pos[a] = pos[a] * sc.Lambda;
            o->dir[a] = L.d[a];
            o->rgb[a] = L.col[a];
        }
        o->status = status;
        o->bounces = L.bounces;
        o->events = L.events;
        o->steps = L.steps;
    }
    L.phase = PH_DONE;
}

// ------------------------------------------------------------------------
// Air: straight segments between the camera, the mirror, the cloak box and
// the background.
// ------------------------------------------------------------------------
// First hit of the line P + t d with the trochoid (Eq. 2), or INFINITY.  The
// line is marched from where it enters the band |y| <= A in increments that
// move the point by at most 1/(8 pi) in the xy-plane; the first increment
// ending at or below the surface brackets the hit, which is refined by
// Illinois.  Arithmetic is in R, in coordinates local to the band entry.
template <class R>
__device__ double trochoid_line_hit(const DevScene& sc, const double P[3], const double d[3], bool on_surface)
{
    const double A = sc.A;
    const double dxy = sqrt(d[0] * d[0] + d[1] * d[1]);
    if (dxy < 1e-300) return INFINITY;
    if (d[1] >= 0.0 && P[1] >= A) return INFINITY;
    double t0 = 0.0;
    if (P[1] > A) t0 = (A - P[1]) / d[1];
    double t_end;
    if (d[1] < 0.0) t_end = (-A - P[1]) / d[1];
    else if (d[1] > 0.0) t_end = (A - P[1]) / d[1];
    else t_end = t0 + 2.0 / fabs(d[0]);
    const double Qx = P[0] + t0 * d[0];
    const double cxd = rint(Qx);
    const R X0 = (R)(Qx - cxd);
    const R y0 = (R)(P[1] + t0 * d[1]);
    const R dx = (R)d[0], dy = (R)d[1];
    const R Ar = (R)A, kA = (R)sc.kA;
    const R L = (R)(t_end - t0);
    const R ds = (R)(0.25 / (kTwoPi * dxy));
    auto height = [&](R s) -> R {
        const R E = trochoid_phase(X0 + s * dx, kA);
        R sn, cs;
        Mth<R>::sincos(E, sn, cs);
        return (y0 + s * dy) - Ar * cs;
    };
    bool first = on_surface && t0 == 0.0;
    R sa = R(0), ha;
    if (first) {
        const R E = trochoid_phase(X0, kA);
        R sn, cs;
        Mth<R>::sincos(E, sn, cs);
        const R slope = -kA * sn / (R(1) - kA * cs);
        ha = dy - slope * dx;
        if (!(ha > R(0))) ha = R(1e-30);
    } else {
        ha = height(sa);
        if (ha <= R(0)) return t0;
    }
    for (int guard = 0; guard < 1 << 20; ++guard) {
        R sb = fmin(sa + ds, L);
        if (first && sb <= Mth<R>::kRehit) {
            if (sb >= L) return INFINITY;
            sb = fmin(Mth<R>::kRehit, L);
        }
        if (!(sb > sa) && !(sb >= L)) return INFINITY;   // no progress (NaN or an absorbed increment)
        R hb = height(sb);
        if (sb >= L && dy < R(0) && hb > R(0)) hb = R(0);
        if (hb <= R(0)) {
            R sr;
            if (first) {
                auto defl = [&](R s) -> R { return height(s) / s; };
                sr = illinois(defl, sa, ha, sb, hb / sb, Mth<R>::kEventTol, Mth<R>::kEventIt);
            } else {
                sr = illinois(height, sa, ha, sb, hb, Mth<R>::kEventTol, Mth<R>::kEventIt);
            }
            return t0 + (double)sr;
        }
        if (sb >= L) break;
        first = false;
        sa = sb;
        ha = hb;
    }
    return INFINITY;
}

__device__ __forceinline__ double flat_line_hit(const double P[3], const double d[3])
{
    if (d[1] < 0.0 && P[1] > 0.0) return -P[1] / d[1];
    return INFINITY;
}

// Entry of the line into the cloak box (slab method), INFINITY if it misses.
__device__ __forceinline__ double box_entry(const DevScene& sc, const double P[3], const double d[3], int& face)
{
    const double lo[3] = {-sc.E2, -sc.A, -sc.E2}, hi[3] = {sc.E2, sc.ytop, sc.E2};
    const int flo[3] = {EV_XM, EV_NONE, EV_ZM}, fhi[3] = {EV_XP, EV_TOP, EV_ZP};
    double tn = -INFINITY, tf = INFINITY;
    int fn = EV_NONE;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (P[a] < lo[a] || P[a] > hi[a]) return INFINITY;
            continue;
        }
        const double t1 = (lo[a] - P[a]) / d[a], t2 = (hi[a] - P[a]) / d[a];
        double tmin = t1, tmax = t2;
        int f = flo[a];
        if (t1 > t2) { tmin = t2; tmax = t1; f = fhi[a]; }
        if (tmin > tn) { tn = tmin; fn = f; }
        if (tmax < tf) tf = tmax;
    }
    if (!(tn <= tf) || !(tn > 1e-12)) return INFINITY;
    face = fn;
    return tn;
}

template <class R>
__device__ void air_segment(const DevScene& sc, Lane<R>& L, rt_ray_record* rec, LaneStats& st)
{
    for (;;) {
        if (L.bounces > sc.max_bounces) { finish_sample(sc, L, RT_RAY_MAX_BOUNCES, rec, st); return; }
        const double tm = sc.mirror ? trochoid_line_hit<R>(sc, L.P, L.d, L.surf == EV_GRATING) : flat_line_hit(L.P, L.d);
        int face = EV_NONE;
        const double tb = sc.cloak ? box_entry(sc, L.P, L.d, face) : INFINITY;
        if (tb < tm) {
            for (int a = 0; a < 3; ++a) L.P[a] += tb * L.d[a];
            double Nf[3];
            face_normal(face, Nf);
            Box<R>& b = L.b;
            const double cxd = rint(L.P[0]);
            b.cx = (int)cxd;
            b.X = (R)(L.P[0] - cxd);
            b.y = (R)L.P[1];
            b.z = (R)L.P[2];
            b.wr = b.wi = R(0);
            w0_eval((R)sc.kA, b.X, b.y, b.wr, b.wi, b.rr, b.ri, st);
            const double n2 = (double)(b.rr * b.rr + b.ri * b.ri);
            const double pn = L.d[0] * Nf[0] + L.d[1] * Nf[1] + L.d[2] * Nf[2];
            double pt[3];
            for (int a = 0; a < 3; ++a) pt[a] = L.d[a] - pn * Nf[a];
            const double pt2 = pt[0] * pt[0] + pt[1] * pt[1] + pt[2] * pt[2];
            if (n2 < pt2) {      // total reflection off the outside of the box
                for (int a = 0; a < 3; ++a) L.d[a] -= 2.0 * pn * Nf[a];
                L.bounces++;
                L.surf = EV_NONE;
                continue;
            }
            const double pin = sqrt(n2 - pt2);
            b.px = (R)(pt[0] - pin * Nf[0]);
            b.py = (R)(pt[1] - pin * Nf[1]);
            b.pz = (R)(pt[2] - pin * Nf[2]);
            b.cX = b.cy = b.cz = b.cpx = b.cpy = R(0);
            ray_force(b.wr, b.wi, b.rr, b.ri, b.Fx, b.Fy);
            L.stepped = false;
            L.surf = face;
            L.phase = PH_BOX;
            return;
        }
        if (tm < INFINITY) {
            for (int a = 0; a < 3; ++a) L.P[a] += tm * L.d[a];
            double N[3] = {0.0, 1.0, 0.0};
            if (sc.mirror) {
                const R E = trochoid_phase((R)(L.P[0] - rint(L.P[0])), (R)sc.kA);
                R sn, cs;
                Mth<R>::sincos(E, sn, cs);
                const double nx = sc.kA * (double)sn, ny = 1.0 - sc.kA * (double)cs;
                const double l = sqrt(nx * nx + ny * ny);
                N[0] = nx / l;
                N[1] = ny / l;
            }
            const double pn = L.d[0] * N[0] + L.d[1] * N[1] + L.d[2] * N[2];
            for (int a = 0; a < 3; ++a) L.d[a] -= 2.0 * pn * N[a];
            L.bounces++;
            L.surf = EV_GRATING;
            continue;
        }
        const int status = background(sc, L.P, L.d, L.col);
        finish_sample(sc, L, status, rec, st);
        return;
    }
}

// ------------------------------------------------------------------------
// One iteration inside the cloak: event check of the step just taken, then
// one RK4 step.
// ------------------------------------------------------------------------
template <class R>
__device__ void box_iteration(const DevScene& sc, Lane<R>& L, rt_ray_record* rec, LaneStats& st)
{
    const R kA = (R)sc.kA;
    const R h = (R)sc.h;
    Box<R>& b = L.b;
    // W0 and the force at the current point
    w0_eval(kA, b.X, b.y, b.wr, b.wi, b.rr, b.ri, st);
    ray_force(b.wr, b.wi, b.rr, b.ri, b.Fx, b.Fy);

    if (L.stepped) {
        int ev_best = EV_NONE;
        R th_best = R(2);
        for (int ev = 0; ev < EV_COUNT; ++ev) {
            const R g1 = event_g(sc, ev, b);
            if (g1 < R(0)) {
                const R th = locate_event(sc, L.prev, h, ev, L.surf == ev, g1, st);
                if (th < th_best) { th_best = th; ev_best = ev; }
            }
        }
        L.surf = EV_NONE;
        if (ev_best != EV_NONE) {
            L.events++;
            st.events += 1;
            rk4_step(kA, L.prev, th_best * h, b, st);
            w0_eval(kA, b.X, b.y, b.wr, b.wi, b.rr, b.ri, st);
            L.stepped = false;
            if (ev_best == EV_GRATING) {
                // mirror reflection about grad v / |grad v| = (Im r, Re r) / |r|
                const R il = R(1) / Mth<R>::sqrt_(b.rr * b.rr + b.ri * b.ri);
                const R nx = b.ri * il, ny = b.rr * il;
                const R pn = b.px * nx + b.py * ny;
                b.px -= R(2) * pn * nx;
                b.py -= R(2) * pn * ny;
                b.cpx = b.cpy = R(0);
                L.bounces++;
                L.surf = EV_GRATING;
                if (L.bounces > sc.max_bounces) {
                    L.phase = PH_BOX;
                    L.P[0] = (double)b.cx + (double)b.X; L.P[1] = (double)b.y; L.P[2] = (double)b.z;
                    const double l = sqrt((double)(b.px * b.px + b.py * b.py + b.pz * b.pz));
                    L.d[0] = b.px / l; L.d[1] = b.py / l; L.d[2] = b.pz / l;
                    finish_sample(sc, L, RT_RAY_MAX_BOUNCES, rec, st);
                }
                return;
            }
            // a face: refract into air (n = 1) or reflect totally
            double Nf[3];
            face_normal(ev_best, Nf);
            const double p[3] = {(double)b.px, (double)b.py, (double)b.pz};
            const double pn = p[0] * Nf[0] + p[1] * Nf[1] + p[2] * Nf[2];
            double pt[3];
            for (int a = 0; a < 3; ++a) pt[a] = p[a] - pn * Nf[a];
            const double pt2 = pt[0] * pt[0] + pt[1] * pt[1] + pt[2] * pt[2];
            if (pt2 >= 1.0) {
                b.px = (R)(p[0] - 2.0 * pn * Nf[0]);
                b.py = (R)(p[1] - 2.0 * pn * Nf[1]);
                b.pz = (R)(p[2] - 2.0 * pn * Nf[2]);
                b.cpx = b.cpy = R(0);
                L.bounces++;
                L.surf = ev_best;
                if (L.bounces > sc.max_bounces) {
                    L.phase = PH_BOX;
                    L.P[0] = (double)b.cx + (double)b.X; L.P[1] = (double)b.y; L.P[2] = (double)b.z;
                    const double l = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
                    L.d[0] = p[0] / l; L.d[1] = p[1] / l; L.d[2] = p[2] / l;
                    finish_sample(sc, L, RT_RAY_MAX_BOUNCES, rec, st);
                }
                return;
            }
            const double pout = sqrt(1.0 - pt2);
            double dd[3], l = 0.0;
            for (int a = 0; a < 3; ++a) { dd[a] = pt[a] + pout * Nf[a]; l += dd[a] * dd[a]; }
            l = sqrt(l);
            L.P[0] = (double)b.cx + (double)b.X;
            L.P[1] = (double)b.y;
            L.P[2] = (double)b.z;
            for (int a = 0; a < 3; ++a) L.d[a] = dd[a] / l;
            L.surf = EV_NONE;
            L.phase = PH_AIR;
            return;
        }
    }
    if (L.steps >= sc.max_steps || !(isfinite(b.X) && isfinite(b.y) && isfinite(b.px) && isfinite(b.py))) {
        const int status = (L.steps >= sc.max_steps) ? RT_RAY_MAX_STEPS : RT_RAY_NAN;
        L.P[0] = (double)b.cx + (double)b.X; L.P[1] = (double)b.y; L.P[2] = (double)b.z;
        const double l = sqrt((double)(b.px * b.px + b.py * b.py + b.pz * b.pz));
        L.d[0] = b.px / l; L.d[1] = b.py / l; L.d[2] = b.pz / l;
        L.phase = PH_BOX;
        finish_sample(sc, L, status, rec, st);
        return;
    }
    L.prev = b;
    rk4_step(kA, L.prev, h, b, st);
    L.steps++;
    st.steps += 1;
    L.stepped = true;
}

template <class R>
__device__ __forceinline__ void start_sample(const DevScene& sc, Lane<R>& L)
{
    camera_ray(sc, L.pix, L.sample, L.d);
    L.P[0] = sc.C[0]; L.P[1] = sc.C[1]; L.P[2] = sc.C[2];
    L.surf = EV_NONE;
    L.bounces = 0;
    L.events = 0;
    L.steps = 0;
    L.col[0] = L.col[1] = L.col[2] = 0.0f;
    L.phase = PH_AIR;
}

__device__ __forceinline__ uint8_t quantize8(float c)
{
    float v = c > 0.0f ? c : 0.0f;
    v = v < 1.0f ? v : 1.0f;
    return (uint8_t)floorf(v * 255.0f + 0.5f);
}

template <class R>
__global__ void __launch_bounds__(kRenderBlock) render_kernel(DevScene sc, float* __restrict__ rgb,
                                                              uint8_t* __restrict__ rgb8, rt_ray_record* rec,
                                                              unsigned long long* counters)
{
    Lane<R> L;
    L.phase = PH_IDLE;
    L.work = -1;
    LaneStats st = {};
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (;;) {
        const unsigned idle = __ballot_sync(0xffffffffu, L.phase == PH_IDLE);
        if (idle) {
            const int leader = __ffs(idle) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(&counters[0], (unsigned long long)__popc(idle));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (L.phase == PH_IDLE) {
                const int64_t k = (int64_t)base + __popc(idle & lt_mask);
                if (k < sc.nwork) {
                    L.work = k;
                    L.pix = sc.pix_list ? sc.pix_list[k] : k;
                    L.sample = 0;
                    L.acc[0] = L.acc[1] = L.acc[2] = 0.0f;
                    start_sample(sc, L);
                } else {
                    L.phase = PH_EXIT;
                }
            }
        }
        if (__all_sync(0xffffffffu, L.phase == PH_EXIT)) break;
        if (L.phase == PH_BOX) box_iteration(sc, L, rec, st);
        if (L.phase == PH_AIR) air_segment(sc, L, rec, st);
        if (L.phase == PH_DONE) {
            if (++L.sample < sc.spp) {
                start_sample(sc, L);
            } else {
                const float inv = 1.0f / (float)sc.spp;
                float c[3];
                for (int a = 0; a < 3; ++a) c[a] = L.acc[a] * inv;
                float* o = rgb + 3 * L.work;
                o[0] = c[0]; o[1] = c[1]; o[2] = c[2];
                if (rgb8) {
                    uint8_t* q = rgb8 + 3 * L.work;
                    q[0] = quantize8(c[0]); q[1] = quantize8(c[1]); q[2] = quantize8(c[2]);
                }
                L.phase = PH_IDLE;
            }
        }
    }
    // warp-reduce the counters, one atomic per warp and counter
    uint32_t v[11] = {st.rays, st.steps, st.evals, st.newton, st.events, st.refine,
                      st.status[0], st.status[1], st.status[2], st.status[3], st.status[4]};
#pragma unroll
    for (int q = 0; q < 11; ++q) {
        unsigned long long x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0 && x) atomicAdd(&counters[1 + q], x);
    }
}

// ------------------------------------------------------------------------
// Medium evaluation (W0, n, force) at arbitrary points.
// ------------------------------------------------------------------------
template <class R>
__global__ void medium_kernel(double kA, double Lambda, const double* __restrict__ xy, int64_t n, double* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = xy[2 * i] / Lambda, y = xy[2 * i + 1] / Lambda;
    const double cxd = rint(x);
    const R X = (R)(x - cxd), yy = (R)y;
    R wr = R(0), wi = R(0), rr, ri;
    LaneStats st = {};
    w0_eval((R)kA, X, yy, wr, wi, rr, ri, st);
    R Fx, Fy;
    ray_force(wr, wi, rr, ri, Fx, Fy);
    out[5 * i + 0] = (double)wr;
    out[5 * i + 1] = (double)wi;
    out[5 * i + 2] = sqrt((double)(rr * rr + ri * ri));
    out[5 * i + 3] = (double)Fx / Lambda;
    out[5 * i + 4] = (double)Fy / Lambda;
}

// ------------------------------------------------------------------------
// Host-side launchers.
// ------------------------------------------------------------------------
template <class R>
static cudaError_t launch_render_t(const DevScene& sc, float* rgb, uint8_t* rgb8, rt_ray_record* rec,
                                   unsigned long long* counters, int grid, cudaStream_t stream)
{
    render_kernel<R><<<grid, kRenderBlock, 0, stream>>>(sc, rgb, rgb8, rec, counters);
    return cudaGetLastError();
}

cudaError_t render_occupancy(int precision, int* blocks_per_sm)
{
    if (precision == RT_FP64)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, render_kernel<double>, kRenderBlock, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, render_kernel<float>, kRenderBlock, 0);
}

cudaError_t launch_render(const DevScene& sc, int precision, float* rgb, uint8_t* rgb8, rt_ray_record* rec,
                          unsigned long long* counters, int grid, cudaStream_t stream)
{
    if (precision == RT_FP64) return launch_render_t<double>(sc, rgb, rgb8, rec, counters, grid, stream);
    return launch_render_t<float>(sc, rgb, rgb8, rec, counters, grid, stream);
}

cudaError_t launch_medium(int precision, double kA, double Lambda, const double* xy, int64_t n, double* out,
                          cudaStream_t stream)
{
    const int block = 128;
    const int64_t grid = (n + block - 1) / block;
    if (grid == 0) return cudaSuccess;
    if (precision == RT_FP64) medium_kernel<double><<<(unsigned)grid, block, 0, stream>>>(kA, Lambda, xy, n, out);
    else medium_kernel<float><<<(unsigned)grid, block, 0, stream>>>(kA, Lambda, xy, n, out);
    return cudaGetLastError();
}

}  // namespace grt
