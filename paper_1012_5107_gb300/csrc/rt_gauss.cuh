// rt_gauss.cuh -- the Gaussian conformal cloak (Sec. 2, Fig. 1(b), Fig. 4).
//
// The virtual half plane v >= 0, whose boundary v = 0 is the flat mirror,
// maps onto the region above the bump by
//     z(w) = w + i h F(w / w_b),     F(s) = exp(-s^2) erfc(-i s),
// the Faddeeva function.  The bump is the image of v = 0:
//     x = u - h Im F(u / w_b),  y = h exp(-(u / w_b)^2),
// Eq. 5 in the shallow-bump limit, and the index is n = |dw/dz| = 1/|z'(w)|.
// At w_b = 0.306, h = 0.13 this gives n_min = 0.873 and n/n_min in [1, 2.2],
// the values printed for Fig. 1(b).
//
// Inside the box the tracer keeps, in the Box fields of the grating's W0,
//     W = -i k (w - z)   (so that v = Im w = y + Re W / k, as for the grating)
// and g = dw/dz in place of 1/(1 + W0): the event function, its gradient
// (Im g, Re g) and the mirror normal are then the grating's expressions.
#pragma once

#include "rt_device.cuh"

namespace grt {

// ------------------------------------------------------------------------
// Faddeeva function by Weideman's rational series (Weideman 1994, "Computation
// of the complex error function", SIAM J. Numer. Anal. 31, 1497-1518): for
// Im s >= 0
//     F(s) = 1/(sqrt(pi) (L - i s)) + 2/(L - i s)^2 sum_{n<N} a_{n+1} Z^n,
//     Z = (L + i s)/(L - i s),  L = 2^(-1/4) N^(1/2),
// with a_n the Fourier coefficients of (L^2 + t^2) exp(-t^2) in the angle
// theta of t = L tan(theta/2).  N = 20 in FP32 (error below 4e-9) and 40 in
// FP64 (below 2e-15).  The coefficients, with L as the last entry, are
// computed on the host and uploaded to every device that renders a Gaussian
// scene (gauss_upload in rt_render.cu).
// ------------------------------------------------------------------------
constexpr int kWNf = 20, kWNd = 40;
static __constant__ float kWaf[kWNf + 1];
static __constant__ double kWad[kWNd + 1];
constexpr double kInvSqrtPi = 0.56418958354775628695;

template <class R> struct WTab;
template <> struct WTab<float> {
    static constexpr int N = kWNf;
    static __device__ __forceinline__ float a(int n) { return kWaf[n]; }
};
template <> struct WTab<double> {
    static constexpr int N = kWNd;
    static __device__ __forceinline__ double a(int n) { return kWad[n]; }
};

// Out of line: the series is evaluated at every solve and in the bump's
// parameter, and inlining each copy overflowed the instruction cache (ncu:
// 3.3 no_instruction stall cycles per issued instruction; 12.5 -> 10.5 ms on
// the 512 x 512 x 4 Gaussian cloak).
template <class R>
__device__ __noinline__ void faddeeva_upper(R sr, R si, R& fr, R& fi)
{
    constexpr int N = WTab<R>::N;
    const R L = WTab<R>::a(N);
    // d = L - i s; q = 1/d
    const R dr = L + si, di = -sr;
    const R id2 = Mth<R>::rcp(dr * dr + di * di);
    const R qr = dr * id2, qi = -di * id2;
    // Z = (L + i s) q
    const R nr = L - si, ni = sr;
    const R zr = nr * qr - ni * qi, zi = nr * qi + ni * qr;
    R pr = WTab<R>::a(N - 1), pi = R(0);
#pragma unroll
    for (int n = N - 2; n >= 0; --n) {
        const R t = pr * zr - pi * zi + WTab<R>::a(n);
        pi = pr * zi + pi * zr;
        pr = t;
    }
    const R q2r = qr * qr - qi * qi, q2i = R(2) * qr * qi;
    fr = R(2) * (pr * q2r - pi * q2i) + R(kInvSqrtPi) * qr;
    fi = R(2) * (pr * q2i + pi * q2r) + R(kInvSqrtPi) * qi;
}

// F(s) anywhere; below the real axis (a step that overshot the bump) by the
// reflection F(s) = 2 exp(-s^2) - F(-s).
template <class R>
__device__ __forceinline__ void faddeeva(R sr, R si, R& fr, R& fi)
{
    if (si >= R(0)) {
        faddeeva_upper(sr, si, fr, fi);
        return;
    }
    R gr, gi;
    faddeeva_upper(-sr, -si, gr, gi);
    // exp(-s^2) = exp(si^2 - sr^2) (cos(2 sr si) - i sin(2 sr si))
    const R m = Mth<R>::ex2((si * si - sr * sr) * R(kLog2e));
    R sn, cs;
    Mth<R>::sincos(R(2) * sr * si, sn, cs);
    fr = R(2) * m * cs - gr;
    fi = R(-2) * m * sn - gi;
}

// ------------------------------------------------------------------------
// Medium of the box: W = -i k (w - z) at the point (X, y) (X absolute: the
// Gaussian box keeps no cell offset) by Newton's method on
//     W + k h F(s) = 0,   s = (z + i W / k) / w_b,
// from the guess in (wr, wi); each step dW = (W + k h F) g with
// g = 1/z'(w), z' = 1 + i (h/w_b) F'(s), limited to a quarter width in w.
// It stops once |dW|^2 <= gtol.  Returned: W, g = dw/dz in (rr, ri), and the
// force F = grad(n^2)/2 = (Re(conj(g) g'), -Im(conj(g) g')) with
// g' = -z''(w) g^3, z'' = i (h/w_b^2) F''(s), all at the last iterate
// evaluated (the update after it is below the stop).  F' = -2 s F + 2i/sqrt(pi)
// and F'' = -2 F - 2 s F' follow from F.
// ------------------------------------------------------------------------
// Also returned: the second derivative of g, 3 z''^2 g^5 - z''' g^4 with
// z''' = i (h/w_b^3) F''' and F''' = -4 F' - 2 s F'', in (gpr, gpi), for
// gauss_continue.
template <class R>
__device__ __forceinline__ void gauss_solve(const StepConst<R>& k, R X, R y, R& wr, R& wi, R& rr, R& ri, R& Fx,
                                            R& Fy, R& gpr, R& gpi, LaneStats& st)
{
    const R ik = R(kInvTwoPi);
    int it = 0;
    for (;;) {
        const R sr = (X - wi * ik) * k.igw, si = (y + wr * ik) * k.igw;
        R fr, fi;
        faddeeva(sr, si, fr, fi);
        const R f1r = R(-2) * (sr * fr - si * fi);
        const R f1i = R(-2) * (sr * fi + si * fr) + R(2.0 * kInvSqrtPi);
        const R zr = R(1) - k.gq * f1i, zi = k.gq * f1r;             // z'
        const R inv = Mth<R>::rcp(zr * zr + zi * zi);
        const R gr = zr * inv, gi = -zi * inv;                       // g = 1/z'
        const R rhr = wr + k.gkh * fr, rhi = wi + k.gkh * fi;        // W + k h F
        R dr = rhr * gr - rhi * gi, di = rhr * gi + rhi * gr;
        const R d2 = dr * dr + di * di;
        if (d2 > k.gcap2) {
            const R sc = Mth<R>::sqrt_(k.gcap2 / d2);
            dr *= sc;
            di *= sc;
        }
        wr -= dr;
        wi -= di;
        ++it;
        if (d2 <= k.gtol || it >= Mth<R>::kMaxIt) {
            rr = gr;
            ri = gi;
            const R f2r = R(-2) * fr - R(2) * (sr * f1r - si * f1i);
            const R f2i = R(-2) * fi - R(2) * (sr * f1i + si * f1r);
            const R c = k.gq * k.igw;
            const R z2r = -c * f2i, z2i = c * f2r;                   // z''
            const R g2r = gr * gr - gi * gi, g2i = R(2) * gr * gi;   // g^2
            const R n2 = gr * gr + gi * gi;
            const R tr = z2r * g2r - z2i * g2i, ti = z2r * g2i + z2i * g2r;   // z'' g^2
            Fx = -n2 * tr;
            Fy = n2 * ti;
            if constexpr (sizeof(R) == 4) {      // only the FP32 path continues (gauss_continue)
                const R f3r = R(-4) * f1r - R(2) * (sr * f2r - si * f2i);
                const R f3i = R(-4) * f1i - R(2) * (sr * f2i + si * f2r);
                const R c3 = c * k.igw;
                const R z3r = -c3 * f3i, z3i = c3 * f3r;                         // third derivative of z
                const R t2r = tr * tr - ti * ti, t2i = R(2) * tr * ti;           // (z'' g^2)^2
                const R g4r = g2r * g2r - g2i * g2i, g4i = R(2) * g2r * g2i;     // g^4
                gpr = R(3) * (t2r * gr - t2i * gi) - (z3r * g4r - z3i * g4i);
                gpi = R(3) * (t2r * gi + t2i * gr) - (z3r * g4i + z3i * g4r);
            } else {
                gpr = gpi = R(0);
            }
            break;
        }
    }
    st.newton += it;
    st.evals += 1;
}

template <class R>
__device__ __forceinline__ void gauss_solve(const StepConst<R>& k, R X, R y, R& wr, R& wi, R& rr, R& ri, R& Fx,
                                            R& Fy, LaneStats& st)
{
    R gpr, gpi;
    gauss_solve(k, X, y, wr, wi, rr, ri, Fx, Fy, gpr, gpi, st);
}

// Second-order continuation of W along a displacement dz = (dx, dy) from a
// point where W, g and the force are known:
//     W(z + dz) = W - i k ((g - 1) + g' dz / 2) dz,
// with g' = (Fx - i Fy) g / |g|^2 from the force.
template <class R>
__device__ __forceinline__ void gauss_predict(R& wr, R& wi, R rr, R ri, R Fx, R Fy, R dx, R dy)
{
    const R in2 = Mth<R>::rcp(rr * rr + ri * ri);
    const R gpr = (Fx * rr + Fy * ri) * in2, gpi = (Fx * ri - Fy * rr) * in2;
    const R er = rr - R(1) + R(0.5) * (gpr * dx - gpi * dy);
    const R ei = ri + R(0.5) * (gpr * dy + gpi * dx);
    const R tr = er * dx - ei * dy, ti = er * dy + ei * dx;
    wr += R(kTwoPi) * ti;
    wi -= R(kTwoPi) * tr;
}

// The medium at a point dz = (dx, dy) from one where W, g, g'' and the force
// are known.  A short step (|dz|^2 / w_b^2 at most gpred) is continued:
//   W by gauss_predict;  g + g' dz + g'' dz^2 / 2;
//   q + conj(g) g'' dz + |g'|^2 conj(dz) for q = conj(g) g', the force being
//   (Re q, -Im q);
// g' from the force as in gauss_predict.  What is left out is of higher order
// in |dz| / w_b, below the working precision for such steps.  Longer steps
// are predicted and solved.  Returns whether it solved.
template <class R>
__device__ __forceinline__ bool gauss_continue(const StepConst<R>& k, R X, R y, R dx, R dy, R& wr, R& wi, R& rr,
                                               R& ri, R& Fx, R& Fy, R& gpr, R& gpi, LaneStats& st)
{
    // FP64 solves every point: its threshold would admit only the shortest
    // steps, and the extra FP64 work costs more than the solves it saves
    if (sizeof(R) == 8 || (dx * dx + dy * dy) * (k.igw * k.igw) > k.gpred) {
        gauss_predict(wr, wi, rr, ri, Fx, Fy, dx, dy);
        gauss_solve(k, X, y, wr, wi, rr, ri, Fx, Fy, gpr, gpi, st);
        return true;
    }
    const R in2 = Mth<R>::rcp(rr * rr + ri * ri);
    const R g1r = (Fx * rr + Fy * ri) * in2, g1i = (Fx * ri - Fy * rr) * in2;     // g'
    gauss_predict(wr, wi, rr, ri, Fx, Fy, dx, dy);
    const R hdr = gpr * dx - gpi * dy, hdi = gpr * dy + gpi * dx;                // g'' dz
    const R m1 = g1r * g1r + g1i * g1i;
    const R dqr = (rr * hdr + ri * hdi) + m1 * dx;                               // conj(g) g'' dz + |g'|^2 conj(dz)
    const R dqi = (rr * hdi - ri * hdr) - m1 * dy;
    Fx += dqr;
    Fy -= dqi;
    const R nr = rr + (g1r * dx - g1i * dy) + R(0.5) * (hdr * dx - hdi * dy);
    const R ni = ri + (g1r * dy + g1i * dx) + R(0.5) * (hdr * dy + hdi * dx);
    rr = nr;
    ri = ni;
    st.evals += 1;
    return false;
}

// ------------------------------------------------------------------------
// The bump in air: x(u) = u - h Im F(u/w_b) is increasing (h/w_b < 0.8 <
// sqrt(pi)/2) and |x - u| <= 0.62 h.
// ------------------------------------------------------------------------
// Parameter u of the bump point above abscissa x: Newton's method on x(u) = x
// with dx/du = 1 - (h/w_b) Im F'(u/w_b), guarded by bisection on [x - h, x + h].
template <class R>
__device__ __noinline__ R bump_u(const StepConst<R>& k, R x)   // out of line for the same reason
{
    R lo = x - k.A, hi = x + k.A, u = x;
    for (int it = 0; it < 60; ++it) {
        const R s = u * k.igw;
        R fr, fi;
        faddeeva(s, R(0), fr, fi);
        const R f = (u - k.A * fi) - x;
        if (f > R(0)) hi = u;
        else lo = u;
        const R dxdu = R(1) - k.gq * (R(-2) * s * fi + R(2.0 * kInvSqrtPi));
        R un = u - f / dxdu;
        if (!(un > lo && un < hi)) un = R(0.5) * (lo + hi);
        const R d = fabs(un - u);
        u = un;
        if (d <= R(4) * Mth<R>::kEps * (R(1) + fabs(u))) break;
    }
    return u;
}

// Tangent (dx/du, dy/du) = z'(u) of the bump at parameter u.
template <class R>
__device__ __forceinline__ void bump_tangent(const StepConst<R>& k, R u, R& tx, R& ty)
{
    const R s = u * k.igw;
    R fr, fi;
    faddeeva(s, R(0), fr, fi);
    const R f1r = R(-2) * s * fr, f1i = R(-2) * s * fi + R(2.0 * kInvSqrtPi);
    tx = R(1) - k.gq * f1i;
    ty = k.gq * f1r;
}

// Height of the point (x, y) above the bump.
template <class R>
__device__ __forceinline__ R bump_height(const StepConst<R>& k, R x, R y)
{
    const R s = bump_u(k, x) * k.igw;
    return y - k.A * Mth<R>::ex2(-(s * s) * R(kLog2e));
}

}  // namespace grt
