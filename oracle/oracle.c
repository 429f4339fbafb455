/*
 * oracle.c -- plain FP64 CPU oracle for Newtonian ray tracing of the conformal
 * grating cloak (Halimeh, Schmied & Wegener, "Newtonian photorealistic ray
 * tracing of grating cloaks and correlation-function-based cloaking-quality
 * assessment", Opt. Express 2010).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package's smoke check and the
 * CPU-baseline leg of bench.py may load this library.  The product path (the
 * CUDA library) never links, imports or calls it; the two share no code,
 * header, table or constant generator.
 *
 * Everything is double precision, one ray at a time, in the order the method
 * states it, with no blocking or reordering.  Pixels are independent, so the
 * render loops run over pixels with OpenMP; each pixel is computed exactly as
 * in a serial run.
 *
 * Readings of the paper taken here (the paper is silent on all of them):
 *   - the ray ODE is integrated in the Hamiltonian parameter tau,
 *     dr/dtau = p, dp/dtau = grad(n^2)/2 = n grad n, |p| = n, which traces
 *     the same curves as the Newtonian form of Eq. 11 (dtau = c0/n^2 dt);
 *     integrator 2 integrates Eq. 11 itself in physical time t (c0 = 1,
 *     state (r, v), |v| = 1/n) with classical RK4 of fixed step h in t;
 *   - W0 is evaluated by Halley's iteration, cold-started at every call;
 *   - the grating hit inside the cloak is the root theta in (0,1] of
 *     v(Phi_{theta h}(s)) = 0 with v = Im w = y + Re(W0)/k, where Phi is one
 *     integrator step from the state s at the start of the step;
 *   - the cloak is a box |x|,|z| <= E/2, -A <= y <= -A + H with n from Eq. 1
 *     inside and n = 1 outside; at its faces Snell's law acts on p (tangential
 *     part kept) with total internal reflection; Fresnel weights are an option
 *     (OR_FLAG_FRESNEL: unpolarised reflectance, one reflected branch per
 *     crossing of a not yet reflected path, at most OR_MAX_BRANCHES per
 *     sample, branches not split again);
 *   - the referenced cloak (Figs. 5-7) divides the index inside the box by
 *     n_min = 1/(1 + kA); its ideal reference is a homogeneous plate of index
 *     1 + kA filling the box from the flat mirror (y = 0) to the box top;
 *   - the Gaussian conformal cloak (Fig. 1(b), Fig. 4) is the map
 *     z(w) = w + i h F(w/w_b) with F the Faddeeva function: it bounds the
 *     bump by the image of v = 0, which tends to Eq. 5 for shallow bumps, and
 *     at w_b = 0.306, h = 0.13 it gives the printed n_min = 0.873 and
 *     n/n_min in [1, 2.2]; its box spans y = 0 (the flat mirror) to H;
 *   - the photograph (Fig. 2a) is replaced by a synthetic background plane.
 *
 * 3-D rays (p_z != 0) are pinned by their planar part: (x, y, p_x, p_y)
 * evolve exactly as those of the same ray with p_z = 0 while z moves
 * linearly; total internal reflection at the side faces by the reflection
 * law, component by component, at the +x and +z faces
 * (tests/test_oracle_box_faces.py); refraction at the faces by the plate's
 * parallel displacement (tests/test_oracle_fresnel.py).
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Scene and record layouts (mirrored by oracle/oracle.py).                 */
/* ------------------------------------------------------------------------ */
typedef struct or_scene {
    double Lambda, A;                 /* grating period, half peak-to-peak amplitude (Eq. 2) */
    double H, E;                      /* cloak box height above y=-A and extent in x and z   */
    double cam_dist, elev_deg, azim_deg, hfov_deg;
    double bg_cell, tex_texel;
    double colour0[3], colour1[3];    /* checkerboard colours in [0,1]                       */
    double h, rtol, atol, h_max;      /* integrator parameters (world units)                 */
    double gauss_w;                   /* Gaussian bump width w (mirror 2); its height is A    */
    uint64_t seed, scene_id;
    int64_t max_steps;
    const float* tex;                 /* tex_size x tex_size greyscale, row-major            */
    int32_t mirror;                   /* 0 flat plane y=0, 1 trochoid grating (Eq. 2),
                                         2 Gaussian bump (Eq. 5, exact form below)           */
    int32_t cloak;                    /* 1: graded-index box above the mirror: Eq. 1 for the
                                         grating, the Gaussian conformal map for the bump    */
    int32_t width, height, spp, centre_line;
    int32_t background;               /* 0 checkerboard, 1 texture                           */
    int32_t tex_size, integrator;     /* integrator: 0 RK4 fixed step, 1 Dormand-Prince 5(4) */
    int32_t max_bounces;
    int32_t flags;                    /* OR_FLAG_* below                                      */
} or_scene;

/* Options of Sec. 3 and Figs. 5-7:
   REFERENCED  the cloak's index profile divided by n_min = 1/(1 + kA), so that
               it is >= 1; the air keeps n = 1 (Sec. 4, Figs. 5-7);
   PLATE       no cloak: a homogeneous dielectric plate of index 1/n_min on the
               flat mirror, filling the cloak's box from the mirror (y = 0) to
               the box top (the "ideal" references of Figs. 5-7 (a));
   FRESNEL     Fresnel weights at the box faces (Sec. 3): a crossing keeps the
               unpolarised transmittance T = 1 - R on the refracted ray, and a
               ray that has not been Fresnel-reflected yet also starts a branch
               along the reflected direction with weight R; branches are not
               split again (rays reflected more than once are neglected).
               Total internal reflection keeps the full weight. */
enum { OR_FLAG_REFERENCED = 1, OR_FLAG_PLATE = 2, OR_FLAG_FRESNEL = 4 };
#define OR_MAX_BRANCHES 8          /* Fresnel branches followed per camera sample */

typedef struct or_record {
    double pos[3], dir[3], rgb[3];
    int64_t steps;                    /* integrator steps taken (accepted + rejected)        */
    int64_t halley;                   /* Halley iterations spent in W0                       */
    int64_t evals;                    /* force evaluations                                   */
    int32_t bounces, status, events, pad;
} or_record;

enum { ST_OK = 0, ST_SKY = 1, ST_MAX_BOUNCES = 2, ST_MAX_STEPS = 3, ST_NAN = 4 };
enum { EV_NONE = -1, EV_GRATING = 0, EV_TOP = 1, EV_XP = 2, EV_XM = 3, EV_ZP = 4, EV_ZM = 5, EV_COUNT = 6 };
enum { MED_AIR = 0, MED_BOX = 1, MED_PLATE = 2 };

typedef struct counters { int64_t halley, evals; } counters;

/* ------------------------------------------------------------------------ */
/* Lambert W0 (Eq. 1 and Eq. 13 name the principal branch).                */
/* Halley's iteration on f(w) = w e^w - z.  Initial guesses: the series in   */
/* p = sqrt(2(e z + 1)) about the branch point and the asymptotic form       */
/* log z - log log z, both from Corless, Gonnet, Hare, Jeffrey & Knuth       */
/* (1996), Sec. 4; in between the [2/2] Pade approximant of the Taylor       */
/* series W0 = z - z^2 + 3/2 z^3 - 8/3 z^4 + ..., i.e.                       */
/* z (6 + 8 z) / (6 + 14 z + 5 z^2).                                          */
/* ------------------------------------------------------------------------ */
static double complex or_w0_c(double complex z, int* iters)
{
    *iters = 0;
    if (z == 0.0) return 0.0;
    const double e = exp(1.0);
    double complex q = e * z + 1.0;               /* e (z + 1/e) */
    if (q == 0.0) return -1.0;                    /* the branch point itself */
    double complex w;
    if (cabs(q) < 0.5 * e) {
        double complex p = csqrt(2.0 * q);
        w = -1.0 + p - p * p / 3.0 + (11.0 / 72.0) * p * p * p - (43.0 / 540.0) * p * p * p * p;
    } else if (cabs(z) < 1.5) {
        w = z * (6.0 + 8.0 * z) / (6.0 + 14.0 * z + 5.0 * z * z);
    } else {
        double complex L1 = clog(z), L2 = clog(L1);
        w = L1 - L2 + L2 / L1;
    }
    for (int it = 1; it <= 100; ++it) {
        double complex ew = cexp(w);
        double complex f = w * ew - z;
        double complex wp1 = w + 1.0;
        double complex dw = f / (ew * wp1 - (w + 2.0) * f / (2.0 * wp1));
        w -= dw;
        *iters = it;
        if (!(cabs(dw) > 8.0 * DBL_EPSILON * cabs(w))) break;
    }
    return w;
}

/* zeta = i c k exp(i k (x + i y)) with c = i A and k = 2 pi / Lambda (Eq. 1, Eq. 13). */
static double complex or_zeta(const or_scene* sc, double x, double y)
{
    const double k = 2.0 * OR_PI / sc->Lambda;
    const double complex c = I * sc->A;
    return I * c * k * cexp(I * k * (x + I * y));
}

/* ------------------------------------------------------------------------ */
/* Faddeeva function F(s) = exp(-s^2) erfc(-i s), for the Gaussian cloak.    */
/* Weideman (1994), "Computation of the complex error function", SIAM J.    */
/* Numer. Anal. 31, 1497-1518: for Im s >= 0                                 */
/*   F(s) ~ 1/(sqrt(pi) (L - i s)) + 2/(L - i s)^2 sum_{n<N} a_{n+1} Z^n,    */
/*   Z = (L + i s)/(L - i s),  L = 2^(-1/4) N^(1/2),                         */
/* with a_n the Fourier coefficients (in theta) of (L^2 + t^2) exp(-t^2),    */
/* t = L tan(theta/2); here N = 48 and the coefficients come from the        */
/* midpoint rule on 8192 angles.  Below the real axis the reflection         */
/* F(s) = 2 exp(-s^2) - F(-s) holds.                                         */
/* ------------------------------------------------------------------------ */
#define OR_WN 48
static double or_wa[OR_WN];
static double or_wL;
static int or_wready;

/* Fills the coefficient table; called once when the library is loaded,
   before any evaluation. */
void or_init(void)
{
    if (or_wready) return;
    const int M = 8192;
    const double L = pow(2.0, -0.25) * sqrt((double)OR_WN);
    for (int n = 1; n <= OR_WN; ++n) {
        double acc = 0.0;
        for (int j = 0; j < M; ++j) {
            const double th = -OR_PI + (j + 0.5) * (2.0 * OR_PI / M);
            const double t = L * tan(0.5 * th);
            acc += (L * L + t * t) * exp(-t * t) * cos(n * th);
        }
        or_wa[n - 1] = acc / M;
    }
    or_wL = L;
    or_wready = 1;
}

static double complex or_faddeeva_upper(double complex s)
{
    const double complex d = or_wL - I * s;
    const double complex Z = (or_wL + I * s) / d;
    double complex p = 0.0;
    for (int n = OR_WN - 1; n >= 0; --n) p = p * Z + or_wa[n];
    return 2.0 * p / (d * d) + 1.0 / (sqrt(OR_PI) * d);
}

static double complex or_faddeeva(double complex s)
{
    if (!or_wready) return NAN;                    /* or_init was not called */
    if (cimag(s) >= 0.0) return or_faddeeva_upper(s);
    return 2.0 * cexp(-s * s) - or_faddeeva_upper(-s);
}

/* ------------------------------------------------------------------------ */
/* Gaussian conformal map (Sec. 2, Fig. 1(b), Fig. 4).  Reading: the virtual  */
/* half plane v >= 0 (flat mirror at v = 0) maps onto the region above the   */
/* bump by                                                                   */
/*     z(w) = w + i h F(w / w_b),                                            */
/* the analytic function of the upper half plane whose boundary image is    */
/*     x = u - h Im F(u/w_b),  y = h Re F(u/w_b) = h exp(-(u/w_b)^2):        */
/* in the shallow-bump limit this is Eq. 5, and the exact bump is implicit  */
/* in x.  n = |dw/dz| = 1/|z'(w)|.  (h = A, w_b = gauss_w.)                  */
/* ------------------------------------------------------------------------ */
static void or_gauss_z(const or_scene* sc, double complex w, double complex* z, double complex* dz,
                       double complex* d2z)
{
    const double hb = sc->A, wb = sc->gauss_w;
    const double complex s = w / wb;
    const double complex F = or_faddeeva(s);
    const double complex F1 = -2.0 * s * F + 2.0 * I / sqrt(OR_PI);   /* F'  */
    const double complex F2 = -2.0 * F - 2.0 * s * F1;                 /* F'' */
    if (z) *z = w + I * hb * F;
    if (dz) *dz = 1.0 + I * hb * F1 / wb;
    if (d2z) *d2z = I * hb * F2 / (wb * wb);
}

/* Virtual coordinate w of the physical point x + i y: Newton's method on
   z(w) = x + i y from w = x + i y, each step limited to w_b / 4. */
static double complex or_gauss_w(const or_scene* sc, double x, double y, int* iters)
{
    const double complex zt = x + I * y;
    double complex w = zt;
    *iters = 0;
    for (int it = 1; it <= 100; ++it) {
        double complex z, dz;
        or_gauss_z(sc, w, &z, &dz, NULL);
        double complex dw = (z - zt) / dz;
        const double m = cabs(dw), cap = 0.25 * sc->gauss_w;
        if (m > cap) dw *= cap / m;
        w -= dw;
        *iters = it;
        if (!(m > 4.0 * DBL_EPSILON * (1.0 + cabs(w)))) break;
    }
    return w;
}

/* Index n and grad n at (x, y), with the virtual coordinate w (v = Im w is
   the mirror's event function) and g = dw/dz (grad v = (Im g, Re g)).
   Grating: Eq. 1 and Eq. 12, with w = z + i W0/k and g = 1/(1 + W0).
   Gaussian cloak: n = |g|, and with g' = d^2w/dz^2 = -z''(w) g^3,
   grad(n^2)/2 = (Re(conj(g) g'), -Im(conj(g) g')). */
static void or_medium(const or_scene* sc, double x, double y, double complex* wv, double complex* gw,
                      double* n, double gn[3], counters* cnt)
{
    int it;
    if (sc->mirror == 2) {
        const double complex w = or_gauss_w(sc, x, y, &it);
        if (cnt) { cnt->halley += it; cnt->evals += 1; }
        double complex dz, d2z;
        or_gauss_z(sc, w, NULL, &dz, &d2z);
        const double complex g = 1.0 / dz;
        const double complex g1 = -d2z * g * g * g;
        const double complex q = conj(g) * g1;
        *n = cabs(g);
        gn[0] = creal(q) / *n;
        gn[1] = -cimag(q) / *n;
        gn[2] = 0.0;
        if (wv) *wv = w;
        if (gw) *gw = g;
        return;
    }
    const double k = 2.0 * OR_PI / sc->Lambda;
    const double complex Wl = or_w0_c(or_zeta(sc, x, y), &it);
    if (wv) *wv = (x + I * y) + I * Wl / k;
    if (gw) *gw = 1.0 / (1.0 + Wl);
    if (cnt) { cnt->halley += it; cnt->evals += 1; }
    const double complex onepw = 1.0 + Wl;
    const double m = cabs(onepw);                 /* |1 + W0| */
    const double re1 = creal(onepw);               /* Re(1 + W0) */
    const double imw = cimag(Wl);                  /* Im(W0)     */
    *n = 1.0 / m;
    gn[0] = (2.0 * re1 * imw / (m * m) - imw) * k / (m * m * m);
    gn[1] = ((imw * imw - re1 * re1) / (m * m) + re1) * k / (m * m * m);
    gn[2] = 0.0;
    if (sc->flags & OR_FLAG_REFERENCED) {         /* n / n_min with n_min = 1 / (1 + kA) */
        const double sidx = 1.0 + k * sc->A;
        *n *= sidx;
        gn[0] *= sidx;
        gn[1] *= sidx;
    }
}

/* Index of the homogeneous plate: 1/n_min of the grating cloak, 1 + kA. */
static double or_plate_index(const or_scene* sc) { return 1.0 + 2.0 * OR_PI * sc->A / sc->Lambda; }

/* Unpolarised Fresnel reflectance R = (rs^2 + rp^2)/2 for a ray going from
   index n1 into index n2, from the normal components of its momentum on both
   sides (|p| = n, so n1 cos(theta_1) = |pn1| and n2 cos(theta_2) = |pn2|):
     rs = (n1 cos1 - n2 cos2) / (n1 cos1 + n2 cos2),
     rp = (n2 cos1 - n1 cos2) / (n2 cos1 + n1 cos2)
        = (n2^2 |pn1| - n1^2 |pn2|) / (n2^2 |pn1| + n1^2 |pn2|). */
static double or_fresnel_R(double n1, double n2, double pn1, double pn2)
{
    const double a = fabs(pn1), b = fabs(pn2);
    const double rs = (a - b) / (a + b);
    const double rp = (n2 * n2 * a - n1 * n1 * b) / (n2 * n2 * a + n1 * n1 * b);
    return 0.5 * (rs * rs + rp * rp);
}

/* Right-hand side in the Hamiltonian parameter: dr/dtau = p, dp/dtau = n grad n.
   Outside the cloak box the medium is air (n = 1) and the force vanishes (Sec. 3);
   the integrator is only run inside the box, so the force is always Eq. 12's. */
static void or_rhs(const or_scene* sc, const double s[6], double ds[6], counters* cnt)
{
    double n, gn[3];
    or_medium(sc, s[0], s[1], NULL, NULL, &n, gn, cnt);
    ds[0] = s[3]; ds[1] = s[4]; ds[2] = s[5];
    if (sc->integrator == 2) {
        /* Eq. 11 in physical time t (c0 = 1): the state is (r, v), |v| = 1/n,
           dv/dt = (|v|^2 grad n - 2 (grad n . v) v) / n */
        const double v2 = s[3] * s[3] + s[4] * s[4] + s[5] * s[5];
        const double gv = gn[0] * s[3] + gn[1] * s[4] + gn[2] * s[5];
        for (int a = 0; a < 3; ++a) ds[3 + a] = (v2 * gn[a] - 2.0 * gv * s[3 + a]) / n;
        return;
    }
    ds[3] = n * gn[0]; ds[4] = n * gn[1]; ds[5] = n * gn[2];
}

/* Classical fourth-order Runge-Kutta step of size h. */
static void or_rk4(const or_scene* sc, const double s[6], double h, double out[6], counters* cnt)
{
    double k1[6], k2[6], k3[6], k4[6], t[6];
    or_rhs(sc, s, k1, cnt);
    for (int i = 0; i < 6; ++i) t[i] = s[i] + 0.5 * h * k1[i];
    or_rhs(sc, t, k2, cnt);
    for (int i = 0; i < 6; ++i) t[i] = s[i] + 0.5 * h * k2[i];
    or_rhs(sc, t, k3, cnt);
    for (int i = 0; i < 6; ++i) t[i] = s[i] + h * k3[i];
    or_rhs(sc, t, k4, cnt);
    for (int i = 0; i < 6; ++i) out[i] = s[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* Dormand & Prince (1980) RK5(4)7M tableau. */
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84},
};
static const double DP_B5[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0};
static const double DP_B4[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200,
                                187.0 / 2100, 1.0 / 40};

/* One Dormand-Prince step of size h from s, given k1 = f(s).  Returns the
   fifth-order solution, the fourth-order solution and f at the fifth-order
   point (first-same-as-last). */
static void or_dp45(const or_scene* sc, const double s[6], const double k1[6], double h,
                    double y5[6], double y4[6], double k7[6], counters* cnt)
{
    double k[7][6], t[6];
    memcpy(k[0], k1, sizeof(double) * 6);
    for (int st = 1; st < 6; ++st) {
        for (int i = 0; i < 6; ++i) {
            double acc = 0.0;
            for (int j = 0; j < st; ++j) acc += DP_A[st][j] * k[j][i];
            t[i] = s[i] + h * acc;
        }
        or_rhs(sc, t, k[st], cnt);
    }
    for (int i = 0; i < 6; ++i) {
        double a5 = 0.0;
        for (int j = 0; j < 6; ++j) a5 += DP_B5[j] * k[j][i];
        y5[i] = s[i] + h * a5;
    }
    or_rhs(sc, y5, k[6], cnt);
    for (int i = 0; i < 6; ++i) {
        double a4 = 0.0;
        for (int j = 0; j < 7; ++j) a4 += DP_B4[j] * k[j][i];
        y4[i] = s[i] + h * a4;
        k7[i] = k[6][i];
    }
}

/* ------------------------------------------------------------------------ */
/* Trochoid grating (Eq. 2): x = xi - A sin(k xi), y = A cos(k xi).          */
/* ------------------------------------------------------------------------ */

/* Solve E - e sin E = M (Kepler's equation, e = kA < 1) by Newton's method
   safeguarded by bisection on [M - e, M + e]. */
static double or_kepler(double M, double e)
{
    double lo = M - e, hi = M + e, E = M;
    for (int it = 0; it < 200; ++it) {
        double f = E - e * sin(E) - M;
        if (f > 0) hi = E; else lo = E;
        double En = E - f / (1.0 - e * cos(E));
        if (!(En > lo && En < hi)) En = 0.5 * (lo + hi);
        double d = fabs(En - E);
        E = En;
        if (d <= 4.0 * DBL_EPSILON * fmax(1.0, fabs(E))) break;
    }
    return E;
}

/* Grating parameter xi at abscissa x (inverse of the first line of Eq. 2). */
static double or_trochoid_xi(const or_scene* sc, double x)
{
    const double k = 2.0 * OR_PI / sc->Lambda;
    return or_kepler(k * x, k * sc->A) / k;
}

/* Surface height y_s(x) (Eq. 2). */
static double or_trochoid_y(const or_scene* sc, double x)
{
    const double k = 2.0 * OR_PI / sc->Lambda;
    return sc->A * cos(k * or_trochoid_xi(sc, x));
}

/* Upward unit normal of the grating at abscissa x, from the tangent of Eq. 2:
   (dx/dxi, dy/dxi) = (1 - kA cos k xi, -kA sin k xi). */
static void or_trochoid_normal(const or_scene* sc, double x, double N[3])
{
    const double k = 2.0 * OR_PI / sc->Lambda;
    const double xi = or_trochoid_xi(sc, x);
    const double nx = k * sc->A * sin(k * xi), ny = 1.0 - k * sc->A * cos(k * xi);
    const double l = sqrt(nx * nx + ny * ny);
    N[0] = nx / l; N[1] = ny / l; N[2] = 0.0;
}

/* Slope dy_s/dx of the grating at abscissa x. */
static double or_trochoid_slope(const or_scene* sc, double x)
{
    const double k = 2.0 * OR_PI / sc->Lambda;
    const double xi = or_trochoid_xi(sc, x);
    return -k * sc->A * sin(k * xi) / (1.0 - k * sc->A * cos(k * xi));
}

/* ------------------------------------------------------------------------ */
/* Gaussian bump, the image of v = 0 under the Gaussian conformal map:      */
/* x = u - h Im F(u/w_b), y = h exp(-(u/w_b)^2) (Eq. 5 in the shallow limit). */
/* ------------------------------------------------------------------------ */

/* Bump parameter u at abscissa x; x(u) is increasing for h/w_b < sqrt(pi)/2
   and |x - u| <= 0.62 h, so Newton's method is guarded by bisection on
   [x - h, x + h]. */
static double or_bump_u(const or_scene* sc, double x)
{
    const double hb = sc->A, wb = sc->gauss_w;
    double lo = x - hb, hi = x + hb, u = x;
    for (int it = 0; it < 200; ++it) {
        const double complex F = or_faddeeva(u / wb);
        const double f = u - hb * cimag(F) - x;
        if (f > 0) hi = u; else lo = u;
        const double dxdu = 1.0 - (hb / wb) * cimag(-2.0 * (u / wb) * F + 2.0 * I / sqrt(OR_PI));
        double un = u - f / dxdu;
        if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);
        const double d = fabs(un - u);
        u = un;
        if (d <= 4.0 * DBL_EPSILON * fmax(1.0, fabs(u))) break;
    }
    return u;
}

/* Tangent (dx/du, dy/du) = z'(u) of the bump at parameter u. */
static void or_bump_tangent(const or_scene* sc, double u, double T[2])
{
    double complex dz;
    or_gauss_z(sc, u, NULL, &dz, NULL);
    T[0] = creal(dz); T[1] = cimag(dz);
}

/* Mirror surface of kind 1 (trochoid) or 2 (bump): height, slope and
   upward unit normal at abscissa x. */
static double or_surface_y(const or_scene* sc, double x)
{
    if (sc->mirror != 2) return or_trochoid_y(sc, x);
    const double u = or_bump_u(sc, x) / sc->gauss_w;
    return sc->A * exp(-u * u);
}

static double or_surface_slope(const or_scene* sc, double x)
{
    if (sc->mirror != 2) return or_trochoid_slope(sc, x);
    double T[2];
    or_bump_tangent(sc, or_bump_u(sc, x), T);
    return T[1] / T[0];
}

static void or_surface_normal(const or_scene* sc, double x, double N[3])
{
    if (sc->mirror != 2) { or_trochoid_normal(sc, x, N); return; }
    double T[2];
    or_bump_tangent(sc, or_bump_u(sc, x), T);
    const double l = sqrt(T[0] * T[0] + T[1] * T[1]);
    N[0] = -T[1] / l; N[1] = T[0] / l; N[2] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Illinois (modified regula falsi) root finder on a bracket [a, b] with     */
/* fa > 0 >= fb.  The function is given by a callback.                       */
/* ------------------------------------------------------------------------ */
typedef double (*or_fn)(void* ctx, double t);

static double or_illinois(or_fn f, void* ctx, double a, double fa, double b, double fb,
                          double ftol, double xtol)
{
    if (fb == 0.0) return b;
    int side = 0;
    double c = b;
    for (int it = 0; it < 200; ++it) {
        c = b - fb * (b - a) / (fb - fa);
        if (!(c > a && c < b)) c = 0.5 * (a + b);
        double fc = f(ctx, c);
        if (fabs(fc) <= ftol) return c;
        if (fc < 0) {
            b = c; fb = fc;
            if (side == -1) fa *= 0.5;
            side = -1;
        } else {
            a = c; fa = fc;
            if (side == +1) fb *= 0.5;
            side = +1;
        }
        if (b - a <= xtol * (1.0 + fabs(b))) return b;
    }
    return c;
}

/* ------------------------------------------------------------------------ */
/* Straight ray in air against the mirror.                                   */
/* ------------------------------------------------------------------------ */
typedef struct line_ctx {
    const or_scene* sc;
    double X[3], p[3];
    int deflate;            /* divide by t: the ray starts on the surface */
} line_ctx;

static double or_line_height(void* vctx, double t)
{
    line_ctx* c = (line_ctx*)vctx;
    double h = (c->X[1] + t * c->p[1]) - or_surface_y(c->sc, c->X[0] + t * c->p[0]);
    return c->deflate ? h / t : h;
}

/* First t > 0 at which the line X + t p meets the trochoid (Eq. 2) or the
   Gaussian bump, or INFINITY.  Inside the band the surface spans (y in
   [-A, A], resp. [0, h]) the line is marched in increments that move the
   point by at most Lambda/(8 pi) (resp. w_b/8) in the xy-plane; the first
   increment at whose end the line is at or below the surface brackets the
   hit, which is then refined.  When the line starts on the surface (just
   reflected there), the zero at t = 0 is divided out. */
static double or_trochoid_line_hit(const or_scene* sc, const double X[3], const double p[3],
                                   int on_surface)
{
    const int bump = sc->mirror == 2;
    const double ylo = bump ? 0.0 : -sc->A, yhi = sc->A;
    const double dxy = sqrt(p[0] * p[0] + p[1] * p[1]);
    if (dxy < 1e-300) return INFINITY;
    if (p[1] >= 0.0 && X[1] >= yhi) return INFINITY;
    double t0 = 0.0;
    if (X[1] > yhi) t0 = (yhi - X[1]) / p[1];
    double t_end;
    if (p[1] < 0.0) t_end = (ylo - X[1]) / p[1];
    else if (p[1] > 0.0) t_end = (yhi - X[1]) / p[1];
    else t_end = t0 + 2.0 * (bump ? 20.0 * sc->gauss_w : sc->Lambda) / fabs(p[0]);
    const double dt = bump ? 0.125 * sc->gauss_w / dxy : 0.25 / (2.0 * OR_PI / sc->Lambda * dxy);
    line_ctx ctx = {sc, {X[0], X[1], X[2]}, {p[0], p[1], p[2]}, 0};
    double ta = t0, ha;
    int first = on_surface && t0 == 0.0;
    if (first) {
        /* derivative of the height along the line at t = 0 */
        ha = p[1] - or_surface_slope(sc, X[0]) * p[0];
        if (!(ha > 0.0)) ha = 1e-300;
    } else {
        ha = or_line_height(&ctx, ta);
        if (ha <= 0.0) return ta;               /* already on or below the surface */
    }
    for (;;) {
        double tb = fmin(ta + dt, t_end);
        /* a ray leaving the surface cannot meet it again within 1e-9 Lambda */
        if (first && tb <= 1e-9 * sc->Lambda) {
            if (tb >= t_end) return INFINITY;
            tb = fmin(1e-9 * sc->Lambda, t_end);
        }
        double hb = or_line_height(&ctx, tb);
        /* a descending line meets the surface by the bottom of its band at the latest */
        if (tb >= t_end && p[1] < 0.0 && hb > 0.0) hb = 0.0;
        if (hb <= 0.0) {
            if (first) {
                ctx.deflate = 1;
                double hbd = hb / tb;
                double r = or_illinois(or_line_height, &ctx, ta, ha, tb, hbd, 1e-13 * sc->Lambda / tb,
                                       1e-15 * sc->Lambda);
                return r;
            }
            return or_illinois(or_line_height, &ctx, ta, ha, tb, hb, 1e-13 * sc->Lambda, 1e-15 * sc->Lambda);
        }
        if (tb >= t_end) break;
        first = 0;
        ta = tb; ha = hb;
    }
    return INFINITY;
}

/* First t > 0 at which the line meets the flat mirror y = 0, or INFINITY. */
static double or_flat_line_hit(const double X[3], const double p[3])
{
    if (p[1] < 0.0 && X[1] > 0.0) return -X[1] / p[1];
    return INFINITY;
}

/* ------------------------------------------------------------------------ */
/* Cloak box.                                                                */
/* ------------------------------------------------------------------------ */
/* The box spans |x|, |z| <= E/2 and, in y, H from the grating's troughs
   (y = -A) or from the flat mirror under the bump (y = 0). */
static double or_box_bottom(const or_scene* sc)
{
    if (sc->mirror == 2 || (sc->flags & OR_FLAG_PLATE)) return 0.0;   /* plate: on the flat mirror */
    return -sc->A;
}

static double or_box_top(const or_scene* sc)
{
    return (sc->mirror == 2 ? 0.0 : -sc->A) + sc->H;
}

static void or_box(const or_scene* sc, double lo[3], double hi[3])
{
    lo[0] = -0.5 * sc->E; hi[0] = 0.5 * sc->E;
    lo[1] = or_box_bottom(sc); hi[1] = or_box_top(sc);
    lo[2] = -0.5 * sc->E; hi[2] = 0.5 * sc->E;
}

/* Entry of the line X + t p (t > 0) into the box by the slab method; returns
   INFINITY when it misses and sets the entry face (event id). */
static double or_box_entry(const or_scene* sc, const double X[3], const double p[3], int* face)
{
    double lo[3], hi[3];
    or_box(sc, lo, hi);
    double tn = -INFINITY, tf = INFINITY;
    int fn = EV_NONE;
    for (int a = 0; a < 3; ++a) {
        if (p[a] == 0.0) {
            if (X[a] < lo[a] || X[a] > hi[a]) return INFINITY;
            continue;
        }
        double t1 = (lo[a] - X[a]) / p[a], t2 = (hi[a] - X[a]) / p[a];
        int f1, f2;                      /* faces crossed at t1 (lo) and t2 (hi) */
        if (a == 0) { f1 = EV_XM; f2 = EV_XP; }
        else if (a == 1) { f1 = EV_NONE; f2 = EV_TOP; }
        else { f1 = EV_ZM; f2 = EV_ZP; }
        double tmin = t1, tmax = t2;
        int fmin_ = f1;
        if (t1 > t2) { tmin = t2; tmax = t1; fmin_ = f2; }
        if (tmin > tn) { tn = tmin; fn = fmin_; }
        if (tmax < tf) tf = tmax;
    }
    if (!(tn <= tf) || !(tn > 1e-12 * sc->Lambda)) return INFINITY;
    *face = fn;
    return tn;
}

static void or_face_normal(int face, double N[3])
{
    N[0] = N[1] = N[2] = 0.0;
    switch (face) {
        case EV_TOP: N[1] = 1.0; break;
        case EV_XP: N[0] = 1.0; break;
        case EV_XM: N[0] = -1.0; break;
        case EV_ZP: N[2] = 1.0; break;
        case EV_ZM: N[2] = -1.0; break;
        default: N[1] = -1.0; break;
    }
}

/* Event functions inside the box: positive while the ray is in the open cloak
   region, negative once it has crossed the grating (v < 0) or a face. */
static double or_event_g(const or_scene* sc, int ev, const double s[6], counters* cnt)
{
    switch (ev) {
        case EV_GRATING: {
            double complex wv;
            double n, gn[3];
            or_medium(sc, s[0], s[1], &wv, NULL, &n, gn, cnt);
            return cimag(wv);                      /* v = Im w (grating: y + Re W0 / k) */
        }
        case EV_TOP: return or_box_top(sc) - s[1];
        case EV_XP: return 0.5 * sc->E - s[0];
        case EV_XM: return 0.5 * sc->E + s[0];
        case EV_ZP: return 0.5 * sc->E - s[2];
        default: return 0.5 * sc->E + s[2];
    }
}

/* Gradient of the event function at s (xy components suffice; z only for z faces). */
static void or_event_grad(const or_scene* sc, int ev, const double s[6], double g[3], counters* cnt)
{
    g[0] = g[1] = g[2] = 0.0;
    if (ev == EV_GRATING) {
        /* grad v = (Im g, Re g) since w is analytic with dw/dz = g (grating: g = 1/(1+W0)) */
        double complex gw;
        double n, gn[3];
        or_medium(sc, s[0], s[1], NULL, &gw, &n, gn, cnt);
        g[0] = cimag(gw); g[1] = creal(gw);
        return;
    }
    double N[3];
    or_face_normal(ev, N);
    g[0] = -N[0]; g[1] = -N[1]; g[2] = -N[2];
}

/* ------------------------------------------------------------------------ */
/* Integrator step with an optional partial step for event location.         */
/* ------------------------------------------------------------------------ */
typedef struct step_ctx {
    const or_scene* sc;
    double s[6], k1[6], h;
    int ev, deflate;
    counters* cnt;
} step_ctx;

static void or_partial_step(step_ctx* c, double theta, double out[6])
{
    if (c->sc->integrator != 1) {
        or_rk4(c->sc, c->s, theta * c->h, out, c->cnt);
    } else {
        double y4[6], k7[6];
        or_dp45(c->sc, c->s, c->k1, theta * c->h, out, y4, k7, c->cnt);
    }
}

static double or_event_along_step(void* vctx, double theta)
{
    step_ctx* c = (step_ctx*)vctx;
    double st[6];
    or_partial_step(c, theta, st);
    double g = or_event_g(c->sc, c->ev, st, c->cnt);
    return c->deflate ? g / theta : g;
}

/* Root theta in (0, 1] of g_ev(Phi_{theta h}(s)) = 0 given g_ev(s1) = g1 < 0. */
static double or_locate_event(step_ctx* c, int ev, int on_surface, double g1)
{
    c->ev = ev;
    c->deflate = 0;
    double ga;
    if (on_surface) {
        double gr[3];
        or_event_grad(c->sc, ev, c->s, gr, c->cnt);
        ga = c->h * (gr[0] * c->s[3] + gr[1] * c->s[4] + gr[2] * c->s[5]);
        if (!(ga > 0.0)) ga = 1e-300;
        c->deflate = 1;
    } else {
        ga = or_event_g(c->sc, ev, c->s, c->cnt);
        if (!(ga > 0.0)) return 0.0;
    }
    return or_illinois(or_event_along_step, c, 0.0, ga, 1.0, g1, 1e-13 * c->sc->Lambda, 1e-15);
}

/* ------------------------------------------------------------------------ */
/* Camera, jitter and background.                                            */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood 2014): the m-th output of the generator
   seeded with `seed` is mix(seed + m * 0x9E3779B97F4A7C15). */
static uint64_t or_splitmix64(uint64_t seed, uint64_t m)
{
    uint64_t z = seed + m * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static double or_uniform24(uint64_t seed, uint64_t m)
{
    return (double)(or_splitmix64(seed, m) >> 40) * (1.0 / 16777216.0);
}

typedef struct camera { double C[3], f[3], r[3], u[3], tx, ty; } camera;

static void or_normalize(double v[3])
{
    double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= l; v[1] /= l; v[2] /= l;
}

static void or_cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static double or_dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Pinhole camera (Sec. 4): at distance D from the origin, elevation theta_e,
   azimuth phi, looking at the origin; horizontal full FOV hfov, square pixels. */
static void or_camera(const or_scene* sc, camera* cam)
{
    const double te = sc->elev_deg * OR_PI / 180.0, ph = sc->azim_deg * OR_PI / 180.0;
    const double D = sc->cam_dist;
    cam->C[0] = -D * cos(te) * cos(ph);
    cam->C[1] = D * sin(te);
    cam->C[2] = -D * cos(te) * sin(ph);
    for (int i = 0; i < 3; ++i) cam->f[i] = -cam->C[i] / D;
    const double up[3] = {0.0, 1.0, 0.0};
    or_cross(cam->f, up, cam->r);
    or_normalize(cam->r);
    or_cross(cam->r, cam->f, cam->u);
    cam->tx = tan(0.5 * sc->hfov_deg * OR_PI / 180.0);
    cam->ty = cam->tx * (double)sc->height / (double)sc->width;
}

/* Sub-pixel offset of sample s of pixel (i, j): pixel centre for one sample,
   an m x m stratified grid with one uniform offset per cell for spp = m^2,
   two uniforms otherwise. */
static void or_jitter(const or_scene* sc, int i, int j, int s, double* ox, double* oy)
{
    if (sc->spp == 1) { *ox = 0.5; *oy = 0.5; return; }
    const int wout = sc->centre_line ? 1 : sc->width;
    const uint64_t c = (((uint64_t)sc->scene_id * (uint64_t)sc->height + (uint64_t)i) * (uint64_t)wout +
                        (uint64_t)j) * (uint64_t)sc->spp + (uint64_t)s;
    const double u1 = or_uniform24(sc->seed, 2 * c + 1), u2 = or_uniform24(sc->seed, 2 * c + 2);
    int m = (int)floor(sqrt((double)sc->spp) + 0.5);
    if (m * m == sc->spp) {
        *ox = ((double)(s % m) + u1) / m;
        *oy = ((double)(s / m) + u2) / m;
    } else {
        *ox = u1; *oy = u2;
    }
}

static void or_camera_ray(const or_scene* sc, const camera* cam, int i, int j, int s, double d[3])
{
    double ox, oy;
    or_jitter(sc, i, j, s, &ox, &oy);
    const double px = sc->centre_line ? 0.0 : 2.0 * ((double)j + ox) / sc->width - 1.0;
    const double py = 1.0 - 2.0 * ((double)i + oy) / sc->height;
    for (int a = 0; a < 3; ++a) d[a] = cam->f[a] + px * cam->tx * cam->r[a] + py * cam->ty * cam->u[a];
    or_normalize(d);
}

/* Background plane standing in for the photograph of Fig. 2(a): normal to the
   mirrored view axis f_r = (f_x, -f_y, f_z), through D f_r. */
static int or_background(const or_scene* sc, const camera* cam, const double X[3], const double d[3],
                         double rgb[3])
{
    const double fr[3] = {cam->f[0], -cam->f[1], cam->f[2]};
    const double dn = or_dot(d, fr);
    rgb[0] = rgb[1] = rgb[2] = 0.0;
    if (!(dn > 0.0)) return ST_SKY;
    double Pb[3], ur[3], rel[3], Y[3];
    for (int a = 0; a < 3; ++a) Pb[a] = sc->cam_dist * fr[a];
    for (int a = 0; a < 3; ++a) rel[a] = Pb[a] - X[a];
    const double t = or_dot(rel, fr) / dn;
    for (int a = 0; a < 3; ++a) Y[a] = X[a] + t * d[a] - Pb[a];
    or_cross(cam->r, fr, ur);
    const double s = or_dot(Y, cam->r), tt = or_dot(Y, ur);
    if (sc->background == 0) {
        const long long a = (long long)floor(s / sc->bg_cell), b = (long long)floor(tt / sc->bg_cell);
        const double* c = (((a + b) % 2) == 0) ? sc->colour0 : sc->colour1;
        rgb[0] = c[0]; rgb[1] = c[1]; rgb[2] = c[2];
    } else {
        const int N = sc->tex_size;
        const double U = s / sc->tex_texel - 0.5, V = tt / sc->tex_texel - 0.5;
        const double fu0 = floor(U), fv0 = floor(V);
        const double fu = U - fu0, fv = V - fv0;
        long long u0 = ((long long)fu0 % N + N) % N, v0 = ((long long)fv0 % N + N) % N;
        long long u1 = (u0 + 1) % N, v1 = (v0 + 1) % N;
        const double val = (1.0 - fu) * (1.0 - fv) * sc->tex[v0 * N + u0] + fu * (1.0 - fv) * sc->tex[v0 * N + u1] +
                           (1.0 - fu) * fv * sc->tex[v1 * N + u0] + fu * fv * sc->tex[v1 * N + u1];
        rgb[0] = rgb[1] = rgb[2] = val;
    }
    return ST_OK;
}

/* ------------------------------------------------------------------------ */
/* Full path of one ray.                                                     */
/* ------------------------------------------------------------------------ */
typedef struct traj_buf { double* data; int cap, len; } traj_buf;

static void traj_push(traj_buf* tb, const double s[6])
{
    if (!tb || !tb->data || tb->len >= tb->cap) return;
    memcpy(tb->data + 6 * (size_t)tb->len, s, sizeof(double) * 6);
    tb->len++;
}

static int or_finite6(const double s[6])
{
    for (int i = 0; i < 6; ++i) if (!isfinite(s[i])) return 0;
    return 1;
}

/* A Fresnel branch waiting to be traced: where it starts, its momentum, its
   weight and the counters of the path it split from. */
typedef struct or_branch {
    double X[3], p[3], w;
    int medium, surface, bounces, events;
    int64_t steps;
} or_branch;

/* Queue a Fresnel branch (reflected momentum pr at X) if the path may split. */
static void or_push_branch(or_branch* br, int* nbr, const double X[3], const double pr[3], double w, int medium,
                           int surface, int bounces, int events, int64_t steps)
{
    if (!br || *nbr >= OR_MAX_BRANCHES) return;
    or_branch* b = &br[(*nbr)++];
    for (int a = 0; a < 3; ++a) { b->X[a] = X[a]; b->p[a] = pr[a]; }
    b->w = w;
    b->medium = medium;
    b->surface = surface;
    b->bounces = bounces;
    b->events = events;
    b->steps = steps;
}

/* Trace one path from position X with momentum p in the given medium.  In air
   p is the unit direction; in the box and the plate |p| = n.  `surface` names
   the surface the ray starts on (EV_NONE, EV_GRATING or a face), whose zero at
   the start is divided out when looking for the next hit.  w0 is the path's
   weight; with br != NULL the path may start Fresnel branches (queued in br).
   The record gets the path's exit, counters and its own (unweighted) colour;
   *w_out its final weight. */
static void or_trace_path(const or_scene* sc, const camera* cam, const double X0[3], const double p0[3],
                          int medium, int surface, double w0, int bounces0, int events0, int64_t steps0,
                          or_branch* br, int* nbr, or_record* rec, double* w_out, traj_buf* tb)
{
    double X[3] = {X0[0], X0[1], X0[2]}, p[3] = {p0[0], p0[1], p0[2]};
    counters cnt = {0, 0};
    int64_t steps = steps0;
    int bounces = bounces0, events = events0, status = ST_OK;
    double w = w0;
    const int fresnel = (sc->flags & OR_FLAG_FRESNEL) != 0;
    const int plate = (sc->flags & OR_FLAG_PLATE) != 0;
    double rgb[3] = {0.0, 0.0, 0.0};
    for (;;) {
        if (bounces > sc->max_bounces) { status = ST_MAX_BOUNCES; break; }
        if (medium == MED_AIR) {
            double t_m = sc->mirror ? or_trochoid_line_hit(sc, X, p, surface == EV_GRATING)
                                    : or_flat_line_hit(X, p);
            int face = EV_NONE;
            double t_b = (sc->cloak || plate) ? or_box_entry(sc, X, p, &face) : INFINITY;
            if (t_b < t_m) {
                for (int a = 0; a < 3; ++a) X[a] += t_b * p[a];
                double Nf[3];
                or_face_normal(face, Nf);              /* outward normal of the entry face */
                double n;
                if (plate) {
                    n = or_plate_index(sc);
                } else {
                    double gn[3];
                    or_medium(sc, X[0], X[1], NULL, NULL, &n, gn, &cnt);
                }
                const double pn = or_dot(p, Nf);
                double pt[3];
                for (int a = 0; a < 3; ++a) pt[a] = p[a] - pn * Nf[a];
                const double pt2 = or_dot(pt, pt);
                if (n * n < pt2) {                      /* total reflection off the box */
                    for (int a = 0; a < 3; ++a) p[a] -= 2.0 * pn * Nf[a];
                    bounces++;
                    surface = EV_NONE;
                    continue;
                }
                const double pn_in = sqrt(n * n - pt2);
                if (fresnel) {
                    const double R = or_fresnel_R(1.0, n, pn, pn_in);
                    double pr[3];
                    for (int a = 0; a < 3; ++a) pr[a] = p[a] - 2.0 * pn * Nf[a];
                    or_push_branch(br, nbr, X, pr, w * R, MED_AIR, EV_NONE, bounces, events, steps);
                    w *= 1.0 - R;
                }
                for (int a = 0; a < 3; ++a) p[a] = pt[a] - pn_in * Nf[a];
                medium = plate ? MED_PLATE : MED_BOX;
                surface = face;
                continue;
            }
            if (t_m < INFINITY) {
                for (int a = 0; a < 3; ++a) X[a] += t_m * p[a];
                double N[3] = {0.0, 1.0, 0.0};
                if (sc->mirror) or_surface_normal(sc, X[0], N);
                const double pn = or_dot(p, N);
                for (int a = 0; a < 3; ++a) p[a] -= 2.0 * pn * N[a];
                bounces++;
                surface = EV_GRATING;
                continue;
            }
            status = or_background(sc, cam, X, p, rgb);
            break;
        }

        if (medium == MED_PLATE) {
            /* Inside the homogeneous plate: a straight segment to the mirror
               (y = 0), the top or a side face. */
            double lo[3], hi[3];
            or_box(sc, lo, hi);
            double tmin = INFINITY;
            int hit = EV_NONE;
            for (int a = 0; a < 3; ++a) {
                if (p[a] == 0.0) continue;
                const double t = ((p[a] > 0.0 ? hi[a] : lo[a]) - X[a]) / p[a];
                int f;
                if (a == 0) f = p[a] > 0.0 ? EV_XP : EV_XM;
                else if (a == 1) f = p[a] > 0.0 ? EV_TOP : EV_GRATING;   /* EV_GRATING: the mirror */
                else f = p[a] > 0.0 ? EV_ZP : EV_ZM;
                if (t < tmin) { tmin = t; hit = f; }
            }
            if (!(tmin < INFINITY) || hit == EV_NONE) { status = ST_NAN; break; }
            if (tmin < 0.0) tmin = 0.0;
            for (int a = 0; a < 3; ++a) X[a] += tmin * p[a];
            if (hit == EV_GRATING) {
                X[1] = 0.0;
                p[1] = -p[1];
                bounces++;
                surface = EV_GRATING;
                continue;
            }
            double Nf[3];
            or_face_normal(hit, Nf);
            const double pn = or_dot(p, Nf);
            double pt[3];
            for (int a = 0; a < 3; ++a) pt[a] = p[a] - pn * Nf[a];
            const double pt2 = or_dot(pt, pt);
            if (pt2 >= 1.0) {                           /* total internal reflection */
                for (int a = 0; a < 3; ++a) p[a] -= 2.0 * pn * Nf[a];
                bounces++;
                surface = hit;
                continue;
            }
            const double pn_out = sqrt(1.0 - pt2);
            if (fresnel) {
                const double R = or_fresnel_R(or_plate_index(sc), 1.0, pn, pn_out);
                double pr[3];
                for (int a = 0; a < 3; ++a) pr[a] = p[a] - 2.0 * pn * Nf[a];
                or_push_branch(br, nbr, X, pr, w * R, MED_PLATE, hit, bounces, events, steps);
                w *= 1.0 - R;
            }
            for (int a = 0; a < 3; ++a) p[a] = pt[a] + pn_out * Nf[a];
            medium = MED_AIR;
            surface = EV_NONE;
            continue;
        }

        /* Inside the cloak: integrate the ray ODE step by step.  p is the
           momentum (|p| = n); the time form of Eq. 11 (integrator 2) carries
           the velocity v = p / n^2 (|v| = c0 / n with c0 = 1) instead. */
        double s[6] = {X[0], X[1], X[2], p[0], p[1], p[2]};
        if (sc->integrator == 2) {
            double n, gn[3];
            or_medium(sc, X[0], X[1], NULL, NULL, &n, gn, &cnt);
            for (int a = 0; a < 3; ++a) s[3 + a] = p[a] / (n * n);
        }
        double k1[6], k7[6];
        double h = sc->h;
        int have_k1 = 0;
        int left = 0;
        traj_push(tb, s);
        while (!left) {
            if (steps >= sc->max_steps) { status = ST_MAX_STEPS; break; }
            if (bounces > sc->max_bounces) { status = ST_MAX_BOUNCES; break; }
            double s1[6];
            double hs = h;
            if (sc->integrator != 1) {
                or_rk4(sc, s, hs, s1, &cnt);
                steps++;
            } else {
                if (!have_k1) { or_rhs(sc, s, k1, &cnt); have_k1 = 1; }
                int accepted = 0;
                while (!accepted) {
                    double y4[6];
                    hs = h;
                    or_dp45(sc, s, k1, hs, s1, y4, k7, &cnt);
                    steps++;
                    /* RMS error over (x, y, p_x, p_y); z and p_z carry no error */
                    const double scp = sc->atol + sc->rtol * sc->Lambda;
                    const int comp[4] = {0, 1, 3, 4};
                    double acc = 0.0;
                    for (int q = 0; q < 4; ++q) {
                        const int i = comp[q];
                        const double scale = (i < 3) ? scp
                            : sc->atol / sc->Lambda + sc->rtol * fmax(fabs(s[i]), fabs(s1[i]));
                        const double e = (s1[i] - y4[i]) / scale;
                        acc += e * e;
                    }
                    const double err = sqrt(acc / 4.0);
                    double fac = (err > 0.0) ? 0.9 * pow(err, -0.2) : 5.0;
                    fac = fmin(5.0, fmax(0.2, fac));
                    if (err <= 1.0) {
                        h = fmin(hs * fac, sc->h_max);
                        accepted = 1;
                    } else {
                        h = fmin(hs * fmin(fac, 1.0), sc->h_max);
                        if (steps >= sc->max_steps || !or_finite6(s1)) break;
                    }
                }
                if (!accepted) { status = or_finite6(s1) ? ST_MAX_STEPS : ST_NAN; break; }
            }
            if (!or_finite6(s1)) { status = ST_NAN; break; }

            /* events at the end of the step */
            int ev_best = EV_NONE;
            double th_best = 2.0;
            step_ctx ctx;
            ctx.sc = sc; memcpy(ctx.s, s, sizeof ctx.s); ctx.h = hs; ctx.cnt = &cnt;
            if (sc->integrator == 1) memcpy(ctx.k1, k1, sizeof ctx.k1);
            for (int ev = 0; ev < EV_COUNT; ++ev) {
                const double g1 = or_event_g(sc, ev, s1, &cnt);
                if (g1 < 0.0) {
                    const double th = or_locate_event(&ctx, ev, surface == ev, g1);
                    if (th < th_best) { th_best = th; ev_best = ev; }
                }
            }
            if (ev_best == EV_NONE) {
                memcpy(s, s1, sizeof s);
                if (sc->integrator == 1) memcpy(k1, k7, sizeof k1);   /* first same as last */
                surface = EV_NONE;
                traj_push(tb, s);
                continue;
            }
            events++;
            or_partial_step(&ctx, th_best, s1);
            memcpy(s, s1, sizeof s);
            have_k1 = 0;
            traj_push(tb, s);
            if (ev_best == EV_GRATING) {
                double N[3];
                or_surface_normal(sc, s[0], N);
                const double pn = s[3] * N[0] + s[4] * N[1] + s[5] * N[2];
                for (int a = 0; a < 3; ++a) s[3 + a] -= 2.0 * pn * N[a];
                bounces++;
                surface = EV_GRATING;
                traj_push(tb, s);
                continue;
            }
            /* a face of the box: refract into air or reflect totally, acting
               on the momentum (p = n^2 v in the time form) */
            double Nf[3];
            or_face_normal(ev_best, Nf);
            double pm[3] = {s[3], s[4], s[5]};
            double n2f = 1.0;
            if (sc->integrator == 2) {
                double nf, gn[3];
                or_medium(sc, s[0], s[1], NULL, NULL, &nf, gn, &cnt);
                n2f = nf * nf;
                for (int a = 0; a < 3; ++a) pm[a] *= n2f;
            }
            const double pn = pm[0] * Nf[0] + pm[1] * Nf[1] + pm[2] * Nf[2];
            double pt[3];
            for (int a = 0; a < 3; ++a) pt[a] = pm[a] - pn * Nf[a];
            const double pt2 = or_dot(pt, pt);
            if (pt2 >= 1.0) {
                for (int a = 0; a < 3; ++a) s[3 + a] -= 2.0 * (pn / n2f) * Nf[a];
                bounces++;
                surface = ev_best;
                traj_push(tb, s);
                continue;
            }
            const double pn_out = sqrt(1.0 - pt2);
            if (fresnel) {
                const double n1 = sqrt(or_dot(pm, pm));                          /* |p| = n */
                const double R = or_fresnel_R(n1, 1.0, pn, pn_out);
                double pr[3];
                for (int a = 0; a < 3; ++a) pr[a] = pm[a] - 2.0 * pn * Nf[a];
                or_push_branch(br, nbr, s, pr, w * R, MED_BOX, ev_best, bounces, events, steps);
                w *= 1.0 - R;
            }
            for (int a = 0; a < 3; ++a) { X[a] = s[a]; p[a] = pt[a] + pn_out * Nf[a]; }
            medium = MED_AIR;
            surface = EV_NONE;
            left = 1;
        }
        if (!left) {
            for (int a = 0; a < 3; ++a) { X[a] = s[a]; p[a] = s[3 + a]; }
            break;
        }
    }

    /* exit record: the start of the final straight segment (the last
       reflection or cloak-exit point; the camera for rays that meet nothing)
       and its unit direction */
    if (status != ST_OK && status != ST_SKY) { rgb[0] = rgb[1] = rgb[2] = 0.0; }
    double pos[3] = {X[0], X[1], X[2]};
    double pl = sqrt(or_dot(p, p));
    double dir[3] = {p[0] / pl, p[1] / pl, p[2] / pl};
    if (rec) {
        memcpy(rec->pos, pos, sizeof pos);
        memcpy(rec->dir, dir, sizeof dir);
        memcpy(rec->rgb, rgb, sizeof rgb);
        rec->steps = steps;
        rec->halley = cnt.halley;
        rec->evals = cnt.evals;
        rec->bounces = bounces;
        rec->status = status;
        rec->events = events;
        rec->pad = 0;
    }
    if (w_out) *w_out = w;
}

/* One camera sample: the path from (X0, p0) and, with Fresnel weights, the
   branches it started, traced in the order they were started.  The record is
   the first path's; its colour is the weighted sum over the paths. */
static void or_trace(const or_scene* sc, const camera* cam, const double X0[3], const double p0[3],
                     int medium, int surface, or_record* rec, traj_buf* tb)
{
    or_record local;
    if (!rec) rec = &local;
    if (!(sc->flags & OR_FLAG_FRESNEL)) {
        or_trace_path(sc, cam, X0, p0, medium, surface, 1.0, 0, 0, 0, NULL, NULL, rec, NULL, tb);
        return;
    }
    or_branch br[OR_MAX_BRANCHES];
    int nbr = 0;
    double w = 0.0;
    or_trace_path(sc, cam, X0, p0, medium, surface, 1.0, 0, 0, 0, br, &nbr, rec, &w, tb);
    double acc[3] = {w * rec->rgb[0], w * rec->rgb[1], w * rec->rgb[2]};
    for (int q = 0; q < nbr; ++q) {
        or_record r;
        double wq = 0.0;
        or_trace_path(sc, cam, br[q].X, br[q].p, br[q].medium, br[q].surface, br[q].w, br[q].bounces,
                      br[q].events, br[q].steps, NULL, NULL, &r, &wq, NULL);
        for (int a = 0; a < 3; ++a) acc[a] += wq * r.rgb[a];
    }
    for (int a = 0; a < 3; ++a) rec->rgb[a] = acc[a];
}

/* ------------------------------------------------------------------------ */
/* Exported entry points (ctypes).                                           */
/* ------------------------------------------------------------------------ */

int or_lambertw0(const double* z, int64_t count, double* w, int32_t* iters)
{
    for (int64_t i = 0; i < count; ++i) {
        int it;
        double complex r = or_w0_c(z[2 * i] + I * z[2 * i + 1], &it);
        w[2 * i] = creal(r);
        w[2 * i + 1] = cimag(r);
        if (iters) iters[i] = it;
    }
    return 0;
}

/* Per point: out[6*i..] = (Re W, Im W, n, dn/dx, dn/dy, dn/dz), W = W0 for
   the grating and the virtual coordinate w for the Gaussian cloak. */
int or_index(const or_scene* sc, const double* xy, int64_t count, double* out)
{
    for (int64_t i = 0; i < count; ++i) {
        double complex W;
        double n, gn[3];
        or_medium(sc, xy[2 * i], xy[2 * i + 1], &W, NULL, &n, gn, NULL);
        if (sc->mirror != 2) {
            int it;
            W = or_w0_c(or_zeta(sc, xy[2 * i], xy[2 * i + 1]), &it);
        }
        out[6 * i + 0] = creal(W); out[6 * i + 1] = cimag(W); out[6 * i + 2] = n;
        out[6 * i + 3] = gn[0]; out[6 * i + 4] = gn[1]; out[6 * i + 5] = gn[2];
    }
    return 0;
}

/* Trochoid helpers: xi(x), y_s(x), and the upward normal (Eq. 2). */
int or_trochoid(const or_scene* sc, const double* x, int64_t count, double* out)
{
    for (int64_t i = 0; i < count; ++i) {
        double N[3];
        out[4 * i + 0] = or_trochoid_xi(sc, x[i]);
        out[4 * i + 1] = or_trochoid_y(sc, x[i]);
        or_trochoid_normal(sc, x[i], N);
        out[4 * i + 2] = N[0]; out[4 * i + 3] = N[1];
    }
    return 0;
}

/* Faddeeva function at the points s (pairs Re, Im): out gets (Re F, Im F). */
int or_faddeeva_eval(const double* s, int64_t count, double* out)
{
    for (int64_t i = 0; i < count; ++i) {
        const double complex F = or_faddeeva(s[2 * i] + I * s[2 * i + 1]);
        out[2 * i] = creal(F);
        out[2 * i + 1] = cimag(F);
    }
    return 0;
}

/* Gaussian conformal map at virtual points w (pairs): out gets
   (Re z, Im z, Re z', Im z') per point. */
int or_gauss_map(const or_scene* sc, const double* w, int64_t count, double* out)
{
    for (int64_t i = 0; i < count; ++i) {
        double complex z, dz;
        or_gauss_z(sc, w[2 * i] + I * w[2 * i + 1], &z, &dz, NULL);
        out[4 * i + 0] = creal(z); out[4 * i + 1] = cimag(z);
        out[4 * i + 2] = creal(dz); out[4 * i + 3] = cimag(dz);
    }
    return 0;
}

/* Mirror surface (trochoid or bump) at abscissae x: (y_s, slope, N_x, N_y). */
int or_surface(const or_scene* sc, const double* x, int64_t count, double* out)
{
    for (int64_t i = 0; i < count; ++i) {
        double N[3];
        out[4 * i + 0] = or_surface_y(sc, x[i]);
        out[4 * i + 1] = or_surface_slope(sc, x[i]);
        or_surface_normal(sc, x[i], N);
        out[4 * i + 2] = N[0]; out[4 * i + 3] = N[1];
    }
    return 0;
}

/* First hit of the line X + t p with the mirror surface (tests). */
double or_surface_line_hit(const or_scene* sc, const double* X, const double* p, int32_t on_surface)
{
    return sc->mirror ? or_trochoid_line_hit(sc, X, p, on_surface) : or_flat_line_hit(X, p);
}

/* Fixed-step integration without events.  method 0: RK4, 1: fifth-order
   Dormand-Prince solution, 2: its embedded fourth-order solution.  Writes the
   state after every step (nsteps x 6). */
int or_integrate_fixed(const or_scene* sc, const double* s0, double h, int64_t nsteps, int32_t method, double* out)
{
    double s[6];
    memcpy(s, s0, sizeof s);
    for (int64_t n = 0; n < nsteps; ++n) {
        double s1[6];
        if (method == 0) {
            or_rk4(sc, s, h, s1, NULL);
        } else {
            double k1[6], y4[6], k7[6];
            or_rhs(sc, s, k1, NULL);
            or_dp45(sc, s, k1, h, s1, y4, k7, NULL);
            if (method == 2) memcpy(s1, y4, sizeof s1);
        }
        memcpy(s, s1, sizeof s);
        memcpy(out + 6 * n, s, sizeof s);
    }
    return 0;
}

/* Camera ray direction of sample s of pixel (i, j). */
int or_camera_dir(const or_scene* sc, int32_t i, int32_t j, int32_t s, double* origin, double* dir)
{
    camera cam;
    or_camera(sc, &cam);
    or_camera_ray(sc, &cam, i, j, s, dir);
    memcpy(origin, cam.C, sizeof cam.C);
    return 0;
}

uint64_t or_splitmix64_out(uint64_t seed, uint64_t m) { return or_splitmix64(seed, m); }

/* Trace one ray from an arbitrary state (tests).  medium 0: air, 1: inside the box. */
/* A texture background needs its texture. */
static int or_scene_ok(const or_scene* sc)
{
    if (sc->background == 1 && (!sc->tex || sc->tex_size <= 0)) return 0;
    if ((sc->flags & OR_FLAG_PLATE) && (sc->cloak || sc->mirror)) return 0;   /* the plate lies on the flat mirror */
    if (sc->mirror < 0 || sc->mirror > 2) return 0;
    if (sc->mirror == 2) {      /* the Gaussian map is one-to-one while h/w_b < sqrt(pi)/2 */
        if (!(sc->gauss_w > 0.0) || !(sc->A >= 0.0) || !(sc->A < 0.8 * sc->gauss_w)) return 0;
        if (sc->flags != 0) return 0;
    }
    return 1;
}

/* Unpolarised Fresnel reflectance from index n1 into index n2 at incidence
   cosine cos_i; 1 beyond the critical angle. */
double or_fresnel(double n1, double n2, double cos_i)
{
    const double sin2 = 1.0 - cos_i * cos_i;
    const double c2 = n2 * n2 - n1 * n1 * sin2;
    if (c2 <= 0.0) return 1.0;
    return or_fresnel_R(n1, n2, n1 * cos_i, sqrt(c2));
}

/* Every path of one sample started at (X, p): the first path's record and
   weight, then each Fresnel branch's, in the order they were started (at most
   cap records).  Returns the number of paths in *n. */
int or_trace_paths(const or_scene* sc, const double* X, const double* p, int32_t medium, int32_t surface,
                   or_record* recs, double* weights, int32_t cap, int32_t* n)
{
    if (!or_scene_ok(sc) || cap < 1) return -1;
    camera cam;
    or_camera(sc, &cam);
    or_branch br[OR_MAX_BRANCHES];
    int nbr = 0;
    or_trace_path(sc, &cam, X, p, medium, surface, 1.0, 0, 0, 0,
                  (sc->flags & OR_FLAG_FRESNEL) ? br : NULL, &nbr, &recs[0], &weights[0], NULL);
    int k = 1;
    for (int q = 0; q < nbr && k < cap; ++q, ++k)
        or_trace_path(sc, &cam, br[q].X, br[q].p, br[q].medium, br[q].surface, br[q].w, br[q].bounces,
                      br[q].events, br[q].steps, NULL, NULL, &recs[k], &weights[k], NULL);
    *n = k;
    return 0;
}

int or_trace_from(const or_scene* sc, const double* X, const double* p, int32_t medium, int32_t surface,
                  or_record* rec, double* traj, int32_t traj_cap, int32_t* traj_len)
{
    if (!or_scene_ok(sc)) return -1;
    camera cam;
    or_camera(sc, &cam);
    traj_buf tb = {traj, traj_cap, 0};
    or_trace(sc, &cam, X, p, medium, surface, rec, traj ? &tb : NULL);
    if (traj_len) *traj_len = tb.len;
    return 0;
}

/* Render the listed pixels (flat indices i * width_out + j).  rgb: npix x 3;
   rec (nullable): npix x spp records in sample order. */
int or_render_pixels(const or_scene* sc, const int64_t* pix, int64_t npix, float* rgb, or_record* rec,
                     int32_t nthreads)
{
    if (!or_scene_ok(sc)) return -1;
    camera cam;
    or_camera(sc, &cam);
    const int wout = sc->centre_line ? 1 : sc->width;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < npix; ++q) {
        const int i = (int)(pix[q] / wout), j = (int)(pix[q] % wout);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int s = 0; s < sc->spp; ++s) {
            double d[3];
            or_camera_ray(sc, &cam, i, j, s, d);
            or_record r;
            or_trace(sc, &cam, cam.C, d, MED_AIR, EV_NONE, &r, NULL);
            for (int a = 0; a < 3; ++a) acc[a] += r.rgb[a];
            if (rec) rec[q * sc->spp + s] = r;
        }
        for (int a = 0; a < 3; ++a) rgb[3 * q + a] = (float)(acc[a] / sc->spp);
    }
    return 0;
}

/* Full image: rgb is height x width_out x 3. */
int or_render(const or_scene* sc, float* rgb, or_record* rec, int32_t nthreads)
{
    const int wout = sc->centre_line ? 1 : sc->width;
    const int64_t npix = (int64_t)sc->height * wout;
    int64_t* pix = (int64_t*)malloc(sizeof(int64_t) * (size_t)npix);
    if (!pix) return -1;
    for (int64_t q = 0; q < npix; ++q) pix[q] = q;
    int rc = or_render_pixels(sc, pix, npix, rgb, rec, nthreads);
    free(pix);
    return rc;
}

/* 8-bit quantisation q = floor(clamp(c, 0, 1) * 255 + 1/2). */
int or_quantize(const float* c, int64_t count, uint8_t* q)
{
    for (int64_t i = 0; i < count; ++i) {
        double v = c[i];
        if (!(v > 0.0)) v = 0.0;
        if (v > 1.0) v = 1.0;
        q[i] = (uint8_t)floor(v * 255.0 + 0.5);
    }
    return 0;
}

/* Image cross-correlation C(0,0) of Eqs. 14-15 over the columns j0..j1-1 of
   H x W x C images f (reference) and g.  out[c] for each channel, out[C] for
   the channels taken together as one stacked image. */
int or_xcorr(const float* f, const float* g, int32_t H, int32_t W, int32_t C, int32_t j0, int32_t j1, double* out)
{
    double num_all = 0.0, den_all = 0.0;
    for (int c = 0; c < C; ++c) {
        double sf = 0.0, sg = 0.0;
        int64_t cnt = 0;
        for (int i = 0; i < H; ++i)
            for (int j = j0; j < j1; ++j) {
                sf += f[((int64_t)i * W + j) * C + c];
                sg += g[((int64_t)i * W + j) * C + c];
                cnt++;
            }
        const double mf = sf / (double)cnt, mg = sg / (double)cnt;   /* Eq. 14 */
        double num = 0.0, den = 0.0;
        for (int i = 0; i < H; ++i)
            for (int j = j0; j < j1; ++j) {
                const double a = f[((int64_t)i * W + j) * C + c] - mf;
                const double b = g[((int64_t)i * W + j) * C + c] - mg;
                num += a * b;                                        /* Eq. 15 numerator   */
                den += a * a;                                        /* Eq. 15 denominator */
            }
        out[c] = num / den;
        num_all += num;
        den_all += den;
    }
    out[C] = num_all / den_all;
    return 0;
}

/* The cross-correlation function C(di, dj) of Eq. 15 for pixel shifts
   |di| <= max_di (rows), |dj| <= max_dj (columns), over the columns j0..j1-1
   of both images (the finite-size photographs):
     f' = f - <f>, g' = g - <g> over that window (Eq. 14);
     C_c(di, dj) = sum f'(i, j) g'(i + di, j + dj) / sum f'(i, j)^2,
   the numerator over the pixels where both lie in the window (the images have
   no values outside it), the denominator over the whole window.  Per channel
   and for the stacked channels (sum of numerators over sum of denominators).
   out[((di + max_di) * (2 max_dj + 1) + (dj + max_dj)) * (C + 1) + c]. */
int or_xcorr_map(const float* f, const float* g, int32_t H, int32_t W, int32_t C, int32_t j0, int32_t j1,
                 int32_t max_di, int32_t max_dj, double* out)
{
    const int ndj = 2 * max_dj + 1;
    double* mf = (double*)calloc((size_t)C, sizeof(double));
    double* mg = (double*)calloc((size_t)C, sizeof(double));
    double* den = (double*)calloc((size_t)C, sizeof(double));
    if (!mf || !mg || !den) { free(mf); free(mg); free(den); return -1; }
    const double cnt = (double)H * (double)(j1 - j0);
    for (int c = 0; c < C; ++c) {
        double sf = 0.0, sg = 0.0;
        for (int i = 0; i < H; ++i)
            for (int j = j0; j < j1; ++j) {
                sf += f[((int64_t)i * W + j) * C + c];
                sg += g[((int64_t)i * W + j) * C + c];
            }
        mf[c] = sf / cnt;                                             /* Eq. 14 */
        mg[c] = sg / cnt;
        double d = 0.0;
        for (int i = 0; i < H; ++i)
            for (int j = j0; j < j1; ++j) {
                const double a = f[((int64_t)i * W + j) * C + c] - mf[c];
                d += a * a;                                           /* Eq. 15 denominator */
            }
        den[c] = d;
    }
    for (int di = -max_di; di <= max_di; ++di)
        for (int dj = -max_dj; dj <= max_dj; ++dj) {
            double* o = out + ((int64_t)(di + max_di) * ndj + (dj + max_dj)) * (C + 1);
            double num_all = 0.0, den_all = 0.0;
            for (int c = 0; c < C; ++c) {
                double num = 0.0;
                for (int i = 0; i < H; ++i) {
                    const int ig = i + di;
                    if (ig < 0 || ig >= H) continue;
                    for (int j = j0; j < j1; ++j) {
                        const int jg = j + dj;
                        if (jg < j0 || jg >= j1) continue;
                        const double a = f[((int64_t)i * W + j) * C + c] - mf[c];
                        const double b = g[((int64_t)ig * W + jg) * C + c] - mg[c];
                        num += a * b;                                 /* Eq. 15 numerator */
                    }
                }
                o[c] = num / den[c];
                num_all += num;
                den_all += den[c];
            }
            o[C] = num_all / den_all;
        }
    free(mf);
    free(mg);
    free(den);
    return 0;
}

/* Columns of a width-W image whose pixel-centre horizontal angle lies within
   the horizontal field of view fov (degrees) about the image centre. */
int or_fov_columns(int32_t W, double hfov_deg, double fov_deg, int32_t* j0, int32_t* j1)
{
    const double tx = tan(0.5 * hfov_deg * OR_PI / 180.0);
    int lo = W, hi = -1;
    for (int j = 0; j < W; ++j) {
        const double px = 2.0 * (j + 0.5) / W - 1.0;
        const double alpha = atan(fabs(px) * tx) * 180.0 / OR_PI;
        if (alpha <= 0.5 * fov_deg + 1e-9) {
            if (j < lo) lo = j;
            if (j > hi) hi = j;
        }
    }
    if (hi < lo) { *j0 = 0; *j1 = 0; return 0; }
    *j0 = lo; *j1 = hi + 1;
    return 0;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
