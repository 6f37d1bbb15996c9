/*
 * rh_oracle.c -- plain, slow FP64 CPU oracle of the column-by-column (1.5D)
 * MALI hot path.  TEST INFRASTRUCTURE ONLY: it is called by the test-suite,
 * by the package's smoke check and by the benchmark's CPU-baseline leg, never
 * by the product path.  It shares no code, header or table with the CUDA path.
 *
 * What it follows (the paper prints no equation of the method, so every
 * formula below is the standard form of the method the paper cites):
 *   - Sect. 2.1: MALI with a local (diagonal) approximate Psi operator and
 *     preconditioned rate equations (Rybicki & Hummer 1992), overlapping
 *     transitions sharing chi and eta at a wavelength.
 *   - Sect. 2.2: each column is an independent plane-parallel problem; only the
 *     vertical emergent spectrum is produced.
 *   - Sect. 2.3: Ng acceleration (order 2), LTE start solution, per-column
 *     convergence on the maximum relative population change (1e-3).
 *   - Sect. 3.1 (pool mode): columns are handed out dynamically to workers
 *     (here: threads pulling column indices from a shared counter).
 * Readings where the paper is silent, each restated at the function that
 * uses it: linear short characteristics (Olson & Kunasz 1987) as the formal
 * solver; no incident radiation at the top and the diffusion approximation
 * I = B + mu dB/dtau at the bottom; a hydrogen-like model atom (Kramers
 * f-values and bound-free cross sections, van Regemorter and Seaton
 * collisions); LTE H- bound-free, hydrogenic free-free and Thomson background;
 * n_e fixed from Saha plus a metal floor; Ng of order 2 with uniform weights,
 * delay 5, period 3; collisional-radiative switching by a decade per
 * iteration; PRD switching eps = min(1, eps0 it^2); Ng and a Jacobi step on
 * the PRD ratio rho; for the hybrid PRD option (Sect. 2.1), the gas-frame
 * mean intensity and ratio transferred between frames by linear
 * interpolation in frequency over the line's points, constant beyond them;
 * for the higher-order formal-solver option, quadratic Bezier short
 * characteristics with a Fritsch-Butland control point held between its
 * neighbours.
 *
 * Parity status: every function is pinned by a test against closed forms,
 * limits or an independent library routine, except the overall multi-level
 * emergent intensities of the synthetic chromosphere, which have no printed
 * values ("parity unpinned" beyond oracle self-consistency, Newton residual
 * and limit checks).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

/* ---- physical constants, SI (CODATA 2018; h, c, k, e exact) ---- */
#define HPLANCK 6.62607015e-34
#define CLIGHT 2.99792458e8
#define KBOLTZ 1.380649e-23
#define QELEC 1.602176634e-19
#define MELEC 9.1093837015e-31
#define EPS0 8.8541878128e-12
#define AMU 1.66053906660e-27
#define SIGMA_T 6.6524587321e-29
#define E_RYDBERG (13.605693122994 * QELEC)
#define PI_D 3.14159265358979323846

#define MAXLEV 16
#define MAXTR 64
#define MAXACT 8

/* ------------------------------------------------------------------ */
/* public descriptor (same field order as the CUDA library's, declared  */
/* separately on purpose)                                               */
typedef struct {
    int32_t nlev;
    const double *E_J, *g;
    int32_t nline;
    const int32_t *line_l, *line_u;
    const double *line_f, *line_a_top, *line_a_bot;
    const int32_t *line_nlambda;
    const double *line_qwing;
    int32_t ncont;
    const int32_t *cont_l;
    const double *cont_alpha0;
    const int32_t *cont_nlambda;
    const double *cont_ratio;
    double mass_amu, T_ref;
    int32_t nmu;
    double metal_floor;
    const int32_t *line_prd;   /* per line: 1 angle-averaged partial redistribution (NULL: none) */
} rho_atom_desc;

typedef struct {
    int32_t maxiter;
    double tol;
    int32_t ng_order, ng_delay, ng_period;
    int32_t start;      /* 0 LTE, 2 user populations, 3 zero radiation, 4 escape probability */
    double crsw_init;   /* collisional-radiative switching start factor; <=1 off */
    double prd_eps0;    /* PRD switching (Eq. 1): eps = min(1, eps0 it^2); <= 0: off (eps = 1) */
    int32_t prd_hybrid; /* 0: angle-averaged in the static frame; 1: the hybrid approximation of
                         * angle-dependent PRD in moving atmospheres (Sect. 2.1) */
    int32_t formal;     /* formal solver: 0 linear short characteristics, 1 quadratic Bezier */
} rho_iter_opts;

typedef struct {
    int64_t n_converged, n_maxiter, n_failed;
    int64_t iterations_total;
    double seconds, pts, max_dn_final;
} rho_iter_stats;

enum { ST_CONV = 0, ST_MAXITER = 1, ST_NONFINITE = 2, ST_SINGULAR = 3, ST_NOTRUN = 4 };

/* ------------------------------------------------------------------ */
typedef struct {
    int nlev, nline, ncont, ntr, nmu;
    double E[MAXLEV], g[MAXLEV];
    /* transitions: t < nline lines, then continua; upper of a continuum = nlev-1 */
    int tl[MAXTR], tu[MAXTR], kind[MAXTR];
    double nu0[MAXTR];            /* line centre or edge frequency */
    double f[MAXTR], A[MAXTR], Blu[MAXTR], Bul[MAXTR];
    double a_top[MAXTR], a_bot[MAXTR], qwing[MAXTR];
    double alpha0[MAXTR], ratio[MAXTR];
    int nlam_t[MAXTR];
    double nu_lo[MAXTR], nu_hi[MAXTR];
    double mass, T_ref, floor_e;
    double mu[16], wmu[16];
    /* wavelength grid */
    int64_t nlam;
    double *nu;                   /* [nlam] */
    int *nact;                    /* [nlam] */
    int *act;                     /* [nlam][MAXACT] transition index */
    double *wq;                   /* [nlam][MAXACT] quadrature weight (Hz) of that transition */
    int *prof_slot;               /* [nlam][MAXACT] line-profile block index, -1 for continua */
    int nprof;                    /* number of (lambda, line) pairs */
    /* partial redistribution: per PRD line its grid points in frequency order */
    int prd[MAXTR];
    int nprd_line, prd_t[MAXTR], prd_np[MAXTR];
    int *prd_pts[MAXTR];          /* grid indices */
    double *prd_w[MAXTR];         /* the line's quadrature weight at each point (Hz) */
} atom_t;

struct rho_ctx {
    char err[512];
    int have_atom;
    atom_t at;
    int64_t ncol;
    int ndep;
    double *z, *T, *nH, *vz, *ne, *np;   /* [ncol][ndep] */
    double *nstar;                        /* [ncol][nlev][ndep] */
    double *pops;                         /* [ncol][nlev][ndep] */
    int32_t *iters;
    uint8_t *status;
    double *dmax;
    /* [ncol] per column the PRD kernels K and J-bar weights f of every PRD
     * line, line after line ([N][np][np] then [N][np]); built by the first
     * column_setup of the column and reused (they depend only on the atom
     * and the column's temperatures) */
    double **prdc;
};
typedef struct rho_ctx rho_ctx;

static int fail(rho_ctx *c, const char *msg)
{
    snprintf(c->err, sizeof c->err, "%s", msg);
    return 1;
}

/* ================================================================== */
/* Special functions                                                   */
/* ================================================================== */

/* Voigt function H(a,v) = Re w(v + i a) = (a/pi) int exp(-u^2) / (a^2 + (u-v)^2) du.
 *  |v| >= 8: Laplace continued fraction of the Faddeeva function
 *     w(z) = (i/sqrt(pi)) / (z - (1/2)/(z - 1/(z - (3/2)/(z - ...)))),
 *     60 levels (converged to ~1e-15 there);
 *  |v| <  8: the convolution integral itself, split at |u - v| = D = 1/2:
 *     near part, with g(s) = exp(-(v+s)^2):
 *        (a/pi) int_{-D}^{D} g(s)/(a^2+s^2) ds
 *          = g(0) (2/pi) atan(D/a) + (a/pi) int_0^D [g(s)+g(-s)-2g(0)]/(a^2+s^2) ds,
 *        the last integral on 24 geometrically shrinking panels towards s = 0
 *        (10-point Gauss-Legendre each), so the Lorentz core of width a is
 *        resolved;
 *     far part, |u - v| > D, u in [-9, 9] (exp(-81) is negligible): panels
 *        of width <= 1/2, 10-point Gauss-Legendre each.
 *  Every integrand is smooth on its panels and (up to the symmetric second
 *  difference) positive.  Pinned against scipy.special.wofz to 1e-13. */
static double gl10_x[10], gl10_w[10];
static pthread_once_t gl10_once = PTHREAD_ONCE_INIT;
static void gauss_legendre01(int n, double *x, double *w);
static void gl10_init(void) { gauss_legendre01(10, gl10_x, gl10_w); }

static double voigt_far(double a, double v, double lo, double hi)
{
    if (!(hi > lo)) return 0.0;
    int np = (int)ceil((hi - lo) / 0.5);
    double h = (hi - lo) / np, s = 0.0;
    for (int p = 0; p < np; ++p)
        for (int i = 0; i < 10; ++i) {
            double u = lo + h * (p + gl10_x[i]);
            double d = u - v;
            s += gl10_w[i] * h * exp(-u * u) / (a * a + d * d);
        }
    return s;
}

double rho_voigt(double a, double v)
{
    double av = fabs(v);
    if (av >= 8.0) {
        /* continued fraction with complex z = av + i a, evaluated from the tail */
        double fr = av, fi = a;
        for (int k = 60; k >= 1; --k) {
            double d = fr * fr + fi * fi;
            /* f = z - (k/2) / f */
            double qr = 0.5 * k * fr / d, qi = -0.5 * k * fi / d;
            fr = av - qr;
            fi = a - qi;
        }
        /* w = (i/sqrt(pi)) / f ; Re w = Im(f) / (sqrt(pi) |f|^2) */
        return fi / (sqrt(PI_D) * (fr * fr + fi * fi));
    }
    pthread_once(&gl10_once, gl10_init);
    const double D = 0.5;
    double g0 = exp(-av * av);
    double near = g0 * (2.0 / PI_D) * atan(D / a);
    double corr = 0.0;
    for (int j = 0; j < 24; ++j) {
        double hi = D * ldexp(1.0, -j), lo = j == 23 ? 0.0 : 0.5 * hi;
        double h = hi - lo;
        for (int i = 0; i < 10; ++i) {
            double sv = lo + h * gl10_x[i];
            double gp = exp(-(av + sv) * (av + sv)), gm = exp(-(av - sv) * (av - sv));
            corr += gl10_w[i] * h * (gp + gm - 2.0 * g0) / (a * a + sv * sv);
        }
    }
    near += a / PI_D * corr;
    double far = a / PI_D * (voigt_far(a, av, -9.0, av - D) + voigt_far(a, av, av + D, 9.0));
    return near + far;
}

/* Faddeeva function w(v + i a) = H(a,v) + i L(a,v), a > 0: H as rho_voigt;
 * the dispersion part L(a,v) = (1/pi) int exp(-u^2) (v - u)/((v-u)^2 + a^2) du
 *  |v| >= 8: from the same continued fraction (Im w = Re f/(sqrt(pi)|f|^2));
 *  |v| <  8: the convolution integral, split at |u - v| = D = 1/2: near part
 *     with s = u - v the kernel is odd, (1/pi) int_0^D [g(-s) - g(s)] s/(s^2+a^2) ds,
 *     g(s) = exp(-(v+s)^2), on 24 geometrically shrinking panels towards s = 0
 *     (10-point Gauss-Legendre); far part |u - v| > D, u in [-9, 9], panels of
 *     width <= 1/2.  L is odd in v.  Pinned against scipy.special.wofz. */
static double disp_far(double a, double v, double lo, double hi)
{
    if (!(hi > lo)) return 0.0;
    int np = (int)ceil((hi - lo) / 0.5);
    double h = (hi - lo) / np, s = 0.0;
    for (int p = 0; p < np; ++p)
        for (int i = 0; i < 10; ++i) {
            double u = lo + h * (p + gl10_x[i]);
            double d = v - u;
            s += gl10_w[i] * h * exp(-u * u) * d / (a * a + d * d);
        }
    return s;
}

void rho_faddeeva(double a, double v, double *H, double *L)
{
    double av = fabs(v), sg = v < 0 ? -1.0 : 1.0;
    if (av >= 8.0) {
        double fr = av, fi = a;
        for (int k = 60; k >= 1; --k) {
            double d = fr * fr + fi * fi;
            double qr = 0.5 * k * fr / d, qi = -0.5 * k * fi / d;
            fr = av - qr;
            fi = a - qi;
        }
        double m = sqrt(PI_D) * (fr * fr + fi * fi);
        *H = fi / m;
        *L = sg * fr / m;
        return;
    }
    *H = rho_voigt(a, v);
    pthread_once(&gl10_once, gl10_init);
    const double D = 0.5;
    double near = 0.0;
    for (int j = 0; j < 24; ++j) {
        double hi = D * ldexp(1.0, -j), lo = j == 23 ? 0.0 : 0.5 * hi;
        double h = hi - lo;
        for (int i = 0; i < 10; ++i) {
            double sv = lo + h * gl10_x[i];
            double gp = exp(-(av + sv) * (av + sv)), gm = exp(-(av - sv) * (av - sv));
            near += gl10_w[i] * h * (gm - gp) * sv / (a * a + sv * sv);
        }
    }
    double far = disp_far(a, av, -9.0, av - D) + disp_far(a, av, av + D, 9.0);
    *L = sg * (near + far) / PI_D;
}

/* Angle-averaged redistribution function R_II-A (Hummer 1962), in Doppler
 * units, normalised so that int R(x', x) dx' = H(a, x)/sqrt(pi):
 *   R(x', x) = pi^{-3/2} int_{(xb - xs)/2}^inf e^{-u^2}
 *                  [atan((xs + u)/a) - atan((xb - u)/a)] du,
 *   xs = min(x, x'), xb = max(x, x') (signed).
 * Adaptive Gauss-Kronrod (7/15 points) with the atan steps of width a at
 * u = xb and u = -xs as breakpoints and the range ended at max + 8 (e^{-64}),
 * to a tolerance relative to a first estimate of the integral.
 * Pinned: normalisation, symmetry, the a -> 0 limit (1/2) erfc(max(|x|, |x'|)). */
static const double gk_x[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                               0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                               0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                               0.207784955007898467600689403773245, 0.0};
static const double gk_wk[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                                0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                                0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                                0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double gk_wg[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                                0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

/* atan((xs+u)/a) - atan((xb-u)/a) = atan2(a (xs + 2u - xb), a^2 + (xs+u)(xb-u)):
 * no cancellation between two arctangents near pi/2 (xs + 2u - xb =
 * 2 (u - u0) >= 0 on the range; atan2 takes the branch where the denominator
 * turns negative) */
static double r2_integrand(double u, double xs, double xb, double a)
{
    return exp(-u * u) * atan2(a * (xs + 2.0 * u - xb), a * a + (xs + u) * (xb - u));
}

static double r2_gk(double lo, double hi, double xs, double xb, double a, double *err)
{
    double c = 0.5 * (lo + hi), h = 0.5 * (hi - lo);
    double fc = r2_integrand(c, xs, xb, a);
    double k = gk_wk[7] * fc, g = gk_wg[3] * fc;
    for (int j = 0; j < 7; ++j) {
        double f = r2_integrand(c - h * gk_x[j], xs, xb, a) + r2_integrand(c + h * gk_x[j], xs, xb, a);
        k += gk_wk[j] * f;
        if (j & 1) g += gk_wg[j / 2] * f;
    }
    *err = fabs(k - g) * h;
    return k * h;
}

static double r2_adapt(double lo, double hi, double xs, double xb, double a, double tol, int depth)
{
    double err, v = r2_gk(lo, hi, xs, xb, a, &err);
    /* stop at the tolerance, at the rounding level of the panel, or at depth 30 */
    if (depth >= 30 || err <= tol || err <= 1e-14 * fabs(v)) return v;
    double c = 0.5 * (lo + hi);
    return r2_adapt(lo, c, xs, xb, a, 0.5 * tol, depth + 1) + r2_adapt(c, hi, xs, xb, a, 0.5 * tol, depth + 1);
}

double rho_r2a(double a, double xp, double x)
{
    double xs = fmin(x, xp), xb = fmax(x, xp);
    double u0 = 0.5 * (xb - xs), top = fmax(u0, fmax(xb, -xs)) + 8.0;
    double br[4] = {u0, xb, -xs, top};
    int nb = 0;
    double pts[4];
    for (int i = 0; i < 4; ++i)
        if (br[i] >= u0 && br[i] <= top) pts[nb++] = br[i];
    for (int i = 1; i < nb; ++i)       /* sort the few breakpoints */
        for (int j = i; j > 0 && pts[j] < pts[j - 1]; --j) {
            double t = pts[j]; pts[j] = pts[j - 1]; pts[j - 1] = t;
        }
    double est = 0.0, e;
    for (int i = 0; i + 1 < nb; ++i) est += fabs(r2_gk(pts[i], pts[i + 1], xs, xb, a, &e));
    double tol = 1e-15 * est + 1e-300, s = 0.0;
    for (int i = 0; i + 1 < nb; ++i)
        if (pts[i + 1] > pts[i]) s += r2_adapt(pts[i], pts[i + 1], xs, xb, a, tol / (nb - 1), 0);
    return s / (PI_D * sqrt(PI_D));
}

/* e^y E1(y) for y > 0: power series for y <= 1, continued fraction
 * E1(y) = e^{-y} / (y + 1 - 1/(y + 3 - 4/(y + 5 - ...))) otherwise
 * (Abramowitz & Stegun 5.1.11 and 5.1.22).  Pinned against scipy.special.exp1. */
double rho_expE1(double y)
{
    if (y <= 1.0) {
        const double gam = 0.57721566490153286061;
        double s = 0.0, term = 1.0;
        for (int n = 1; n < 200; ++n) {
            term *= -y / n;
            double add = term / n;
            s += add;
            if (fabs(add) < 1e-18 * fabs(s) + 1e-300) break;
        }
        return exp(y) * (-gam - log(y) - s);
    }
    /* evaluate the continued fraction from the tail (fixed depth is ample for y > 1) */
    double f = 0.0;
    for (int n = 300; n >= 1; --n) f = (double)n * n / (y + 2.0 * n + 1.0 - f);
    return 1.0 / (y + 1.0 - f);
}

/* Planck function B_nu(T) [W m^-2 Hz^-1 sr^-1] */
double rho_planck(double nu, double T)
{
    double x = HPLANCK * nu / (KBOLTZ * T);
    return 2.0 * HPLANCK * nu * nu * nu / (CLIGHT * CLIGHT) / expm1(x);
}

/* Gauss-Legendre nodes and weights on (0,1), weights summing to 1 */
static void gauss_legendre01(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(PI_D * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute derivative at converged root */
        double p0 = 1.0, p1 = z;
        for (int j = 2; j <= n; ++j) {
            double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[n - 1 - i] = 0.5 * (z + 1.0);
        w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);   /* (2/((1-z^2)p'^2)) / 2 */
    }
}

int rho_gauss_legendre01(int n, double *x, double *w)
{
    if (n < 1 || n > 16) return 1;
    gauss_legendre01(n, x, w);
    return 0;
}

/* ================================================================== */
/* Formal solver: linear short characteristics (Olson & Kunasz 1987).    */
/* The paper (Sect. 2.1) names no scheme; this is the reading taken.     */
/* ================================================================== */

/* Weights of the linear short-characteristics step over optical path d:
 * e0 = 1 - exp(-d), e1 = d - e0, w_o = e1/d, w_u = e0 - w_o.  For d < 0.5
 * e1 comes from its power series; otherwise 1 - w_o = e0/d and
 * w_u = e0/d - exp(-d) are evaluated directly, because w_u ~ 1/d and
 * 1 - w_o ~ 1/d at large d would otherwise be differences of two numbers
 * close to one (relative error ~ 1e-16 d, and d reaches 1e8 in the Lyman
 * line cores). */
static void sc_step_weights(double d, double *ex, double *wu, double *wo, double *omwo)
{
    if (d < 0.5) {
        /* e1 = sum_{n>=2} (-d)^n / n!,  e0 = d - e1 */
        double term = -d, s = 0.0;
        for (int n = 2; n < 60; ++n) {
            term *= -d / n;
            s += term;
            if (fabs(term) < 1e-18 * fabs(s)) break;
        }
        double e0 = d - s;
        *wo = s / d;
        *wu = e0 - *wo;
        *omwo = 1.0 - *wo;
        *ex = 1.0 - e0;
    } else {
        double e0 = -expm1(-d);
        *ex = exp(-d);
        *omwo = e0 / d;
        *wo = 1.0 - *omwo;
        *wu = *omwo - *ex;
    }
}

/* One sweep along a ray.  dtau[k] is the optical path between points k and
 * k+1 along the ray (k = 0..N-2).  dir = +1 sweeps k = 0 -> N-1 (starting
 * value at k = 0), dir = -1 sweeps k = N-1 -> 0.  Output I[k] and the local
 * operator lam[k] = dI_k/dS_k (0 at the starting point).  Optional outputs
 * (NULL to skip): Ieff[k], the intensity at k with the local source S[k]
 * replaced by Sloc[k] (for the preconditioned rates, Sloc is the background
 * part of the source function, so Ieff = I - Psi* eta_active), and
 * omlam[k] = 1 - lam[k]. */
static void sc_sweep_full(int N, const double *dtau, const double *S, const double *Sloc, double I0, int dir,
                          double *I, double *lam, double *Ieff, double *omlam)
{
    int k0 = dir > 0 ? 0 : N - 1;
    I[k0] = I0;
    lam[k0] = 0.0;
    if (Ieff) Ieff[k0] = I0;
    if (omlam) omlam[k0] = 1.0;
    for (int s = 1; s < N; ++s) {
        int ko = dir > 0 ? s : N - 1 - s;
        int ku = ko - dir;
        double d = dtau[dir > 0 ? ku : ko];
        double ex, wu, wo, omwo;
        sc_step_weights(d, &ex, &wu, &wo, &omwo);
        double base = I[ku] * ex + wu * S[ku];
        I[ko] = base + wo * S[ko];
        lam[ko] = wo;
        if (Ieff) Ieff[ko] = base + wo * Sloc[ko];
        if (omlam) omlam[ko] = omwo;
    }
}

void rho_sc_sweep(int N, const double *dtau, const double *S, double I0, int dir, double *I, double *lam)
{
    sc_sweep_full(N, dtau, S, NULL, I0, dir, I, lam, NULL, NULL);
}

/* Quadratic Bezier short characteristics (the higher-order formal solver of
 * the option formal = 1; the paper names no scheme).  Between the upwind
 * point u and the point o the source function is the quadratic Bezier curve
 * S(t) = (1-t)^2 S_u + 2 t (1-t) C + t^2 S_o in t = tau'/d, so
 *   I_o = I_u e^{-d} + w_u S_u + w_o S_o + w_c C,
 *   w_u = int_0^1 s^2 e^{-d s} d ds = [2 - e^{-d} (d^2 + 2d + 2)] / d^2,
 *   w_o = int_0^1 (1-s)^2 e^{-d s} d ds = [d^2 - 2d + 2 - 2 e^{-d}] / d^2,
 *   w_c = 2 int_0^1 s (1-s) e^{-d s} d ds = [2d - 4 + (2d + 4) e^{-d}] / d^2
 * (w_u + w_o + w_c = 1 - e^{-d}).  The local operator is Psi* = w_o + w_c
 * (C follows S_o), and 1 - Psi* = 2 [1 - e^{-d} (1 + d)] / d^2 is formed
 * directly: at large d it is ~2/d^2 and 1 - (w_o + w_c) would cancel.  For
 * d < 1 every weight comes from its power series in d (the closed forms
 * cancel there). */
static void bez_step_weights(double d, double *ex, double *wu, double *wo, double *wc, double *omp)
{
    if (d < 1.0) {
        double t = 1.0, su = 0.0, so = 0.0, sc = 0.0, sp = 0.0;   /* t = (-d)^n / n! */
        for (int n = 0; n < 40; ++n) {
            if (n > 0) t *= -d / n;
            su += t / (n + 3.0);
            so += t * 2.0 / ((n + 1.0) * (n + 2.0) * (n + 3.0));
            sc += t * 2.0 / ((n + 2.0) * (n + 3.0));
            sp += t * 2.0 / (n + 2.0);
            if (fabs(t) < 1e-22) break;
        }
        *wu = d * su;
        *wo = d * so;
        *wc = d * sc;
        *omp = sp;
        *ex = exp(-d);
    } else {
        double e = exp(-d), d2 = d * d;
        *ex = e;
        *wu = (2.0 - e * (d2 + 2.0 * d + 2.0)) / d2;
        *wo = (d2 - 2.0 * d + 2.0 - 2.0 * e) / d2;
        *wc = (2.0 * d - 4.0 + (2.0 * d + 4.0) * e) / d2;
        *omp = 2.0 * (1.0 - e * (1.0 + d)) / d2;
    }
}

void rho_bez_weights(double d, double *out5)
{
    bez_step_weights(d, out5, out5 + 1, out5 + 2, out5 + 3, out5 + 4);
}

/* The Bezier control point of the step u -> o: C = S_o - (d_u / 2) S'_o, the
 * derivative at o the weighted harmonic mean of the two neighbouring slopes
 * (Fritsch & Butland 1984), 0 where they differ in sign, and C held between
 * S_u and S_o (no overshoot on the interval); without a downwind point the
 * midpoint, which makes the step the linear one. */
static double bez_control(double Su, double So, double Sd, double du, double dd, int has_d)
{
    if (!has_d) return 0.5 * (Su + So);
    double su = (So - Su) / du, sd = (Sd - So) / dd, der = 0.0;
    if (su * sd > 0.0) {
        double a = (1.0 + dd / (du + dd)) / 3.0;
        der = su * sd / (a * sd + (1.0 - a) * su);
    }
    double C = So - 0.5 * du * der;
    double lo = Su < So ? Su : So, hi = Su < So ? So : Su;
    return C < lo ? lo : (C > hi ? hi : C);
}

/* One sweep along a ray with the Bezier step (outputs as sc_sweep_full;
 * lam = Psi* = w_o + w_c, Ieff = I with the local S_o replaced by Sloc_o
 * through Psi*) */
static void sc_sweep_bezier(int N, const double *dtau, const double *S, const double *Sloc, double I0, int dir,
                            double *I, double *lam, double *Ieff, double *omlam)
{
    int k0 = dir > 0 ? 0 : N - 1;
    I[k0] = I0;
    lam[k0] = 0.0;
    if (Ieff) Ieff[k0] = I0;
    if (omlam) omlam[k0] = 1.0;
    for (int s = 1; s < N; ++s) {
        int ko = dir > 0 ? s : N - 1 - s;
        int ku = ko - dir, kd = ko + dir;
        int has_d = kd >= 0 && kd < N;
        double du = dtau[dir > 0 ? ku : ko];
        double dd = has_d ? dtau[dir > 0 ? ko : kd] : 0.0;
        double ex, wu, wo, wc, omp;
        bez_step_weights(du, &ex, &wu, &wo, &wc, &omp);
        double C = bez_control(S[ku], S[ko], has_d ? S[kd] : 0.0, du, dd, has_d);
        double base = I[ku] * ex + wu * S[ku] + wc * (C - S[ko]);
        I[ko] = base + (wo + wc) * S[ko];
        lam[ko] = wo + wc;
        if (Ieff) Ieff[ko] = base + (wo + wc) * Sloc[ko];
        if (omlam) omlam[ko] = omp;
    }
}

void rho_sc_sweep_bezier(int N, const double *dtau, const double *S, double I0, int dir, double *I, double *lam)
{
    sc_sweep_bezier(N, dtau, S, NULL, I0, dir, I, lam, NULL, NULL);
}

/* ================================================================== */
/* Atom and wavelength grid                                              */
/* ================================================================== */

static int cmp_dbl_idx(const void *a, const void *b)
{
    const double *x = a, *y = b;
    return (x[0] > y[0]) - (x[0] < y[0]);
}

static void atom_free(atom_t *a)
{
    for (int q = 0; q < a->nprd_line; ++q) {
        free(a->prd_pts[q]);
        free(a->prd_w[q]);
    }
    free(a->nu);
    free(a->nact);
    free(a->act);
    free(a->wq);
    free(a->prof_slot);
    memset(a, 0, sizeof *a);
}

static int atom_build(rho_ctx *c, const rho_atom_desc *d)
{
    atom_t *a = &c->at;
    if (d->nlev < 2 || d->nlev > MAXLEV) return fail(c, "nlev out of range");
    if (d->nline < 0 || d->ncont < 0 || d->nline + d->ncont > MAXTR || d->nline + d->ncont < 1)
        return fail(c, "number of transitions out of range");
    if (d->nmu < 1 || d->nmu > 16) return fail(c, "nmu out of range");
    if (!(d->mass_amu > 0) || !(d->T_ref > 0)) return fail(c, "mass_amu and T_ref must be positive");
    atom_free(a);
    a->nlev = d->nlev;
    a->nline = d->nline;
    a->ncont = d->ncont;
    a->ntr = d->nline + d->ncont;
    a->nmu = d->nmu;
    a->mass = d->mass_amu * AMU;
    a->T_ref = d->T_ref;
    a->floor_e = d->metal_floor;
    for (int i = 0; i < a->nlev; ++i) {
        a->E[i] = d->E_J[i];
        a->g[i] = d->g[i];
        if (!(a->g[i] > 0)) return fail(c, "statistical weights must be positive");
    }
    const int ic = a->nlev - 1;
    for (int t = 0; t < d->nline; ++t) {
        int l = d->line_l[t], u = d->line_u[t];
        if (l < 0 || u >= ic || l >= u) return fail(c, "line levels out of range");
        if (d->line_nlambda[t] < 2) return fail(c, "line_nlambda must be >= 2");
        a->tl[t] = l;
        a->tu[t] = u;
        a->kind[t] = 0;
        double nu0 = (a->E[u] - a->E[l]) / HPLANCK;
        a->nu0[t] = nu0;
        a->f[t] = d->line_f[t];
        /* Einstein coefficients from the oscillator strength (SI) */
        a->A[t] = 2.0 * PI_D * QELEC * QELEC * nu0 * nu0 / (EPS0 * MELEC * CLIGHT * CLIGHT * CLIGHT)
                  * (a->g[l] / a->g[u]) * a->f[t];
        a->Bul[t] = a->A[t] * CLIGHT * CLIGHT / (2.0 * HPLANCK * nu0 * nu0 * nu0);
        a->Blu[t] = a->Bul[t] * a->g[u] / a->g[l];
        a->a_top[t] = d->line_a_top[t];
        a->a_bot[t] = d->line_a_bot[t];
        a->qwing[t] = d->line_qwing[t];
        a->nlam_t[t] = d->line_nlambda[t];
        double dnu_ref = nu0 / CLIGHT * sqrt(2.0 * KBOLTZ * a->T_ref / a->mass);
        a->nu_lo[t] = nu0 - a->qwing[t] * dnu_ref;
        a->nu_hi[t] = nu0 + a->qwing[t] * dnu_ref;
    }
    for (int q = 0; q < d->ncont; ++q) {
        int t = d->nline + q, l = d->cont_l[q];
        if (l < 0 || l >= ic) return fail(c, "continuum lower level out of range");
        if (d->cont_nlambda[q] < 2) return fail(c, "cont_nlambda must be >= 2");
        if (!(d->cont_ratio[q] > 1.0)) return fail(c, "cont_ratio must exceed 1");
        a->tl[t] = l;
        a->tu[t] = ic;
        a->kind[t] = 1;
        a->nu0[t] = (a->E[ic] - a->E[l]) / HPLANCK;
        a->alpha0[t] = d->cont_alpha0[q];
        a->ratio[t] = d->cont_ratio[q];
        a->nlam_t[t] = d->cont_nlambda[q];
        a->nu_lo[t] = a->nu0[t];
        a->nu_hi[t] = a->nu0[t] * a->ratio[t];
    }
    gauss_legendre01(a->nmu, a->mu, a->wmu);

    /* grid: bands in transition order; lines on a sinh-stretched symmetric grid
     * x_j = qwing sinh(beta s_j)/sinh(beta), s_j in [-1,1] (beta = 5), continua
     * geometric in frequency from the edge to ratio*edge */
    int64_t n = 0;
    for (int t = 0; t < a->ntr; ++t) n += a->nlam_t[t];
    a->nlam = n;
    a->nu = malloc(n * sizeof(double));
    a->nact = calloc(n, sizeof(int));
    a->act = malloc(n * MAXACT * sizeof(int));
    a->wq = calloc(n * MAXACT, sizeof(double));
    a->prof_slot = malloc(n * MAXACT * sizeof(int));
    int64_t p = 0;
    const double beta = 5.0;
    for (int t = 0; t < a->ntr; ++t) {
        int m = a->nlam_t[t];
        for (int j = 0; j < m; ++j) {
            double nu;
            if (a->kind[t] == 0) {
                double s = -1.0 + 2.0 * j / (m - 1);
                double dnu_ref = a->nu0[t] / CLIGHT * sqrt(2.0 * KBOLTZ * a->T_ref / a->mass);
                nu = a->nu0[t] + a->qwing[t] * sinh(beta * s) / sinh(beta) * dnu_ref;
            } else {
                nu = a->nu0[t] * pow(a->ratio[t], (double)j / (m - 1));
            }
            a->nu[p++] = nu;
        }
    }
    /* active transitions per grid point: owner band plus every transition whose
     * frequency range contains the point (overlapping transitions, Sect. 2.1) */
    int64_t q0 = 0;
    for (int t = 0; t < a->ntr; ++t) {
        for (int j = 0; j < a->nlam_t[t]; ++j) {
            int64_t i = q0 + j;
            double nu = a->nu[i];
            int na = 0;
            for (int s = 0; s < a->ntr; ++s) {
                int inside = (s == t) || (nu >= a->nu_lo[s] * (1 - 1e-13) && nu <= a->nu_hi[s] * (1 + 1e-13));
                if (inside) {
                    if (na >= MAXACT) return fail(c, "too many overlapping transitions at one wavelength");
                    a->act[i * MAXACT + na++] = s;
                }
            }
            a->nact[i] = na;
        }
        q0 += a->nlam_t[t];
    }
    /* quadrature weights: for each transition, trapezoid in frequency over all
     * grid points where it is active */
    double *buf = malloc(2 * n * sizeof(double));
    for (int t = 0; t < a->ntr; ++t) {
        int cnt = 0;
        for (int64_t i = 0; i < n; ++i)
            for (int s = 0; s < a->nact[i]; ++s)
                if (a->act[i * MAXACT + s] == t) {
                    buf[2 * cnt] = a->nu[i];
                    buf[2 * cnt + 1] = (double)(i * MAXACT + s);
                    ++cnt;
                }
        qsort(buf, cnt, 2 * sizeof(double), cmp_dbl_idx);
        for (int j = 0; j < cnt; ++j) {
            double lo = j > 0 ? buf[2 * (j - 1)] : buf[0];
            double hi = j < cnt - 1 ? buf[2 * (j + 1)] : buf[2 * j];
            int64_t slot = (int64_t)buf[2 * j + 1];
            a->wq[slot] = 0.5 * (hi - lo);
        }
    }
    free(buf);
    int np = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int s = 0; s < MAXACT; ++s)
            a->prof_slot[i * MAXACT + s] = (s < a->nact[i] && a->kind[a->act[i * MAXACT + s]] == 0) ? np++ : -1;
    a->nprof = np;
    /* partial redistribution lines: their grid points in frequency order with
     * the line's quadrature weights; two PRD lines may not share a point */
    for (int t = 0; t < d->nline; ++t) {
        if (!(d->line_prd && d->line_prd[t])) continue;
        int q = a->nprd_line++;
        a->prd[t] = 1;
        a->prd_t[q] = t;
        int cnt = 0;
        for (int64_t i = 0; i < n; ++i)
            for (int s2 = 0; s2 < a->nact[i]; ++s2)
                if (a->act[i * MAXACT + s2] == t) ++cnt;
        a->prd_np[q] = cnt;
        a->prd_pts[q] = malloc(cnt * sizeof(int));
        a->prd_w[q] = malloc(cnt * sizeof(double));
        double *b2 = malloc(2 * cnt * sizeof(double));
        int j = 0;
        for (int64_t i = 0; i < n; ++i)
            for (int s2 = 0; s2 < a->nact[i]; ++s2)
                if (a->act[i * MAXACT + s2] == t) {
                    b2[2 * j] = a->nu[i];
                    b2[2 * j + 1] = (double)i;
                    ++j;
                }
        qsort(b2, cnt, 2 * sizeof(double), cmp_dbl_idx);
        for (j = 0; j < cnt; ++j) {
            int64_t i = (int64_t)b2[2 * j + 1];
            a->prd_pts[q][j] = (int)i;
            for (int s2 = 0; s2 < a->nact[i]; ++s2) {
                int t2 = a->act[i * MAXACT + s2];
                if (t2 == t) a->prd_w[q][j] = a->wq[i * MAXACT + s2];
                else if (t2 < d->nline && d->line_prd && d->line_prd[t2])
                    return free(b2), fail(c, "two PRD lines share a wavelength point");
            }
        }
        free(b2);
    }
    return 0;
}

/* ================================================================== */
/* LTE populations and collisional rates                                */
/* ================================================================== */

/* Saha-Boltzmann for the model atom at (T, n_e): n*_i = n*_c n_e Phi_i,
 * Phi_i = g_i/(2 g_c) (h^2/(2 pi m_e k T))^{3/2} exp((E_c - E_i)/kT),
 * normalised so that sum_i n*_i = n_H. */
static void lte_pops(const atom_t *a, double T, double ne, double nH, double *nstar)
{
    int ic = a->nlev - 1;
    double lam3 = pow(HPLANCK * HPLANCK / (2.0 * PI_D * MELEC * KBOLTZ * T), 1.5);
    double phi[MAXLEV], sum = 0.0;
    for (int i = 0; i < ic; ++i) {
        phi[i] = a->g[i] / (2.0 * a->g[ic]) * lam3 * exp((a->E[ic] - a->E[i]) / (KBOLTZ * T));
        sum += phi[i];
    }
    double nc = nH / (1.0 + ne * sum);
    for (int i = 0; i < ic; ++i) nstar[i] = nc * ne * phi[i];
    nstar[ic] = nc;
}

/* electron density: hydrogen Saha plus a metal electron floor f*n_H:
 * n_e = n_p + f n_H with n_p n_e Phi = n_H - n_p  (Phi = sum_i Phi_i), i.e.
 * Phi n_p^2 + (1 + f n_H Phi) n_p - n_H = 0 (stable root). */
double rho_electron_density(const rho_ctx *c, double T, double nH)
{
    const atom_t *a = &c->at;
    int ic = a->nlev - 1;
    double lam3 = pow(HPLANCK * HPLANCK / (2.0 * PI_D * MELEC * KBOLTZ * T), 1.5);
    double Phi = 0.0;
    for (int i = 0; i < ic; ++i)
        Phi += a->g[i] / (2.0 * a->g[ic]) * lam3 * exp((a->E[ic] - a->E[i]) / (KBOLTZ * T));
    double b = 1.0 + a->floor_e * nH * Phi;
    double np = 2.0 * nH / (b + sqrt(b * b + 4.0 * Phi * nH));
    return np + a->floor_e * nH;
}

/* collisional rates C[i][j] (s^-1, from i to j) at one depth:
 *  bound-bound: van Regemorter (1962), C_lu = n_e K Omega/(g_l sqrt T) e^{-y},
 *    K = h^2/((2 pi m_e)^{3/2} sqrt(k)), Omega = (8 pi/sqrt 3)(E_H/dE) g_l f P(y),
 *    P(y) = max(0.2, 0.276 e^y E1(y)), y = dE/kT
 *  bound-free: Seaton (1962), C_lc = 1.55e13 n_e[cm^-3] gbar alpha0[cm^2] e^{-u}/(u sqrt T)
 *    in SI: 1.55e11 n_e alpha0 gbar e^{-u}/(u sqrt T), gbar = 0.1 (hydrogen)
 *  downward by detailed balance with the LTE populations. */
static void collision_rates(const atom_t *a, double T, double ne, const double *nstar, double *C)
{
    int L = a->nlev;
    memset(C, 0, sizeof(double) * L * L);
    const double K = HPLANCK * HPLANCK / (pow(2.0 * PI_D * MELEC, 1.5) * sqrt(KBOLTZ));
    for (int t = 0; t < a->ntr; ++t) {
        int l = a->tl[t], u = a->tu[t];
        double up;
        if (a->kind[t] == 0) {
            double dE = a->E[u] - a->E[l];
            double y = dE / (KBOLTZ * T);
            double P = 0.276 * rho_expE1(y);
            if (P < 0.2) P = 0.2;
            double Omega = 8.0 * PI_D / sqrt(3.0) * (E_RYDBERG / dE) * a->g[l] * a->f[t] * P;
            up = ne * K * Omega / (a->g[l] * sqrt(T)) * exp(-y);
        } else {
            double u0 = HPLANCK * a->nu0[t] / (KBOLTZ * T);
            up = 1.55e11 * ne * a->alpha0[t] * 0.1 * exp(-u0) / (u0 * sqrt(T));
        }
        C[l * L + u] += up;
        C[u * L + l] += up * nstar[l] / nstar[u];
    }
}

/* ================================================================== */
/* Context and column loading                                            */
/* ================================================================== */

int rho_create(rho_ctx **out)
{
    *out = calloc(1, sizeof(rho_ctx));
    return *out ? 0 : 2;
}

static void free_columns(rho_ctx *c)
{
    free(c->z); free(c->T); free(c->nH); free(c->vz); free(c->ne); free(c->np);
    free(c->nstar); free(c->pops); free(c->iters); free(c->status); free(c->dmax);
    if (c->prdc) {
        for (int64_t col = 0; col < c->ncol; ++col) free(c->prdc[col]);
        free(c->prdc);
        c->prdc = NULL;
    }
    c->z = c->T = c->nH = c->vz = c->ne = c->np = c->nstar = c->pops = c->dmax = NULL;
    c->iters = NULL;
    c->status = NULL;
    c->ncol = 0;
}

void rho_destroy(rho_ctx *c)
{
    if (!c) return;
    free_columns(c);
    atom_free(&c->at);
    free(c);
}

const char *rho_last_error(const rho_ctx *c) { return c->err; }

int rho_setup_atom(rho_ctx *c, const rho_atom_desc *d)
{
    if (c->ncol) return fail(c, "atom must be set before columns are loaded"), 4;
    if (atom_build(c, d)) return 1;
    c->have_atom = 1;
    return 0;
}

int64_t rho_nlambda(const rho_ctx *c) { return c->at.nlam; }

int rho_get_grid(const rho_ctx *c, double *nu_out, int32_t *nact_out, int32_t *act_out, double *wq_out)
{
    const atom_t *a = &c->at;
    for (int64_t i = 0; i < a->nlam; ++i) {
        if (nu_out) nu_out[i] = a->nu[i];
        if (nact_out) nact_out[i] = a->nact[i];
        for (int s = 0; s < MAXACT; ++s) {
            if (act_out) act_out[i * MAXACT + s] = s < a->nact[i] ? a->act[i * MAXACT + s] : -1;
            if (wq_out) wq_out[i * MAXACT + s] = s < a->nact[i] ? a->wq[i * MAXACT + s] : 0.0;
        }
    }
    return 0;
}

int rho_atom_info(const rho_ctx *c, double *nu0, double *A, double *Blu, double *Bul, double *mu, double *wmu)
{
    const atom_t *a = &c->at;
    for (int t = 0; t < a->ntr; ++t) {
        if (nu0) nu0[t] = a->nu0[t];
        if (A) A[t] = a->A[t];
        if (Blu) Blu[t] = a->Blu[t];
        if (Bul) Bul[t] = a->Bul[t];
    }
    for (int m = 0; m < a->nmu; ++m) {
        if (mu) mu[m] = a->mu[m];
        if (wmu) wmu[m] = a->wmu[m];
    }
    return 0;
}

int rho_load_columns(rho_ctx *c, int64_t ncol, int32_t ndep, const double *z, const double *T,
                     const double *ne, const double *nH, const double *vz)
{
    if (!c->have_atom) return fail(c, "no atom"), 4;
    if (ncol < 0 || ndep < 2) return fail(c, "ncol >= 0 and ndep >= 2 required");
    for (int64_t i = 0; i < ncol * ndep; ++i) {
        if (!(isfinite(T[i]) && T[i] > 0 && isfinite(nH[i]) && nH[i] > 0 && isfinite(z[i]) &&
              isfinite(vz[i]) && (!ne || (isfinite(ne[i]) && ne[i] > 0)))) {
            char m[200];
            snprintf(m, sizeof m, "invalid input at column %lld depth %lld",
                     (long long)(i / ndep), (long long)(i % ndep));
            return fail(c, m);
        }
        if (i % ndep && !(z[i] < z[i - 1])) return fail(c, "z must decrease with depth index");
    }
    free_columns(c);
    int L = c->at.nlev;
    size_t nd = (size_t)ncol * ndep;
    c->ncol = ncol;
    c->ndep = ndep;
    c->z = malloc(nd * 8); c->T = malloc(nd * 8); c->nH = malloc(nd * 8); c->vz = malloc(nd * 8);
    c->ne = malloc(nd * 8); c->np = malloc(nd * 8);
    c->nstar = malloc(nd * L * 8); c->pops = malloc(nd * L * 8);
    c->iters = calloc(ncol, 4); c->status = malloc(ncol); c->dmax = calloc(ncol, 8);
    if (c->at.nprd_line) c->prdc = calloc(ncol, sizeof(double *));
    memcpy(c->z, z, nd * 8); memcpy(c->T, T, nd * 8); memcpy(c->nH, nH, nd * 8); memcpy(c->vz, vz, nd * 8);
    for (int64_t col = 0; col < ncol; ++col) {
        c->status[col] = ST_NOTRUN;
        for (int k = 0; k < ndep; ++k) {
            size_t i = (size_t)col * ndep + k;
            c->ne[i] = ne ? ne[i] : rho_electron_density(c, T[i], nH[i]);
            double ns[MAXLEV];
            lte_pops(&c->at, T[i], c->ne[i], nH[i], ns);
            c->np[i] = ns[L - 1];
            for (int l = 0; l < L; ++l) {
                c->nstar[((size_t)col * L + l) * ndep + k] = ns[l];
                c->pops[((size_t)col * L + l) * ndep + k] = ns[l];
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Depth-grid optimisation (Sect. 2.3): the atmosphere of every column is
 * interpolated onto a grid that places more points where the temperature,
 * the velocity or the optical depth change fastest, optionally without the
 * layers above a height z_top.  The paper gives no formula; this reading:
 *   - optical depth is represented by the hydrogen column density N_H(z) =
 *     int_z^top n_H dz' (the continuum opacity scales with it), integrated
 *     exactly for n_H exponential between grid points, with n_H(z_0) H_0
 *     above the top point (H_0 the scale height of the top two points);
 *   - the monitor s(z) grows between neighbouring points by
 *       ds = sqrt((d log10 N_H / dN)^2 + (d ln T / dT)^2 + (d v_z / dv)^2
 *                 + (dz / dz_max)^2),
 *     dz_max = spacing_factor x (column height / (ndep_out - 1)) so that no
 *     step exceeds spacing_factor times the uniform one;
 *   - the new points are equidistant in s (equal monitor increments), the
 *     first and last at the column's ends; T and v_z are interpolated
 *     linearly in z, ln n_H and ln n_e linearly in z (exact for exponential
 *     profiles), along the piecewise-linear path of the old grid;
 *   - z_top (use_z_top != 0): the column above z_top is removed, its new top
 *     point at z_top itself.
 * n_e is interpolated (not recomputed), then LTE populations and rates are
 * rebuilt on the new grid by loading the new columns. */
typedef struct {
    double dlog_colden;     /* dN: resolution scale of log10 N_H (dex) */
    double dlnT;            /* dT: of ln T */
    double dvz;             /* dv: of v_z (m/s) */
    double spacing_factor;  /* largest step in units of the uniform step */
    double z_top;           /* m */
    int32_t use_z_top;
} rho_grid_opts;

/* one column: input zi..nei [N], output zo..neo [M]; returns nonzero on bad
 * options for this column (z_top outside it) */
static int regrid_column(int N, const double *zi, const double *Ti, const double *nHi, const double *vzi,
                         const double *nei, int M, const rho_grid_opts *o, double *zo, double *To, double *nHo,
                         double *vzo, double *neo)
{
    /* truncation at z_top: the kept part of the column, top point first */
    double *z = malloc(N * 8), *T = malloc(N * 8), *lnH = malloc(N * 8), *v = malloc(N * 8), *lne = malloc(N * 8);
    double *s = malloc(N * 8), *col = malloc(N * 8);
    int n = 0, k0 = 0, rc = 0;
    if (o->use_z_top && o->z_top < zi[0]) {
        if (!(o->z_top > zi[N - 1])) { rc = 1; goto done; }   /* the cut must leave a layer */
        while (zi[k0] > o->z_top) ++k0;                        /* first point at or below z_top */
        if (zi[k0] < o->z_top) {
            double t = (o->z_top - zi[k0 - 1]) / (zi[k0] - zi[k0 - 1]);
            z[0] = o->z_top;
            T[0] = Ti[k0 - 1] + t * (Ti[k0] - Ti[k0 - 1]);
            lnH[0] = log(nHi[k0 - 1]) + t * (log(nHi[k0]) - log(nHi[k0 - 1]));
            v[0] = vzi[k0 - 1] + t * (vzi[k0] - vzi[k0 - 1]);
            lne[0] = log(nei[k0 - 1]) + t * (log(nei[k0]) - log(nei[k0 - 1]));
            n = 1;
        }
    }
    for (int k = k0; k < N; ++k, ++n) {
        z[n] = zi[k];
        T[n] = Ti[k];
        lnH[n] = log(nHi[k]);
        v[n] = vzi[k];
        lne[n] = log(nei[k]);
    }
    /* hydrogen column density from the top */
    {
        double r = lnH[1] - lnH[0];
        double H0 = r > 1e-12 ? (z[0] - z[1]) / r : (z[0] - z[1]);
        col[0] = exp(lnH[0]) * H0;
        for (int k = 0; k + 1 < n; ++k) {
            double dz = z[k] - z[k + 1], a = exp(lnH[k]), b = exp(lnH[k + 1]), d = lnH[k + 1] - lnH[k];
            col[k + 1] = col[k] + (fabs(d) > 1e-12 ? dz * (b - a) / d : dz * a);
        }
    }
    {
        double dzmax = o->spacing_factor * (z[0] - z[n - 1]) / (M - 1);
        s[0] = 0.0;
        for (int k = 0; k + 1 < n; ++k) {
            double a1 = log10(col[k + 1] / col[k]) / o->dlog_colden;
            double a2 = log(T[k + 1] / T[k]) / o->dlnT;
            double a3 = (v[k + 1] - v[k]) / o->dvz;
            double a4 = (z[k] - z[k + 1]) / dzmax;
            s[k + 1] = s[k] + sqrt(a1 * a1 + a2 * a2 + a3 * a3 + a4 * a4);
        }
    }
    for (int j = 0, k = 0; j < M; ++j) {
        if (j == M - 1) {
            zo[j] = z[n - 1]; To[j] = T[n - 1]; nHo[j] = exp(lnH[n - 1]); vzo[j] = v[n - 1]; neo[j] = exp(lne[n - 1]);
            break;
        }
        double sj = s[n - 1] * j / (M - 1);
        while (k + 2 < n && s[k + 1] < sj) ++k;
        double t = (sj - s[k]) / (s[k + 1] - s[k]);
        zo[j] = z[k] + t * (z[k + 1] - z[k]);
        To[j] = T[k] + t * (T[k + 1] - T[k]);
        nHo[j] = exp(lnH[k] + t * (lnH[k + 1] - lnH[k]));
        vzo[j] = v[k] + t * (v[k + 1] - v[k]);
        neo[j] = exp(lne[k] + t * (lne[k + 1] - lne[k]));
    }
done:
    free(z); free(T); free(lnH); free(v); free(lne); free(s); free(col);
    return rc;
}

int rho_regrid(rho_ctx *c, int32_t ndep_out, const rho_grid_opts *o)
{
    if (!c->ncol) return fail(c, "no columns loaded"), 4;
    if (ndep_out < 2 || !o || !(o->dlog_colden > 0) || !(o->dlnT > 0) || !(o->dvz > 0) ||
        !(o->spacing_factor >= 1.0))
        return fail(c, "invalid regrid options");
    int64_t nc = c->ncol;
    int N = c->ndep, M = ndep_out;
    size_t nd = (size_t)nc * M;
    double *z = malloc(nd * 8), *T = malloc(nd * 8), *nH = malloc(nd * 8), *vz = malloc(nd * 8), *ne = malloc(nd * 8);
    int bad = -1;
    for (int64_t col = 0; col < nc && bad < 0; ++col)
        if (regrid_column(N, c->z + col * N, c->T + col * N, c->nH + col * N, c->vz + col * N, c->ne + col * N, M, o,
                          z + col * M, T + col * M, nH + col * M, vz + col * M, ne + col * M))
            bad = (int)col;
    int rc = 0;
    if (bad >= 0) {
        char m[160];
        snprintf(m, sizeof m, "z_top leaves fewer than two points of column %d", bad);
        rc = fail(c, m);
    } else {
        rc = rho_load_columns(c, nc, M, z, T, ne, nH, vz);
    }
    free(z); free(T); free(nH); free(vz); free(ne);
    return rc;
}

/* the loaded atmosphere [ncol][ndep] (any output may be NULL) */
int rho_get_columns(const rho_ctx *c, double *z, double *T, double *nH, double *vz)
{
    size_t nd = (size_t)c->ncol * c->ndep;
    if (z) memcpy(z, c->z, nd * 8);
    if (T) memcpy(T, c->T, nd * 8);
    if (nH) memcpy(nH, c->nH, nd * 8);
    if (vz) memcpy(vz, c->vz, nd * 8);
    return 0;
}

int rho_get_lte(const rho_ctx *c, double *nstar, double *ne)
{
    size_t nd = (size_t)c->ncol * c->ndep;
    if (nstar) memcpy(nstar, c->nstar, nd * c->at.nlev * 8);
    if (ne) memcpy(ne, c->ne, nd * 8);
    return 0;
}

int rho_get_populations(const rho_ctx *c, double *n, int32_t *iters, uint8_t *status, double *dmax)
{
    size_t nd = (size_t)c->ncol * c->ndep;
    if (n) memcpy(n, c->pops, nd * c->at.nlev * 8);
    if (iters) memcpy(iters, c->iters, c->ncol * 4);
    if (status) memcpy(status, c->status, c->ncol);
    if (dmax) memcpy(dmax, c->dmax, c->ncol * 8);
    return 0;
}

int rho_set_populations(rho_ctx *c, const double *n)
{
    size_t nd = (size_t)c->ncol * c->ndep * c->at.nlev;
    for (size_t i = 0; i < nd; ++i)
        if (!(isfinite(n[i]) && n[i] > 0)) return fail(c, "populations must be finite and positive");
    memcpy(c->pops, n, nd * 8);
    return 0;
}

/* ================================================================== */
/* Per-column workspace: atmosphere-only quantities                      */
/* ================================================================== */
typedef struct {
    int N;
    double *dz;       /* [N-1] */
    double *Bnu;      /* [nlam][N] */
    double *chic;     /* [nlam][N] background opacity */
    double *etac;     /* [nlam][N] background emissivity */
    double *ex;       /* [nlam][N] exp(-h nu / k T) */
    double *prof;     /* [nprof][nmu][2][N] line profile (Hz^-1) */
    double *C;        /* [N][L][L] collisional rates */
    double *Gam;      /* [N][L][L] rate matrix */
    /* sweep scratch */
    double *chi, *eta, *etaact, *S, *dtau, *I, *lam, *Ieff, *omlam, *Sbg;
    double *chit, *Vlu, *Vul, *Ut;   /* [MAXACT][N] */
    double *hist;     /* Ng history [4][L*N] */
    /* partial redistribution */
    double *rho;      /* [nlam][N] psi/phi of the PRD line at each grid point (1 elsewhere) */
    double *Jp;       /* [nlam][N] angle-averaged mean intensity at the PRD points */
    double *Dp;       /* [nlam][N] local derivative dJ/drho of the mean intensity at a PRD point
                       * with respect to its own rho (through the line's emission, Psi*) */
    double *U0;       /* [MAXACT][N] U of each active transition without the factor rho */
    double *rplain;   /* [nlam][N] the last update's plain ratio r (before switching) */
    double *rhist;    /* Ng history of rho at the PRD points [4][npt N], newest first */
    double *Pup, *Pdn;    /* [ntr][N] plain radiative rate coefficients (actual I, not I_eff) */
    double *Iray;     /* [2 nmu][nlam][N] intensity of each ray at the PRD points (hybrid PRD) */
    double *Dray;     /* [2 nmu][nlam][N] each ray's dI/drho through the line's own emission */
    const double *vz; /* the column's vertical velocity (hybrid PRD) */
    int hybrid;       /* 1: rho in the fluid frame (hybrid PRD) */
    int bezier;       /* 1: quadratic Bezier formal solver */
    double *prdK[MAXTR];   /* per PRD line [N][np][np]: normalised redistribution kernel */
    double *prdf[MAXTR];   /* per PRD line [N][np]: weights of J-bar */
} work_t;

static void work_alloc(work_t *w, const atom_t *a, int N)
{
    int L = a->nlev;
    memset(w, 0, sizeof *w);
    w->N = N;
    w->dz = malloc(N * 8);
    w->Bnu = malloc(a->nlam * N * 8);
    w->chic = malloc(a->nlam * N * 8);
    w->etac = malloc(a->nlam * N * 8);
    w->ex = malloc(a->nlam * N * 8);
    w->prof = malloc((size_t)(a->nprof > 0 ? a->nprof : 1) * a->nmu * 2 * N * 8);
    w->C = malloc(N * L * L * 8);
    w->Gam = malloc(N * L * L * 8);
    w->chi = malloc(N * 8); w->eta = malloc(N * 8); w->etaact = malloc(N * 8);
    w->S = malloc(N * 8); w->dtau = malloc(N * 8); w->I = malloc(N * 8); w->lam = malloc(N * 8);
    w->Ieff = malloc(N * 8); w->omlam = malloc(N * 8); w->Sbg = malloc(N * 8);
    w->chit = malloc(MAXACT * N * 8); w->Vlu = malloc(MAXACT * N * 8);
    w->Vul = malloc(MAXACT * N * 8); w->Ut = malloc(MAXACT * N * 8);
    w->hist = malloc(4 * L * N * 8);
    w->rho = malloc(a->nlam * N * 8);
    w->Jp = malloc(a->nlam * N * 8);
    w->Dp = malloc(a->nlam * N * 8);
    w->U0 = malloc(MAXACT * N * 8);
    w->rplain = malloc(a->nlam * N * 8);
    {
        size_t npt = 0;
        for (int q = 0; q < a->nprd_line; ++q) npt += (size_t)a->prd_np[q];
        w->rhist = malloc(4 * (npt > 0 ? npt : 1) * N * 8);
    }
    w->Pup = malloc((size_t)a->ntr * N * 8);
    w->Pdn = malloc((size_t)a->ntr * N * 8);
    w->Iray = a->nprd_line ? malloc((size_t)2 * a->nmu * a->nlam * N * 8) : NULL;
    w->Dray = a->nprd_line ? calloc((size_t)2 * a->nmu * a->nlam * N, 8) : NULL;
    for (int64_t i = 0; i < a->nlam * N; ++i) w->rho[i] = 1.0;
    for (int q = 0; q < a->nprd_line; ++q) {
        w->prdK[q] = malloc((size_t)N * a->prd_np[q] * a->prd_np[q] * 8);
        w->prdf[q] = malloc((size_t)N * a->prd_np[q] * 8);
    }
}

static void work_free(work_t *w)
{
    free(w->dz); free(w->Bnu); free(w->chic); free(w->etac); free(w->ex); free(w->prof);
    free(w->C); free(w->Gam); free(w->chi); free(w->eta); free(w->etaact); free(w->S);
    free(w->dtau); free(w->I); free(w->lam); free(w->chit); free(w->Vlu); free(w->Vul);
    free(w->Ieff); free(w->omlam); free(w->Sbg);
    free(w->Ut); free(w->hist);
    free(w->rho); free(w->Jp); free(w->Pup); free(w->Pdn); free(w->Iray); free(w->Dray);
    free(w->Dp); free(w->U0); free(w->rplain); free(w->rhist);
    for (int q = 0; q < MAXTR; ++q) {
        if (w->prdK[q]) free(w->prdK[q]);
        if (w->prdf[q]) free(w->prdf[q]);
    }
}

/* free-free (Kramers, g_ff = 1) absorption coefficient constant, SI:
 * chi_ff = C_ff n_e n_p T^{-1/2} nu^{-3} (1 - e^{-h nu/kT}),
 * C_ff = (e^2/(4 pi eps0))^3 4/(3 m_e h c) sqrt(2 pi/(3 k m_e)) */
double rho_cff(void)
{
    double e2 = QELEC * QELEC / (4.0 * PI_D * EPS0);
    return e2 * e2 * e2 * 4.0 / (3.0 * MELEC * HPLANCK * CLIGHT) * sqrt(2.0 * PI_D / (3.0 * KBOLTZ * MELEC));
}

/* H- bound-free cross section [m^2] (John 1988, A&A 193, 189, fit for
 * lambda < 1.6419 um): sigma = 1e-18 lambda^3 (1/lambda - 1/lambda0)^{3/2}
 * f(lambda) cm^2 with f = sum_n C_n (1/lambda - 1/lambda0)^{(n-1)/2}, lambda in um. */
double rho_hminus_sigma(double lambda_m)
{
    const double l0 = 1.6419;
    const double Cn[6] = {152.519, 49.534, -118.858, 92.536, -34.194, 4.982};
    double lum = lambda_m * 1e6;
    if (!(lum < l0)) return 0.0;
    double x = 1.0 / lum - 1.0 / l0;
    double f = 0.0, xp = 1.0, sx = sqrt(x);
    for (int n = 0; n < 6; ++n) {
        f += Cn[n] * xp;
        xp *= sx;
    }
    return 1e-18 * lum * lum * lum * x * sx * f * 1e-4;
}

/* LTE H- number density: n(H-) = n(H I, ground) n_e (1/4) (h^2/(2 pi m_e k T))^{3/2} e^{0.754 eV/kT}
 * (g(H-) = 1, g(H I, 1s) = 2) */
static double hminus_density(double nH1, double ne, double T)
{
    double lam3 = pow(HPLANCK * HPLANCK / (2.0 * PI_D * MELEC * KBOLTZ * T), 1.5);
    return 0.25 * nH1 * ne * lam3 * exp(0.754 * QELEC / (KBOLTZ * T));
}

/* Voigt damping at depth k: log-interpolated in depth index from top to bottom */
static double damping(const atom_t *a, int t, int k, int N)
{
    double s = N > 1 ? (double)k / (N - 1) : 0.0;
    return exp((1.0 - s) * log(a->a_top[t]) + s * log(a->a_bot[t]));
}

/* Line profile phi(nu) = H(a, v)/(sqrt(pi) dnu_D) for a ray with vertical
 * direction cosine mu_z (positive upward).  The Doppler shift of the ray:
 * v = (nu - nu0)/dnu_D - mu_z v_z / v_th (v_z > 0 upward). */
static double line_profile(const atom_t *a, int t, double nu, double T, double vz, double mu_z, double adamp)
{
    double vth = sqrt(2.0 * KBOLTZ * T / a->mass);
    double dnuD = a->nu0[t] * vth / CLIGHT;
    double v = (nu - a->nu0[t]) / dnuD - mu_z * vz / vth;
    return rho_voigt(adamp, v) / (sqrt(PI_D) * dnuD);
}

/* Partial redistribution: the redistribution kernel of PRD line q at depth k
 * of column col on the line's points, K[i][j] = R(x_j, x_i) w_j / sum_j (...)
 * (the discrete normalisation makes a frequency-independent J give rho = 1),
 * and the weights of J-bar, f_j = H(a, x_j) w_j / sum (...); x in Doppler
 * units of the depth, static frame.  R is symmetric in its arguments, so
 * each unordered pair is evaluated once. */
static void prd_kernel_depth(const rho_ctx *c, int64_t col, int q, int k, double *K, double *f)
{
    const atom_t *a = &c->at;
    int N = c->ndep, t = a->prd_t[q], m = a->prd_np[q];
    double T = c->T[col * N + k];
    double dnuD = a->nu0[t] / CLIGHT * sqrt(2.0 * KBOLTZ * T / a->mass);
    double ad = damping(a, t, k, N);
    double fs = 0.0;
    for (int j = 0; j < m; ++j) {
        double xj = (a->nu[a->prd_pts[q][j]] - a->nu0[t]) / dnuD;
        f[j] = rho_voigt(ad, xj) * a->prd_w[q][j];
        fs += f[j];
    }
    for (int j = 0; j < m; ++j) f[j] /= fs;
    for (int i = 0; i < m; ++i) {
        double xi = (a->nu[a->prd_pts[q][i]] - a->nu0[t]) / dnuD;
        for (int j = i; j < m; ++j) {
            double xj = (a->nu[a->prd_pts[q][j]] - a->nu0[t]) / dnuD;
            double r = rho_r2a(ad, xj, xi);
            K[i * m + j] = r * a->prd_w[q][j];
            K[j * m + i] = r * a->prd_w[q][i];
        }
    }
    for (int i = 0; i < m; ++i) {
        double rs = 0.0;
        for (int j = 0; j < m; ++j) rs += K[i * m + j];
        for (int j = 0; j < m; ++j) K[i * m + j] /= rs;
    }
}

/* offsets of line q's kernel and weights inside a column's cache entry */
static size_t prd_cache_koff(const atom_t *a, int N, int q)
{
    size_t off = 0;
    for (int p = 0; p < q; ++p) off += (size_t)N * a->prd_np[p] * (a->prd_np[p] + 1);
    return off;
}

static double *prd_cache_alloc(const rho_ctx *c, int64_t col)
{
    const atom_t *a = &c->at;
    if (!c->prdc) return NULL;
    if (!c->prdc[col]) c->prdc[col] = malloc(sizeof(double) * prd_cache_koff(a, c->ndep, a->nprd_line));
    return c->prdc[col];
}

/* build the cache entry of one column (one thread) */
static void prd_cache_column(const rho_ctx *c, int64_t col)
{
    const atom_t *a = &c->at;
    int N = c->ndep;
    double *e = prd_cache_alloc(c, col);
    if (!e) return;
    for (int q = 0; q < a->nprd_line; ++q) {
        size_t m = a->prd_np[q];
        double *K = e + prd_cache_koff(a, N, q), *f = K + (size_t)N * m * m;
        for (int k = 0; k < N; ++k) prd_kernel_depth(c, col, q, k, K + (size_t)k * m * m, f + (size_t)k * m);
    }
}

/* build the cache entries of every column that has none, in parallel over
 * (column, line, depth) */
typedef struct {
    const rho_ctx *c;
    const int64_t *cols;   /* the columns to build */
    int64_t ntask, next;
    pthread_mutex_t mu;
} kpool_t;

static void *kpool_worker(void *arg)
{
    kpool_t *p = arg;
    const rho_ctx *c = p->c;
    const atom_t *a = &c->at;
    int N = c->ndep, nq = a->nprd_line;
    for (;;) {
        pthread_mutex_lock(&p->mu);
        int64_t tk = p->next++;
        pthread_mutex_unlock(&p->mu);
        if (tk >= p->ntask) break;
        int64_t col = p->cols[tk / ((int64_t)nq * N)];
        int q = (int)(tk / N % nq), k = (int)(tk % N);
        size_t m = a->prd_np[q];
        double *K = c->prdc[col] + prd_cache_koff(a, N, q), *f = K + (size_t)N * m * m;
        prd_kernel_depth(c, col, q, k, K + (size_t)k * m * m, f + (size_t)k * m);
    }
    return NULL;
}

static void prd_cache_build(rho_ctx *c, int nthreads)
{
    const atom_t *a = &c->at;
    if (!a->nprd_line || !c->prdc) return;
    int64_t *cols = malloc(sizeof(int64_t) * c->ncol), n = 0;
    for (int64_t col = 0; col < c->ncol; ++col)
        if (!c->prdc[col] && prd_cache_alloc(c, col)) cols[n++] = col;
    if (n) {
        kpool_t p = {c, cols, n * a->nprd_line * c->ndep, 0, PTHREAD_MUTEX_INITIALIZER};
        pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
        for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, kpool_worker, &p);
        for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
        free(th);
    }
    free(cols);
}

static void column_setup(const rho_ctx *c, int64_t col, work_t *w)
{
    const atom_t *a = &c->at;
    int N = c->ndep, L = a->nlev;
    const double *z = c->z + col * N, *T = c->T + col * N, *vz = c->vz + col * N;
    const double *ne = c->ne + col * N, *np = c->np + col * N;
    const double Cff = rho_cff();
    for (int k = 0; k < N - 1; ++k) w->dz[k] = fabs(z[k] - z[k + 1]);
    for (int64_t i = 0; i < a->nlam; ++i) {
        double nu = a->nu[i];
        for (int k = 0; k < N; ++k) {
            double x = HPLANCK * nu / (KBOLTZ * T[k]);
            double B = rho_planck(nu, T[k]);
            double nhm = hminus_density(c->nstar[((size_t)col * L + 0) * N + k], ne[k], T[k]);
            double chi = (Cff * ne[k] * np[k] / sqrt(T[k]) / (nu * nu * nu) + nhm * rho_hminus_sigma(CLIGHT / nu))
                         * (-expm1(-x)) + SIGMA_T * ne[k];
            w->Bnu[i * N + k] = B;
            w->chic[i * N + k] = chi;
            w->etac[i * N + k] = chi * B;   /* background in LTE (Thomson treated as thermal) */
            w->ex[i * N + k] = exp(-x);
        }
        for (int s = 0; s < a->nact[i]; ++s) {
            int ps = a->prof_slot[i * MAXACT + s];
            if (ps < 0) continue;
            int t = a->act[i * MAXACT + s];
            for (int m = 0; m < a->nmu; ++m)
                for (int d = 0; d < 2; ++d) {
                    double muz = d == 0 ? -a->mu[m] : a->mu[m];   /* d=0 downward, d=1 upward */
                    double *p = w->prof + (((size_t)ps * a->nmu + m) * 2 + d) * N;
                    for (int k = 0; k < N; ++k)
                        p[k] = line_profile(a, t, nu, T[k], vz[k], muz, damping(a, t, k, N));
                }
        }
    }
    for (int k = 0; k < N; ++k) {
        double ns[MAXLEV];
        for (int l = 0; l < L; ++l) ns[l] = c->nstar[((size_t)col * L + l) * N + k];
        collision_rates(a, T[k], ne[k], ns, w->C + (size_t)k * L * L);
    }
    /* partial redistribution: the kernels of every PRD line and depth
     * (prd_kernel_depth), from the column's cache entry */
    if (!a->nprd_line) return;
    if (!(c->prdc && c->prdc[col])) prd_cache_column(c, col);
    const double *src = c->prdc ? c->prdc[col] : NULL;
    if (src) {
        for (int q = 0; q < a->nprd_line; ++q) {
            size_t m = a->prd_np[q];
            memcpy(w->prdK[q], src, sizeof(double) * N * m * m);
            src += (size_t)N * m * m;
            memcpy(w->prdf[q], src, sizeof(double) * N * m);
            src += (size_t)N * m;
        }
    } else {
        for (int q = 0; q < a->nprd_line; ++q)
            for (int k = 0; k < N; ++k)
                prd_kernel_depth(c, col, q, k, w->prdK[q] + (size_t)k * a->prd_np[q] * a->prd_np[q],
                                 w->prdf[q] + (size_t)k * a->prd_np[q]);
    }
}

/* PRD switching (Sect. 2.3, Eq. 1): rho' = eps rho + (1 - eps).  The paper
 * starts eps at a small eps0, raises it with the square of the iteration
 * number until it reaches unity, and states that this takes about
 * eps0^{-1/2} iterations; read as eps_it = min(1, eps0 it^2) for the rho that
 * the formal solution of iteration it uses (eps_1 = eps0; the literal
 * compounding product eps0 1^2 2^2 ... 3^2 would reach unity far sooner than
 * eps0^{-1/2}).  eps0 <= 0 switches it off (eps = 1). */
double rho_prd_switch_eps(double eps0, int32_t it)
{
    if (!(eps0 > 0.0)) return 1.0;
    return fmin(1.0, eps0 * (double)it * (double)it);
}

/* Collisional-radiative switching (Sect. 2.3, after Hummer & Voels 1988):
 * the collisional rates of iteration it are multiplied by
 * max(1, f0 10^{-(it-1)}), so the first iteration uses f0 and the factor
 * falls by a decade per iteration until it reaches unity (the paper gives
 * only the range of f0, 10 to 1e5, and "decreased until it reaches unity").
 * f0 <= 1 switches it off. */
double rho_crsw_factor(double f0, int32_t it)
{
    if (!(f0 > 1.0)) return 1.0;
    double f = f0 * pow(10.0, -(double)(it - 1));
    return f > 1.0 ? f : 1.0;
}

/* Hybrid approximation of angle-dependent PRD in moving atmospheres (Sect.
 * 2.1, Leenaarts et al. 2012): the redistribution is angle-averaged in the
 * frame of the moving gas, where the atmosphere is locally static.  A photon
 * of observer-frame frequency nu travelling with direction cosine mu_z has
 * the frequency nu - nu0 mu_z v_z / c in the gas (the same shift the line
 * profile carries), so
 *   J_f(nu_i) = sum over rays (w_mu / 2) I_ray(nu_i + nu0 mu_z v_z / c),
 * the mean intensity at the line's points in the gas frame, replaces J in
 * the update of rho (which is then rho_f, a function of the gas-frame
 * frequency), and the ray (mu_z) at observer frequency nu emits with
 * rho_f(nu - nu0 mu_z v_z / c).  Both transfers are linear interpolations
 * in frequency over the line's points, held constant beyond its first and
 * last point.  Without velocity every shifted frequency is a grid point and
 * the scheme is the static-frame one exactly. */

/* v at frequency nu by linear interpolation over PRD line q's points (sorted
 * by increasing frequency) at depth k; v[pt * N + k] holds the value at grid
 * point pt */
static double prd_interp(const atom_t *a, int q, int N, int k, const double *v, double nu)
{
    const int m = a->prd_np[q];
    const int *pt = a->prd_pts[q];
    if (nu <= a->nu[pt[0]]) return v[(size_t)pt[0] * N + k];
    if (nu >= a->nu[pt[m - 1]]) return v[(size_t)pt[m - 1] * N + k];
    int lo = 0, hi = m - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (a->nu[pt[mid]] <= nu) lo = mid;
        else hi = mid;
    }
    double na = a->nu[pt[lo]], nb = a->nu[pt[hi]];
    if (!(nb > na)) return v[(size_t)pt[lo] * N + k];
    double t = (nu - na) / (nb - na);
    return (1.0 - t) * v[(size_t)pt[lo] * N + k] + t * v[(size_t)pt[hi] * N + k];
}

/* PRD line of transition t (-1: none) */
static int prd_line_of(const atom_t *a, int t)
{
    for (int q = 0; q < a->nprd_line; ++q)
        if (a->prd_t[q] == t) return q;
    return -1;
}

/* the bracket of frequency nu among PRD line q's points: interpolation
 * between points lo and hi = lo + 1 with weight t on hi, or lo = hi with
 * t = 0 beyond the line's first or last point (prd_interp's rule) */
static void prd_bracket(const atom_t *a, int q, double nu, int *lo_out, int *hi_out, double *t_out)
{
    const int m = a->prd_np[q];
    const int *pt = a->prd_pts[q];
    if (nu <= a->nu[pt[0]] || nu >= a->nu[pt[m - 1]]) {
        *lo_out = *hi_out = nu <= a->nu[pt[0]] ? 0 : m - 1;
        *t_out = 0.0;
        return;
    }
    int lo = 0, hi = m - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (a->nu[pt[mid]] <= nu) lo = mid;
        else hi = mid;
    }
    *lo_out = lo;
    *hi_out = hi;
    *t_out = (nu - a->nu[pt[lo]]) / (a->nu[pt[hi]] - a->nu[pt[lo]]);
}

/* weight of point i of PRD line q in the interpolation at frequency nu */
static double prd_weight(const atom_t *a, int q, int i, double nu)
{
    int lo, hi;
    double t;
    prd_bracket(a, q, nu, &lo, &hi, &t);
    if (lo == hi) return lo == i ? 1.0 : 0.0;
    return (lo == i ? 1.0 - t : 0.0) + (hi == i ? t : 0.0);
}

/* the hybrid scheme's local derivative of J_f at point i with respect to
 * rho_f at the same point, through the line's own emission: J_f(i) takes
 * ray r's intensity at nu_i + s_r (s_r = nu0 mu_z v_z / c) from the points
 * j around it (weights c_j), and the ray emits at point j with rho_f
 * interpolated at nu_j - s_r, where point i has the weight e_ij; with dr_j
 * = dI_r(nu_j)/drho there (Psi* n_u U0),
 *   D_f(i) = sum over rays (w_mu / 2) sum_j c_j dr_j e_ij. */
static void prd_fluid_D(const atom_t *a, const work_t *w, int q, int N, int k, double *Dl)
{
    const int t = a->prd_t[q], m = a->prd_np[q];
    const int *pt = a->prd_pts[q];
    for (int i = 0; i < m; ++i) Dl[i] = 0.0;
    for (int mu = 0; mu < a->nmu; ++mu)
        for (int d = 0; d < 2; ++d) {
            const double muz = d == 0 ? -a->mu[mu] : a->mu[mu];
            const double sh = a->nu0[t] * muz * w->vz[k] / CLIGHT;
            const double *dr = w->Dray + (size_t)(mu * 2 + d) * a->nlam * N;
            for (int i = 0; i < m; ++i) {
                int lo, hi;
                double tt;
                prd_bracket(a, q, a->nu[pt[i]] + sh, &lo, &hi, &tt);
                double s = (1.0 - tt) * dr[(size_t)pt[lo] * N + k] * prd_weight(a, q, i, a->nu[pt[lo]] - sh);
                if (hi != lo) s += tt * dr[(size_t)pt[hi] * N + k] * prd_weight(a, q, i, a->nu[pt[hi]] - sh);
                Dl[i] += 0.5 * a->wmu[mu] * s;
            }
        }
}

/* gas-frame mean intensity of PRD line q at depth k at its points (Jl[m]);
 * rays in the order the formal solution accumulates the static-frame J */
static void prd_fluid_J(const atom_t *a, const work_t *w, int q, int N, int k, double *Jl)
{
    const int t = a->prd_t[q], m = a->prd_np[q];
    for (int i = 0; i < m; ++i) Jl[i] = 0.0;
    for (int mu = 0; mu < a->nmu; ++mu)
        for (int d = 0; d < 2; ++d) {
            const double muz = d == 0 ? -a->mu[mu] : a->mu[mu];
            const double sh = a->nu0[t] * muz * w->vz[k] / CLIGHT;
            const double *Ir = w->Iray + (size_t)(mu * 2 + d) * a->nlam * N;
            for (int i = 0; i < m; ++i)
                Jl[i] += 0.5 * a->wmu[mu] * prd_interp(a, q, N, k, Ir, a->nu[a->prd_pts[q][i]] + sh);
        }
}

/* rho = psi/phi of every PRD line after a solve (Uitenbroek 2001, Eq. 14,
 * angle-averaged, coherent scattering in the atom's frame, gamma = 1):
 *   r_i = 1 + F [sum_j K_ij J_j / Jbar - 1],  Jbar = sum_j f_j J_j,
 *   F = n_l R_lu / sum_k n_k P_ku,
 * the fraction of the upper level's supply that is absorption in the line,
 * with the actual (not preconditioned) radiative rates of the formal solution
 * just done plus collisions and the populations of the next iteration; at
 * statistical equilibrium sum_k n_k P_ku = n_u P_u and R_lu = B_lu Jbar, the
 * usual n_l B_lu (sum K J - Jbar)/(n_u P_u), and F in [0, 1] keeps r >= 0.
 * PRD switching (Eq. 1): r' = eps r + (1 - eps), eps = rho_prd_switch_eps(eps0,
 * it_next) for the iteration it_next that uses the new rho.
 *
 * The map rho -> r' is iterated with the formal solution in between: in
 * optically thick wings, where the redistribution is coherent, that is a
 * Lambda iteration on the scattered light and converges at the pace of one.
 * With Ng acceleration (jacobi = 1) the update takes one Jacobi (diagonal
 * Newton) step,
 *   rho_new = rho + (r' - rho) / max(1 - eps g_ii, RHO_JACOBI_FLOOR),
 *   g_ii = d r_i / d rho_i = F D_i (K_ii - f_i sum_j K_ij J_j / Jbar) / Jbar,
 * D_i = dJ_i/drho_i the local derivative of the mean intensity through the
 * line's own emission (Psi*, accumulated in rate_matrix): the ALI idea applied
 * to rho.  The floor bounds the step at 50 times the plain one where the
 * local derivative nears unity; Ng acceleration of the rho sequence (Sect.
 * 2.3: Ng "both for the Lambda-iterations and the PRD iterations", applied by
 * the caller) controls the oscillating mode of the coupled update.  Without
 * Ng (jacobi = 0) the plain update is damped instead, rho_new = (rho + r')/2:
 * undamped, it oscillates and diverges in thick Lyman alpha wings.  Either
 * way the fixed point is rho = r'. */
#define RHO_JACOBI_FLOOR 0.02
static void prd_update(const rho_ctx *c, int64_t col, work_t *w, const double *n, int it_next, double eps0,
                       int jacobi)
{
    const atom_t *a = &c->at;
    int N = c->ndep, L = a->nlev;
    double eps = rho_prd_switch_eps(eps0, it_next);
    (void)col;
    for (int q = 0; q < a->nprd_line; ++q) {
        int t = a->prd_t[q], m = a->prd_np[q], l = a->tl[t], u = a->tu[t];
        double *Jl = malloc(sizeof(double) * m), *Dl = malloc(sizeof(double) * m);
        for (int k = 0; k < N; ++k) {
            const double *K = w->prdK[q] + (size_t)k * m * m, *f = w->prdf[q] + (size_t)k * m;
            /* the mean intensity at the line's points: static frame, or the
             * gas frame for the hybrid scheme */
            if (w->hybrid) {
                prd_fluid_J(a, w, q, N, k, Jl);
                if (jacobi) prd_fluid_D(a, w, q, N, k, Dl);
            } else {
                for (int j = 0; j < m; ++j) {
                    Jl[j] = w->Jp[(size_t)a->prd_pts[q][j] * N + k];
                    Dl[j] = w->Dp[(size_t)a->prd_pts[q][j] * N + k];
                }
            }
            /* supply of the upper level: radiative (plain) and collisional */
            double in = 0.0;
            for (int t2 = 0; t2 < a->ntr; ++t2) {
                if (a->tu[t2] == u) in += n[a->tl[t2] * N + k] * w->Pup[(size_t)t2 * N + k];
                if (a->tl[t2] == u) in += n[a->tu[t2] * N + k] * w->Pdn[(size_t)t2 * N + k];
            }
            for (int p = 0; p < L; ++p)
                if (p != u) in += n[p * N + k] * w->C[(size_t)k * L * L + p * L + u];
            double F = n[l * N + k] * w->Pup[(size_t)t * N + k] / in;
            double jbar = 0.0;
            for (int j = 0; j < m; ++j) jbar += f[j] * Jl[j];
            for (int i = 0; i < m; ++i) {
                size_t gi = (size_t)a->prd_pts[q][i] * N + k;
                double sr = 0.0;
                for (int j = 0; j < m; ++j) sr += K[i * m + j] * Jl[j];
                double r = 1.0 + F * (sr / jbar - 1.0);
                w->rplain[gi] = r;
                double den = 2.0;
                if (jacobi) {
                    double g = F * (K[i * m + i] - f[i] * sr / jbar) * Dl[i] / jbar;
                    den = 1.0 - eps * g;
                    if (den < RHO_JACOBI_FLOOR) den = RHO_JACOBI_FLOOR;
                }
                w->rho[gi] += ((eps * r + (1.0 - eps)) - w->rho[gi]) / den;
            }
        }
        free(Jl);
        free(Dl);
    }
}

/* rho of every PRD point and depth gathered into (dir 0) or scattered from
 * (dir 1) one vector, lines and points in order, depth fastest */
static void rho_vector(const atom_t *a, int N, double *rho, double *v, int dir)
{
    size_t p = 0;
    for (int q = 0; q < a->nprd_line; ++q)
        for (int i = 0; i < a->prd_np[q]; ++i)
            for (int k = 0; k < N; ++k, ++p) {
                double *r = rho + (size_t)a->prd_pts[q][i] * N + k;
                if (dir == 0) v[p] = *r;
                else *r = v[p];
            }
}

/* per-transition V_lu, V_ul, U_ul and chi_t on all depths for grid point i, ray (m,d) */
static void transition_coeffs(const rho_ctx *c, int64_t col, const work_t *w, const double *n,
                              int64_t i, int m, int d)
{
    const atom_t *a = &c->at;
    int N = c->ndep, L = a->nlev;
    double nu = a->nu[i];
    for (int s = 0; s < a->nact[i]; ++s) {
        int t = a->act[i * MAXACT + s], l = a->tl[t], u = a->tu[t];
        double *Vlu = w->Vlu + s * N, *Vul = w->Vul + s * N, *U = w->Ut + s * N, *ch = w->chit + s * N;
        double *U0 = w->U0 + s * N;
        if (a->kind[t] == 0) {
            const double *p = w->prof + (((size_t)a->prof_slot[i * MAXACT + s] * a->nmu + m) * 2 + d) * N;
            double h4 = HPLANCK * nu / (4.0 * PI_D);
            const int q = (a->prd[t] && w->hybrid) ? prd_line_of(a, t) : -1;
            const double muz = d == 0 ? -a->mu[m] : a->mu[m];
            for (int k = 0; k < N; ++k) {
                /* partial redistribution: emission and stimulated emission
                 * with psi = rho phi (hybrid: rho of the gas-frame frequency) */
                double r = a->prd[t] ? w->rho[i * N + k] : 1.0;
                if (q >= 0) r = prd_interp(a, q, N, k, w->rho, nu - a->nu0[t] * muz * w->vz[k] / CLIGHT);
                Vlu[k] = h4 * a->Blu[t] * p[k];
                Vul[k] = a->g[l] / a->g[u] * Vlu[k] * r;
                U0[k] = h4 * a->A[t] * p[k];
                U[k] = U0[k] * r;
            }
        } else {
            double r = a->nu0[t] / nu;
            double alpha = a->alpha0[t] * r * r * r;
            double tw = 2.0 * HPLANCK * nu * nu * nu / (CLIGHT * CLIGHT);
            for (int k = 0; k < N; ++k) {
                double G = c->nstar[((size_t)col * L + l) * N + k] / c->nstar[((size_t)col * L + u) * N + k];
                Vlu[k] = alpha;
                Vul[k] = G * w->ex[i * N + k] * alpha;
                U[k] = tw * Vul[k];
                U0[k] = U[k];
            }
        }
        for (int k = 0; k < N; ++k) ch[k] = n[l * N + k] * Vlu[k] - n[u * N + k] * Vul[k];
    }
}

/* Formal solution for grid point i, ray (m, d) with populations n; fills
 * w->I, w->lam (dI/dS) and the opacities.  d = 0: downward ray from the top
 * (no incident radiation); d = 1: upward ray from the bottom with the
 * diffusion approximation I = B + mu dB/dtau (vertical tau). */
static void formal_ray(const rho_ctx *c, int64_t col, work_t *w, const double *n, int64_t i, int m, int d)
{
    const atom_t *a = &c->at;
    int N = c->ndep, L = a->nlev;
    (void)L;
    for (int k = 0; k < N; ++k) {
        double chi = w->chic[i * N + k], eta = w->etac[i * N + k], ea = 0.0;
        for (int s = 0; s < a->nact[i]; ++s) {
            int t = a->act[i * MAXACT + s];
            chi += w->chit[s * N + k];
            ea += n[a->tu[t] * N + k] * w->Ut[s * N + k];
        }
        w->chi[k] = chi;
        w->eta[k] = eta + ea;
        w->etaact[k] = ea;
        w->S[k] = w->eta[k] / chi;
        w->Sbg[k] = eta / chi;
    }
    double mu = a->mu[m];
    for (int k = 0; k < N - 1; ++k) w->dtau[k] = 0.5 * (w->chi[k] + w->chi[k + 1]) * w->dz[k] / mu;
    void (*sweep)(int, const double *, const double *, const double *, double, int, double *, double *, double *,
                  double *) = w->bezier ? sc_sweep_bezier : sc_sweep_full;
    if (d == 0) {
        sweep(N, w->dtau, w->S, w->Sbg, 0.0, +1, w->I, w->lam, w->Ieff, w->omlam);
    } else {
        double dtv = 0.5 * (w->chi[N - 1] + w->chi[N - 2]) * w->dz[N - 2];
        double B1 = w->Bnu[i * N + N - 1], B2 = w->Bnu[i * N + N - 2];
        sweep(N, w->dtau, w->S, w->Sbg, B1 + mu * (B1 - B2) / dtv, -1, w->I, w->lam, w->Ieff, w->omlam);
    }
}

/* ------------------------------------------------------------------ */
/* Rate matrix.  A[r][q] is the coefficient of n_q in dn_r/dt (columns sum
 * to zero).  mode 0: MALI (Rybicki & Hummer 1992): the radiative terms use
 * I_eff = I - Psi* eta_act (the intensity without the local emission of the
 * active atom, at the old populations), the downward rate of transition t
 * gets the preconditioning term -W Psi* chi_t(old) U_t, and every other
 * transition t' active at the wavelength couples through -W Psi* chi_t U_t'.
 * I_eff comes from the sweep with the local source replaced by its
 * background part, and U_t - Psi* chi_t U_t = U_t [(1 - Lambda*) +
 * Lambda* (chi - chi_t)/chi] with chi - chi_t summed from the other
 * contributions: the same quantities without subtracting nearly equal
 * numbers in optically thick layers.  mode 1: plain rates with I from the
 * formal solution (Psi* = 0); mode 2: plain rates with each transition seeing
 * the Planck function (lines at their centre frequency, continua at the
 * actual frequency).  Collisions are always added. */
static void rate_matrix(const rho_ctx *c, int64_t col, work_t *w, const double *n, int mode)
{
    const atom_t *a = &c->at;
    int N = c->ndep, L = a->nlev;
    const double *T = c->T + col * N;
    double *G = w->Gam;
    memset(G, 0, sizeof(double) * N * L * L);
    if (a->nprd_line) {
        memset(w->Jp, 0, sizeof(double) * a->nlam * N);
        memset(w->Dp, 0, sizeof(double) * a->nlam * N);
        memset(w->Pup, 0, sizeof(double) * a->ntr * N);
        memset(w->Pdn, 0, sizeof(double) * a->ntr * N);
    }
    for (int64_t i = 0; i < a->nlam; ++i) {
        double nu = a->nu[i];
        int prd_pt = 0;
        for (int s = 0; s < a->nact[i]; ++s) prd_pt |= a->prd[a->act[i * MAXACT + s]];
        for (int m = 0; m < a->nmu; ++m)
            for (int d = 0; d < 2; ++d) {
                transition_coeffs(c, col, w, n, i, m, d);
                if (mode != 2) formal_ray(c, col, w, n, i, m, d);
                if (prd_pt && mode != 2) {
                    for (int k = 0; k < N; ++k) w->Jp[i * N + k] += 0.5 * a->wmu[m] * w->I[k];
                    memcpy(w->Iray + ((size_t)(m * 2 + d) * a->nlam + i) * N, w->I, sizeof(double) * N);
                    /* dI_k/drho_k = Psi*_k n_u U0_k of the PRD line (its emission
                     * is the only term of S that rho multiplies; stimulated
                     * emission in chi is left out of this derivative) */
                    for (int s = 0; s < a->nact[i]; ++s) {
                        int t = a->act[i * MAXACT + s];
                        if (!a->prd[t]) continue;
                        double *dr = w->Dray + ((size_t)(m * 2 + d) * a->nlam + i) * N;
                        for (int k = 0; k < N; ++k) {
                            dr[k] = (w->lam[k] / w->chi[k]) * n[a->tu[t] * N + k] * w->U0[s * N + k];
                            w->Dp[i * N + k] += 0.5 * a->wmu[m] * dr[k];
                        }
                    }
                }
                for (int k = 0; k < N; ++k) {
                    double psi = (mode == 0) ? w->lam[k] / w->chi[k] : 0.0;
                    double Ieff = (mode == 2) ? 0.0 : (mode == 0 ? w->Ieff[k] : w->I[k]);
                    double *Gk = G + (size_t)k * L * L;
                    for (int s = 0; s < a->nact[i]; ++s) {
                        int t = a->act[i * MAXACT + s], l = a->tl[t], u = a->tu[t];
                        double W = 4.0 * PI_D * a->wq[i * MAXACT + s] * (0.5 * a->wmu[m]) / (HPLANCK * nu);
                        double Ik = Ieff;
                        if (mode == 2) Ik = a->kind[t] == 0 ? rho_planck(a->nu0[t], T[k]) : w->Bnu[i * N + k];
                        double Ut = w->Ut[s * N + k];
                        double spont = Ut;
                        if (mode == 0) {
                            double other = w->chic[i * N + k];
                            for (int s2 = 0; s2 < a->nact[i]; ++s2)
                                if (s2 != s) other += w->chit[s2 * N + k];
                            spont = Ut * (w->omlam[k] + w->lam[k] * other / w->chi[k]);
                        }
                        Gk[u * L + l] += W * w->Vlu[s * N + k] * Ik;
                        Gk[l * L + u] += W * (spont + w->Vul[s * N + k] * Ik);
                        if (a->nprd_line && mode != 2) {
                            /* plain rates (actual intensity), for the PRD update */
                            w->Pup[(size_t)t * N + k] += W * w->Vlu[s * N + k] * w->I[k];
                            w->Pdn[(size_t)t * N + k] += W * (Ut + w->Vul[s * N + k] * w->I[k]);
                        }
                        if (psi != 0.0) {
                            for (int s2 = 0; s2 < a->nact[i]; ++s2) {
                                if (s2 == s) continue;
                                int t2 = a->act[i * MAXACT + s2], u2 = a->tu[t2];
                                double cc = W * psi * w->chit[s * N + k] * w->Ut[s2 * N + k];
                                if (l != u2) Gk[l * L + u2] -= cc;
                                if (u != u2) Gk[u * L + u2] += cc;
                            }
                        }
                    }
                }
            }
    }
    for (int k = 0; k < N; ++k) {
        double *Gk = G + (size_t)k * L * L;
        const double *Ck = w->C + (size_t)k * L * L;
        for (int p = 0; p < L; ++p)
            for (int q = 0; q < L; ++q)
                if (p != q) Gk[q * L + p] += Ck[p * L + q];
        for (int q = 0; q < L; ++q) {
            double s = 0.0;
            for (int p = 0; p < L; ++p)
                if (p != q) s += Gk[p * L + q];
            Gk[q * L + q] = -s;
        }
    }
}

/* Solve A x = b (L x L) by Gaussian elimination with partial pivoting.
 * Returns nonzero if a pivot is zero. */
static int lu_solve(int L, double *A, double *b)
{
    for (int p = 0; p < L; ++p) {
        int piv = p;
        for (int r = p + 1; r < L; ++r)
            if (fabs(A[r * L + p]) > fabs(A[piv * L + p])) piv = r;
        if (A[piv * L + p] == 0.0) return 1;
        if (piv != p) {
            for (int q = 0; q < L; ++q) {
                double tmp = A[p * L + q]; A[p * L + q] = A[piv * L + q]; A[piv * L + q] = tmp;
            }
            double tb = b[p]; b[p] = b[piv]; b[piv] = tb;
        }
        for (int r = p + 1; r < L; ++r) {
            double f = A[r * L + p] / A[p * L + p];
            for (int q = p; q < L; ++q) A[r * L + q] -= f * A[p * L + q];
            b[r] -= f * b[p];
        }
    }
    for (int p = L - 1; p >= 0; --p) {
        double s = b[p];
        for (int q = p + 1; q < L; ++q) s -= A[p * L + q] * b[q];
        b[p] = s / A[p * L + p];
    }
    return 0;
}

/* statistical equilibrium at every depth: the row of the most populated
 * level (old populations) is replaced by particle conservation sum n = n_H.
 * The unknowns are scaled by the old populations (y = n / n_old) and every
 * row by its largest entry before elimination: populations of one depth span
 * up to ~20 decades, and the scaling keeps the small ones accurate (it does
 * not change the exact solution). */
static int stateq(const rho_ctx *c, int64_t col, work_t *w, const double *nold, double *nnew)
{
    int N = c->ndep, L = c->at.nlev;
    for (int k = 0; k < N; ++k) {
        double A[MAXLEV * MAXLEV], b[MAXLEV], s[MAXLEV];
        memcpy(A, w->Gam + (size_t)k * L * L, sizeof(double) * L * L);
        int r = 0;
        for (int l = 0; l < L; ++l) {
            s[l] = nold[l * N + k];
            if (s[l] > s[r]) r = l;
        }
        for (int q = 0; q < L; ++q) A[r * L + q] = 1.0;
        for (int l = 0; l < L; ++l) b[l] = 0.0;
        b[r] = c->nH[col * N + k];
        for (int p = 0; p < L; ++p) {
            double mx = 0.0;
            for (int q = 0; q < L; ++q) {
                A[p * L + q] *= s[q];
                if (fabs(A[p * L + q]) > mx) mx = fabs(A[p * L + q]);
            }
            if (!(mx > 0)) return ST_SINGULAR;
            for (int q = 0; q < L; ++q) A[p * L + q] /= mx;
            b[p] /= mx;
        }
        if (lu_solve(L, A, b)) return ST_SINGULAR;
        for (int l = 0; l < L; ++l) nnew[l * N + k] = b[l] * s[l];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Start solutions other than LTE (Sect. 2.3: "LTE populations, zero
 * radiation, and ... escape probability iterations").
 *
 * Rate matrix with the radiation field replaced by zero: no radiative
 * excitation or ionisation; radiative de-excitation is spontaneous only --
 * A_ul for a line, and for a continuum the spontaneous recombination
 * 4 pi sum_lambda w_lambda (2 h nu^3/c^2) alpha(nu) (n*_l/n*_c) e^{-h nu/kT} / (h nu)
 * over the continuum's own quadrature weights.  esc[t * N + k] multiplies the
 * spontaneous rate of transition t at depth k (NULL: 1, zero radiation; the
 * escape probability for the escape-probability start, where it is the net
 * radiative bracket).  Collisions are added as in rate_matrix. */
static void spont_rate_matrix(const rho_ctx *c, int64_t col, work_t *w, const double *esc)
{
    const atom_t *a = &c->at;
    int N = c->ndep, L = a->nlev;
    double *G = w->Gam;
    memset(G, 0, sizeof(double) * N * L * L);
    for (int t = 0; t < a->ntr; ++t) {
        int l = a->tl[t], u = a->tu[t];
        for (int k = 0; k < N; ++k) {
            double R;
            if (a->kind[t] == 0) {
                R = a->A[t];
            } else {
                double G_lu = c->nstar[((size_t)col * L + l) * N + k] / c->nstar[((size_t)col * L + u) * N + k];
                R = 0.0;
                for (int64_t i = 0; i < a->nlam; ++i)
                    for (int s2 = 0; s2 < a->nact[i]; ++s2) {
                        if (a->act[i * MAXACT + s2] != t) continue;
                        double nu = a->nu[i], r = a->nu0[t] / nu;
                        double alpha = a->alpha0[t] * r * r * r;
                        double tw = 2.0 * HPLANCK * nu * nu * nu / (CLIGHT * CLIGHT);
                        R += 4.0 * PI_D * a->wq[i * MAXACT + s2] * tw * alpha * G_lu * w->ex[i * N + k] / (HPLANCK * nu);
                    }
            }
            if (esc) R *= esc[(size_t)t * N + k];
            G[(size_t)k * L * L + l * L + u] += R;
        }
    }
    for (int k = 0; k < N; ++k) {
        double *Gk = G + (size_t)k * L * L;
        const double *Ck = w->C + (size_t)k * L * L;
        for (int p = 0; p < L; ++p)
            for (int q = 0; q < L; ++q)
                if (p != q) Gk[q * L + p] += Ck[p * L + q];
        for (int q = 0; q < L; ++q) {
            double sum = 0.0;
            for (int p = 0; p < L; ++p)
                if (p != q) sum += Gk[p * L + q];
            Gk[q * L + q] = -sum;
        }
    }
}

/* Escape probability of every transition at every depth for populations n:
 * the line-centre (Doppler core, phi_0 = 1/(sqrt(pi) dnu_D)) or edge opacity
 * chi_0 = (n_l - n_u g_l/g_u) (h nu0/4 pi) B_lu phi_0, resp. (n_l - n_u
 * (n*_l/n*_u) e^{-h nu0/kT}) alpha0, clipped at zero; its optical depth
 * from the top tau(k) by the trapezoid rule along z; and the probability of
 * escape through the top of a semi-infinite atmosphere, averaged over
 * directions, p = beta(tau)/2 with beta(tau) = (1 - e^{-tau})/tau (the
 * single-flight escape probability; beta(0) = 1). */
static void escape_probabilities(const rho_ctx *c, int64_t col, const work_t *w, const double *n, double *esc)
{
    const atom_t *a = &c->at;
    int N = c->ndep, L = a->nlev;
    const double *T = c->T + col * N;
    for (int t = 0; t < a->ntr; ++t) {
        int l = a->tl[t], u = a->tu[t];
        double tau = 0.0, chip = 0.0;
        for (int k = 0; k < N; ++k) {
            double chi;
            if (a->kind[t] == 0) {
                double dnuD = a->nu0[t] / CLIGHT * sqrt(2.0 * KBOLTZ * T[k] / a->mass);
                chi = (n[l * N + k] - n[u * N + k] * a->g[l] / a->g[u]) * HPLANCK * a->nu0[t] / (4.0 * PI_D) *
                      a->Blu[t] / (sqrt(PI_D) * dnuD);
            } else {
                double G_lu = c->nstar[((size_t)col * L + l) * N + k] / c->nstar[((size_t)col * L + u) * N + k];
                chi = (n[l * N + k] - n[u * N + k] * G_lu * exp(-HPLANCK * a->nu0[t] / (KBOLTZ * T[k]))) * a->alpha0[t];
            }
            if (chi < 0.0) chi = 0.0;
            if (k > 0) tau += 0.5 * (chi + chip) * w->dz[k - 1];
            chip = chi;
            double beta = tau > 0.0 ? -expm1(-tau) / tau : 1.0;
            esc[(size_t)t * N + k] = 0.5 * beta;
        }
    }
}

#define EP_ITERATIONS 3

/* Start populations of one column: kind 3 zero radiation (one solve of the
 * spontaneous-only rate equations, row choice and scaling from n*); kind 4
 * escape probability (from LTE, EP_ITERATIONS solves, each with the escape
 * probabilities of the previous populations).  Requires column_setup. */
static int start_column(const rho_ctx *c, int64_t col, work_t *w, int kind, double *n)
{
    const atom_t *a = &c->at;
    int N = c->ndep, L = a->nlev;
    size_t nv = (size_t)L * N;
    memcpy(n, c->nstar + (size_t)col * nv, nv * 8);
    double *nn = malloc(nv * 8), *esc = malloc((size_t)a->ntr * N * 8);
    int st = 0;
    int nit = kind == 3 ? 1 : EP_ITERATIONS;
    for (int it = 0; it < nit && !st; ++it) {
        if (kind == 4) escape_probabilities(c, col, w, n, esc);
        spont_rate_matrix(c, col, w, kind == 4 ? esc : NULL);
        st = stateq(c, col, w, n, nn);
        if (!st) memcpy(n, nn, nv * 8);
    }
    free(nn);
    free(esc);
    return st;
}

/* Ng (1974) acceleration of order 2 in the formulation of Auer (1987):
 * x0 newest .. x3 oldest; minimise |d0 - a(d0 - d1) - b(d0 - d2)|_w with
 * d_j = x_j - x_{j+1}; return (1-a-b) x0 + a x1 + b x2.  Weights: uniform
 * (used by the iterations) or relative (1/x0^2).  The paper gives no
 * weights; relative weights made the extrapolation stall on hot columns and
 * diverge on the two-level problem, uniform weights converged all of them.
 * Returns nonzero if the 2x2 normal equations are singular. */
static int ng2_w(int64_t n, const double *x0, const double *x1, const double *x2, const double *x3,
                 double *out, int relative)
{
    double A11 = 0, A12 = 0, A22 = 0, b1 = 0, b2 = 0;
    for (int64_t i = 0; i < n; ++i) {
        double wgt = relative ? 1.0 / (x0[i] * x0[i]) : 1.0;
        double d0 = x0[i] - x1[i], d1 = x1[i] - x2[i], d2 = x2[i] - x3[i];
        double p = d0 - d1, q = d0 - d2;
        A11 += wgt * p * p;
        A12 += wgt * p * q;
        A22 += wgt * q * q;
        b1 += wgt * d0 * p;
        b2 += wgt * d0 * q;
    }
    double det = A11 * A22 - A12 * A12;
    if (!(fabs(det) > 0) || !isfinite(det)) return 1;
    double ca = (b1 * A22 - b2 * A12) / det;
    double cb = (A11 * b2 - A12 * b1) / det;
    for (int64_t i = 0; i < n; ++i) out[i] = (1.0 - ca - cb) * x0[i] + ca * x1[i] + cb * x2[i];
    return 0;
}

int rho_ng2(int64_t n, const double *x0, const double *x1, const double *x2, const double *x3, double *out,
            int32_t relative)
{
    return ng2_w(n, x0, x1, x2, x3, out, relative);
}

/* ------------------------------------------------------------------ */
/* One column: MALI iterations with Ng acceleration until
 * max |dn/n| < tol (Sect. 2.3) or maxiter formal solutions. */
static void iterate_column(rho_ctx *c, int64_t col, const rho_iter_opts *o, work_t *w, double *pts_out)
{
    const atom_t *a = &c->at;
    int N = c->ndep, L = a->nlev;
    size_t nv = (size_t)L * N;
    double *n = c->pops + (size_t)col * nv;
    double *nnew = malloc(nv * 8), *Cbase = malloc(sizeof(double) * N * L * L);
    column_setup(c, col, w);
    w->hybrid = o->prd_hybrid != 0;
    w->bezier = o->formal == 1;
    w->vz = c->vz + col * N;
    memcpy(Cbase, w->C, sizeof(double) * N * L * L);
    if (o->start == 0)
        memcpy(n, c->nstar + (size_t)col * nv, nv * 8);
    int hcount = 0, rcount = 0, it = 0, status = ST_MAXITER;
    size_t nrv = 0;   /* length of the rho vector (PRD points x depths) */
    for (int q = 0; q < a->nprd_line; ++q) nrv += (size_t)a->prd_np[q] * N;
    double dmax = INFINITY;
    for (int64_t q = 0; q < a->nlam * N; ++q) w->rho[q] = 1.0;   /* PRD starts as CRD */
    if (o->start == 3 || o->start == 4) {
        int st0 = start_column(c, col, w, o->start, n);
        if (st0) {
            c->iters[col] = 0;
            c->status[col] = (uint8_t)st0;
            c->dmax[col] = dmax;
            *pts_out = 0.0;
            free(nnew);
            free(Cbase);
            return;
        }
    }
    for (it = 1; it <= o->maxiter; ++it) {
        /* collisional-radiative switching (Hummer & Voels 1988) */
        double fcr = rho_crsw_factor(o->crsw_init, it);
        for (int q = 0; q < N * L * L; ++q) w->C[q] = Cbase[q] * fcr;
        rate_matrix(c, col, w, n, 0);
        int st = stateq(c, col, w, n, nnew);
        if (st) { status = st; break; }
        dmax = 0.0;
        int bad = 0;
        for (size_t q = 0; q < nv; ++q) {
            if (!(isfinite(nnew[q]) && nnew[q] > 0)) { bad = 1; break; }
            double dd = fabs(nnew[q] - n[q]) / nnew[q];
            if (dd > dmax) dmax = dd;
        }
        if (bad) { status = ST_NONFINITE; break; }
        int converged = dmax < o->tol && fcr == 1.0;
        /* Ng history (newest first) */
        memmove(w->hist + nv, w->hist, 3 * nv * 8);
        memcpy(w->hist, nnew, nv * 8);
        if (hcount < 4) ++hcount;
        if (!converged && o->ng_order == 2 && it >= o->ng_delay && hcount >= 4 &&
            (it - o->ng_delay) % o->ng_period == 0) {
            double *acc = malloc(nv * 8);
            if (!ng2_w(nv, w->hist, w->hist + nv, w->hist + 2 * nv, w->hist + 3 * nv, acc, 0)) {
                int ok = 1;
                for (size_t q = 0; q < nv; ++q)
                    if (!(isfinite(acc[q]) && acc[q] > 0)) { ok = 0; break; }
                if (ok) {
                    memcpy(nnew, acc, nv * 8);
                    memcpy(w->hist, acc, nv * 8);
                    hcount = 1;
                }
            }
            free(acc);
        }
        memcpy(n, nnew, nv * 8);
        if (converged) { status = ST_CONV; break; }
        if (a->nprd_line) {
            prd_update(c, col, w, n, it + 1, o->prd_eps0, o->ng_order == 2);
            /* Ng acceleration of the PRD iterations (Sect. 2.3), on the rho
             * vector with its own history and the populations' schedule; an
             * extrapolation with a negative rho is rejected */
            memmove(w->rhist + nrv, w->rhist, 3 * nrv * 8);
            rho_vector(a, N, w->rho, w->rhist, 0);
            if (rcount < 4) ++rcount;
            if (o->ng_order == 2 && it >= o->ng_delay && rcount >= 4 && (it - o->ng_delay) % o->ng_period == 0) {
                double *acc = malloc(nrv * 8);
                if (!ng2_w(nrv, w->rhist, w->rhist + nrv, w->rhist + 2 * nrv, w->rhist + 3 * nrv, acc, 0)) {
                    int ok = 1;
                    for (size_t q = 0; q < nrv; ++q)
                        if (!(isfinite(acc[q]) && acc[q] >= 0.0)) { ok = 0; break; }
                    if (ok) {
                        memcpy(w->rhist, acc, nrv * 8);
                        rho_vector(a, N, w->rho, acc, 1);
                        rcount = 1;
                    }
                }
                free(acc);
            }
        }
    }
    if (it > o->maxiter) it = o->maxiter;
    c->iters[col] = it;
    c->status[col] = (uint8_t)status;
    c->dmax[col] = dmax;
    *pts_out = (double)it * N * a->nlam * a->nmu;
    memcpy(w->C, Cbase, sizeof(double) * N * L * L);
    free(nnew);
    free(Cbase);
}

typedef struct {
    rho_ctx *c;
    const rho_iter_opts *o;
    int64_t next;
    pthread_mutex_t mu;
    double pts;
} pool_t;

static void *pool_worker(void *arg)
{
    pool_t *p = arg;
    work_t w;
    work_alloc(&w, &p->c->at, p->c->ndep);
    double pts = 0.0;
    for (;;) {
        pthread_mutex_lock(&p->mu);
        int64_t col = p->next++;
        pthread_mutex_unlock(&p->mu);
        if (col >= p->c->ncol) break;
        double pc = 0.0;
        iterate_column(p->c, col, p->o, &w, &pc);
        pts += pc;
    }
    pthread_mutex_lock(&p->mu);
    p->pts += pts;
    pthread_mutex_unlock(&p->mu);
    work_free(&w);
    return NULL;
}

/* Pool mode (Sect. 3.1): worker threads pull columns from a shared counter. */
int rho_iterate(rho_ctx *c, const rho_iter_opts *o, rho_iter_stats *st, int32_t nthreads)
{
    if (!c->ncol) return fail(c, "no columns loaded"), 4;
    if (o->maxiter < 1 || !(o->tol >= 0)) return fail(c, "invalid iteration options");
    if (o->ng_order != 0 && o->ng_order != 2) return fail(c, "ng_order must be 0 or 2");
    if (o->ng_order == 2 && (o->ng_period < 1 || o->ng_delay < 0)) return fail(c, "invalid Ng schedule");
    if (o->formal != 0 && o->formal != 1) return fail(c, "formal must be 0 (linear) or 1 (Bezier)");
    if (nthreads < 1) nthreads = 1;
    struct timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    prd_cache_build(c, nthreads);
    pool_t p = {c, o, 0, PTHREAD_MUTEX_INITIALIZER, 0.0};
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, pool_worker, &p);
    for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
    free(th);
    clock_gettime(CLOCK_MONOTONIC, &t1);
    if (st) {
        memset(st, 0, sizeof *st);
        st->seconds = (t1.tv_sec - t0.tv_sec) + 1e-9 * (t1.tv_nsec - t0.tv_nsec);
        st->pts = p.pts;
        for (int64_t col = 0; col < c->ncol; ++col) {
            if (c->status[col] == ST_CONV) st->n_converged++;
            else if (c->status[col] == ST_MAXITER) st->n_maxiter++;
            else st->n_failed++;
            st->iterations_total += c->iters[col];
            if (c->dmax[col] > st->max_dn_final || col == 0) st->max_dn_final = c->dmax[col];
        }
    }
    return 0;
}

/* Rate matrix of one column at given populations (see rate_matrix for modes
 * 0-2; mode 3 zero radiation, mode 4 escape probabilities from n; see
 * spont_rate_matrix); A_out is [ndep][nlev][nlev]. */
int rho_rate_matrix(rho_ctx *c, int64_t col, const double *n, int32_t mode, double *A_out)
{
    if (col < 0 || col >= c->ncol) return fail(c, "column out of range");
    work_t w;
    work_alloc(&w, &c->at, c->ndep);
    column_setup(c, col, &w);
    if (mode == 3) {
        spont_rate_matrix(c, col, &w, NULL);
    } else if (mode == 4) {
        double *esc = malloc((size_t)c->at.ntr * c->ndep * 8);
        escape_probabilities(c, col, &w, n, esc);
        spont_rate_matrix(c, col, &w, esc);
        free(esc);
    } else {
        rate_matrix(c, col, &w, n, mode);
    }
    memcpy(A_out, w.Gam, sizeof(double) * c->ndep * c->at.nlev * c->at.nlev);
    work_free(&w);
    return 0;
}

/* Start populations (kind 0 LTE, 3 zero radiation, 4 escape probability)
 * of every loaded column into the current populations; columns whose start
 * solve fails get status ST_SINGULAR (others ST_NOTRUN). */
int rho_start_populations(rho_ctx *c, int32_t kind)
{
    if (!c->ncol) return fail(c, "no columns loaded"), 4;
    if (kind != 0 && kind != 3 && kind != 4) return fail(c, "start kind must be 0, 3 or 4");
    const atom_t *a = &c->at;
    size_t nv = (size_t)a->nlev * c->ndep;
    work_t w;
    work_alloc(&w, a, c->ndep);
    for (int64_t col = 0; col < c->ncol; ++col) {
        double *n = c->pops + (size_t)col * nv;
        int st = 0;
        if (kind == 0) {
            memcpy(n, c->nstar + (size_t)col * nv, nv * 8);
        } else {
            column_setup(c, col, &w);
            st = start_column(c, col, &w, kind, n);
        }
        c->status[col] = (uint8_t)(st ? st : ST_NOTRUN);
    }
    work_free(&w);
    return 0;
}

/* redistribution kernel of PRD line q (in the order of the atom's PRD lines)
 * in column col, as the iteration builds it: *np_out = its points; with
 * non-NULL outputs also their grid indices pts_out[np] (frequency order),
 * quadrature weights w_out[np], K_out[N][np][np] and the J-bar weights
 * f_out[N][np] */
int rho_prd_kernel(rho_ctx *c, int64_t col, int32_t q, int32_t *np_out, int32_t *pts_out, double *w_out,
                   double *K_out, double *f_out)
{
    const atom_t *a = &c->at;
    if (col < 0 || col >= c->ncol) return fail(c, "column out of range");
    if (q < 0 || q >= a->nprd_line) return fail(c, "no such PRD line");
    const int m = a->prd_np[q], N = c->ndep;
    if (np_out) *np_out = m;
    if (!K_out && !f_out && !pts_out && !w_out) return 0;
    for (int j = 0; j < m; ++j) {
        if (pts_out) pts_out[j] = a->prd_pts[q][j];
        if (w_out) w_out[j] = a->prd_w[q][j];
    }
    work_t w;
    work_alloc(&w, a, N);
    column_setup(c, col, &w);
    if (K_out) memcpy(K_out, w.prdK[q], (size_t)N * m * m * sizeof(double));
    if (f_out) memcpy(f_out, w.prdf[q], (size_t)N * m * sizeof(double));
    work_free(&w);
    return 0;
}

/* background opacity chi_c[nlam][N] (m^-1) of column col on the wavelength
 * grid, as the iteration uses it: free-free, H- bound-free, stimulated
 * emission, Thomson scattering */
int rho_column_background(rho_ctx *c, int64_t col, double *chi_out)
{
    if (col < 0 || col >= c->ncol) return fail(c, "column out of range");
    work_t w;
    work_alloc(&w, &c->at, c->ndep);
    column_setup(c, col, &w);
    memcpy(chi_out, w.chic, sizeof(double) * c->at.nlam * c->ndep);
    work_free(&w);
    return 0;
}

/* One PRD update of line q in column col from rho = 1 with populations n
 * and the formal solution they give, the plain ratio before switching and
 * before the Jacobi step:
 * r_out[N][np] = 1 + F (sum_j K_ij J_j / Jbar - 1), points in frequency order */
int rho_prd_update_ratio(rho_ctx *c, int64_t col, const double *n, int32_t q, double *r_out)
{
    const atom_t *a = &c->at;
    if (col < 0 || col >= c->ncol) return fail(c, "column out of range");
    if (q < 0 || q >= a->nprd_line) return fail(c, "no such PRD line");
    const int N = c->ndep, m = a->prd_np[q];
    work_t w;
    work_alloc(&w, a, N);
    column_setup(c, col, &w);
    rate_matrix(c, col, &w, n, 1);
    prd_update(c, col, &w, n, 1, 0.0, 0);
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < m; ++j) r_out[(size_t)k * m + j] = w.rplain[(size_t)a->prd_pts[q][j] * N + k];
    work_free(&w);
    return 0;
}

/* escape probabilities esc[t][k] of one column for populations n */
int rho_escape_probabilities(rho_ctx *c, int64_t col, const double *n, double *esc_out)
{
    if (col < 0 || col >= c->ncol) return fail(c, "column out of range");
    work_t w;
    work_alloc(&w, &c->at, c->ndep);
    column_setup(c, col, &w);
    escape_probabilities(c, col, &w, n, esc_out);
    work_free(&w);
    return 0;
}

/* collisional rate matrix C[k][i][j] (i -> j) of one column */
int rho_collision_rates(rho_ctx *c, int64_t col, double *C_out)
{
    if (col < 0 || col >= c->ncol) return fail(c, "column out of range");
    int N = c->ndep, L = c->at.nlev;
    for (int k = 0; k < N; ++k) {
        double ns[MAXLEV];
        for (int l = 0; l < L; ++l) ns[l] = c->nstar[((size_t)col * L + l) * N + k];
        collision_rates(&c->at, c->T[col * N + k], c->ne[col * N + k], ns, C_out + (size_t)k * L * L);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Emergent intensity I(mu, nu) at the top for the current populations,
 * at arbitrary wavelengths (Sect. 2.2: vertical emergent spectrum). */
typedef struct {
    rho_ctx *c;
    double mu;
    int64_t nl;
    const double *lam;
    double *out;
    int64_t next;
    pthread_mutex_t m;
} spec_pool_t;

static void emergent_column(rho_ctx *c, int64_t col, double mu, int64_t nl, const double *lam, double *out)
{
    const atom_t *a = &c->at;
    int N = c->ndep, L = a->nlev;
    const double *z = c->z + col * N, *T = c->T + col * N, *vz = c->vz + col * N;
    const double *ne = c->ne + col * N, *np = c->np + col * N;
    const double *n = c->pops + (size_t)col * L * N;
    double *chi = malloc(N * 8), *S = malloc(N * 8), *dtau = malloc(N * 8), *I = malloc(N * 8), *lm = malloc(N * 8);
    double *B = malloc(N * 8);
    const double Cff = rho_cff();
    for (int64_t j = 0; j < nl; ++j) {
        double nu = CLIGHT / lam[j];
        for (int k = 0; k < N; ++k) {
            double x = HPLANCK * nu / (KBOLTZ * T[k]);
            B[k] = rho_planck(nu, T[k]);
            double nhm = hminus_density(c->nstar[((size_t)col * L + 0) * N + k], ne[k], T[k]);
            double ch = (Cff * ne[k] * np[k] / sqrt(T[k]) / (nu * nu * nu) + nhm * rho_hminus_sigma(lam[j]))
                        * (-expm1(-x)) + SIGMA_T * ne[k];
            double et = ch * B[k];
            for (int t = 0; t < a->ntr; ++t) {
                if (!(nu >= a->nu_lo[t] * (1 - 1e-13) && nu <= a->nu_hi[t] * (1 + 1e-13))) continue;
                int l = a->tl[t], u = a->tu[t];
                double Vlu, Vul, U;
                if (a->kind[t] == 0) {
                    double p = line_profile(a, t, nu, T[k], vz[k], mu, damping(a, t, k, N));
                    double h4 = HPLANCK * nu / (4.0 * PI_D);
                    Vlu = h4 * a->Blu[t] * p;
                    Vul = a->g[l] / a->g[u] * Vlu;
                    U = h4 * a->A[t] * p;
                } else {
                    double r = a->nu0[t] / nu;
                    double G = c->nstar[((size_t)col * L + l) * N + k] / c->nstar[((size_t)col * L + u) * N + k];
                    Vlu = a->alpha0[t] * r * r * r;
                    Vul = G * exp(-x) * Vlu;
                    U = 2.0 * HPLANCK * nu * nu * nu / (CLIGHT * CLIGHT) * Vul;
                }
                ch += n[l * N + k] * Vlu - n[u * N + k] * Vul;
                et += n[u * N + k] * U;
            }
            chi[k] = ch;
            S[k] = et / ch;
        }
        for (int k = 0; k < N - 1; ++k) dtau[k] = 0.5 * (chi[k] + chi[k + 1]) * fabs(z[k] - z[k + 1]) / mu;
        double dtv = 0.5 * (chi[N - 1] + chi[N - 2]) * fabs(z[N - 2] - z[N - 1]);
        rho_sc_sweep(N, dtau, S, B[N - 1] + mu * (B[N - 1] - B[N - 2]) / dtv, -1, I, lm);
        out[j] = I[0];
    }
    free(chi); free(S); free(dtau); free(I); free(lm); free(B);
}

static void *spec_worker(void *arg)
{
    spec_pool_t *p = arg;
    for (;;) {
        pthread_mutex_lock(&p->m);
        int64_t col = p->next++;
        pthread_mutex_unlock(&p->m);
        if (col >= p->c->ncol) break;
        emergent_column(p->c, col, p->mu, p->nl, p->lam, p->out + col * p->nl);
    }
    return NULL;
}

int rho_emergent_spectrum(rho_ctx *c, double mu, int64_t nl, const double *lam, double *out, int32_t nthreads)
{
    if (!(mu > 0 && mu <= 1)) return fail(c, "mu must be in (0, 1]");
    if (!c->ncol) return fail(c, "no columns loaded"), 4;
    for (int64_t j = 0; j < nl; ++j)
        if (!(lam[j] > 0)) return fail(c, "wavelengths must be positive");
    if (nthreads < 1) nthreads = 1;
    spec_pool_t p = {c, mu, nl, lam, out, 0, PTHREAD_MUTEX_INITIALIZER};
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, spec_worker, &p);
    for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
    free(th);
    return 0;
}

/* ================================================================== */
/* Two-level atom, complete redistribution (the textbook reduction of     */
/* MALI): S = (1 - eps) Jbar + eps B with the ALI update                   */
/* S_new = [(1-eps)(Jbar - Lstar S) + eps B] / [1 - (1-eps) Lstar].         */
/* Grid: line-centre optical depth tau0[k]; Doppler profile at x_f in      */
/* [-xmax, xmax]; trapezoid weights renormalised so sum w phi = 1;          */
/* tau_x = tau0 phi(x)/phi(0); no incident radiation at the top, I = B +    */
/* mu dB/dtau (= B here) at the bottom.                                    */
/* ================================================================== */

/* Jbar and Lambda-bar* for a given S */
/* ------------------------------------------------------------------ */
/* Polarised formal solution (NEXT: Zeeman Stokes spectra of one line).
 * dI/dtau = I - S_eff along the ray, tau measured with eta_I, S_eff = S - K' I,
 * K' = K/eta_I - 1 (zero diagonal), in the convention
 *     K = [[eI, eQ, eU, eV], [eQ, eI, rV, -rU], [eU, -rV, eI, rQ], [eV, rU, -rQ, eI]]
 * (Landi Degl'Innocenti & Landolfi 2004).  DELO-linear (Rees, Durrant &
 * Murphy 1989): S_eff interpolated linearly on each interval, the local K'I
 * taken implicitly:
 *     (1 + w_o K'_o) I_o = e^{-dtau} I_u + w_u (S_u - K'_u I_u) + w_o S_o
 * with the weights of the scalar linear short characteristics (which it
 * reduces to when K' = 0).  Kp[k] = (eQ, eU, eV, rQ, rU, rV)/eI, S[k] the
 * emission vector / eI.  The ray starts at k = N-1 with Ib and ends at k = 0. */
static void kprime(const double *kp, double M[4][4])
{
    double eQ = kp[0], eU = kp[1], eV = kp[2], rQ = kp[3], rU = kp[4], rV = kp[5];
    double m[4][4] = {{0, eQ, eU, eV}, {eQ, 0, rV, -rU}, {eU, -rV, 0, rQ}, {eV, rU, -rQ, 0}};
    memcpy(M, m, sizeof m);
}

void rho_stokes_sweep(int N, const double *dtau, const double *Kp, const double *S, const double *Ib, double *Itop)
{
    double I[4];
    memcpy(I, Ib, sizeof I);
    for (int k = N - 2; k >= 0; --k) {
        double ex, wu, wo, omwo;
        sc_step_weights(dtau[k], &ex, &wu, &wo, &omwo);
        double Mu[4][4], Mo[4][4];
        kprime(Kp + (size_t)(k + 1) * 6, Mu);
        kprime(Kp + (size_t)k * 6, Mo);
        double rhs[4], A[16];
        for (int i = 0; i < 4; ++i) {
            double ku = 0.0;
            for (int j = 0; j < 4; ++j) ku += Mu[i][j] * I[j];
            rhs[i] = ex * I[i] + wu * (S[(size_t)(k + 1) * 4 + i] - ku) + wo * S[(size_t)k * 4 + i];
            for (int j = 0; j < 4; ++j) A[i * 4 + j] = (i == j ? 1.0 : 0.0) + wo * Mo[i][j];
        }
        lu_solve(4, A, rhs);
        memcpy(I, rhs, sizeof I);
    }
    memcpy(Itop, I, sizeof I);
}

/* Emergent Stokes vector at mu = 1 (vertical ray) of one column for line t
 * with Zeeman splitting (normal triplet of effective Lande factor g_eff):
 * sigma_b / pi / sigma_r profiles H(a, v - v_B), H(a, v), H(a, v + v_B) and
 * dispersion profiles L likewise, v = (nu - nu0)/dnu_D - v_z/v_th,
 * v_B = g_eff e B/(4 pi m_e) / dnu_D; field strength B [T], inclination
 * theta to the vertical and azimuth chi per depth.
 *   eI = chi_c + chi_others + (k_l/2)[p sin^2 th + (b + r)(1 + cos^2 th)/2]
 *   eQ = (k_l/2)[p - (b + r)/2] sin^2 th cos 2chi, eU likewise with sin 2chi,
 *   eV = (k_l/2)(r - b) cos th,  rQ, rU, rV the same with the dispersion
 *   profiles, k_l = (n_l B_lu - n_u B_ul) h nu/(4 pi) / (sqrt(pi) dnu_D);
 * emission: background and the other transitions unpolarised, the line
 * S_l (eI_l, eQ, eU, eV) with S_l = n_u A_ul/(n_l B_lu - n_u B_ul) (no atomic
 * polarisation; the same profile for absorption and emission).  Bottom: I =
 * B + dB/dtau (diffusion), Q = U = V = 0. */
static void emergent_stokes_column(rho_ctx *c, int64_t col, int t0, double geff, const double *Bf, const double *th,
                                   const double *az, int64_t nl, const double *lam, double *out)
{
    const atom_t *a = &c->at;
    int N = c->ndep, L = a->nlev;
    const double *z = c->z + col * N, *T = c->T + col * N, *vz = c->vz + col * N;
    const double *ne = c->ne + col * N, *np = c->np + col * N;
    const double *n = c->pops + (size_t)col * L * N;
    double *Kp = malloc((size_t)N * 6 * 8), *Sv = malloc((size_t)N * 4 * 8), *eI = malloc(N * 8);
    double *dtau = malloc(N * 8), *B = malloc(N * 8);
    const double Cff = rho_cff();
    int l0 = a->tl[t0], u0 = a->tu[t0];
    for (int64_t j = 0; j < nl; ++j) {
        double nu = CLIGHT / lam[j];
        for (int k = 0; k < N; ++k) {
            double x = HPLANCK * nu / (KBOLTZ * T[k]);
            B[k] = rho_planck(nu, T[k]);
            double nhm = hminus_density(c->nstar[((size_t)col * L + 0) * N + k], ne[k], T[k]);
            double ch = (Cff * ne[k] * np[k] / sqrt(T[k]) / (nu * nu * nu) + nhm * rho_hminus_sigma(lam[j]))
                        * (-expm1(-x)) + SIGMA_T * ne[k];
            double et = ch * B[k];
            for (int t = 0; t < a->ntr; ++t) {
                if (t == t0) continue;
                if (!(nu >= a->nu_lo[t] * (1 - 1e-13) && nu <= a->nu_hi[t] * (1 + 1e-13))) continue;
                int l = a->tl[t], u = a->tu[t];
                double Vlu, Vul, U;
                if (a->kind[t] == 0) {
                    double p = line_profile(a, t, nu, T[k], vz[k], 1.0, damping(a, t, k, N));
                    double h4 = HPLANCK * nu / (4.0 * PI_D);
                    Vlu = h4 * a->Blu[t] * p;
                    Vul = a->g[l] / a->g[u] * Vlu;
                    U = h4 * a->A[t] * p;
                } else {
                    double r = a->nu0[t] / nu;
                    double G = c->nstar[((size_t)col * L + l) * N + k] / c->nstar[((size_t)col * L + u) * N + k];
                    Vlu = a->alpha0[t] * r * r * r;
                    Vul = G * exp(-x) * Vlu;
                    U = 2.0 * HPLANCK * nu * nu * nu / (CLIGHT * CLIGHT) * Vul;
                }
                ch += n[l * N + k] * Vlu - n[u * N + k] * Vul;
                et += n[u * N + k] * U;
            }
            /* the polarised line */
            double vth = sqrt(2.0 * KBOLTZ * T[k] / a->mass);
            double dnuD = a->nu0[t0] * vth / CLIGHT;
            double v = (nu - a->nu0[t0]) / dnuD - vz[k] / vth;
            double vB = geff * QELEC * Bf[k] / (4.0 * PI_D * MELEC) / dnuD;
            double ad = damping(a, t0, k, N);
            double Hb, Lb, Hp, Lp, Hr, Lr;
            rho_faddeeva(ad, v - vB, &Hb, &Lb);
            rho_faddeeva(ad, v, &Hp, &Lp);
            rho_faddeeva(ad, v + vB, &Hr, &Lr);
            double h4 = HPLANCK * nu / (4.0 * PI_D);
            double kl = (n[l0 * N + k] * a->Blu[t0] - n[u0 * N + k] * a->Bul[t0]) * h4 / (sqrt(PI_D) * dnuD);
            double Sl = n[u0 * N + k] * a->A[t0] / (n[l0 * N + k] * a->Blu[t0] - n[u0 * N + k] * a->Bul[t0]);
            double s2 = sin(th[k]) * sin(th[k]), ct = cos(th[k]), c2 = cos(2.0 * az[k]), sn2 = sin(2.0 * az[k]);
            double lI = 0.5 * kl * (Hp * s2 + 0.5 * (Hb + Hr) * (1.0 + ct * ct));
            double lq = 0.5 * kl * (Hp - 0.5 * (Hb + Hr)) * s2;
            double lV = 0.5 * kl * (Hr - Hb) * ct;
            double rq = 0.5 * kl * (Lp - 0.5 * (Lb + Lr)) * s2;
            double rV = 0.5 * kl * (Lr - Lb) * ct;
            double etaI = ch + lI;
            eI[k] = etaI;
            double e[6] = {lq * c2, lq * sn2, lV, rq * c2, rq * sn2, rV};
            for (int i = 0; i < 6; ++i) Kp[(size_t)k * 6 + i] = e[i] / etaI;
            Sv[(size_t)k * 4 + 0] = (et + Sl * lI) / etaI;
            Sv[(size_t)k * 4 + 1] = Sl * e[0] / etaI;
            Sv[(size_t)k * 4 + 2] = Sl * e[1] / etaI;
            Sv[(size_t)k * 4 + 3] = Sl * e[2] / etaI;
        }
        for (int k = 0; k < N - 1; ++k) dtau[k] = 0.5 * (eI[k] + eI[k + 1]) * fabs(z[k] - z[k + 1]);
        double dtv = 0.5 * (eI[N - 1] + eI[N - 2]) * fabs(z[N - 2] - z[N - 1]);
        double Ib[4] = {B[N - 1] + (B[N - 1] - B[N - 2]) / dtv, 0.0, 0.0, 0.0};
        rho_stokes_sweep(N, dtau, Kp, Sv, Ib, out + (size_t)j * 4);
    }
    free(Kp); free(Sv); free(eI); free(dtau); free(B);
}

/* Stokes I, Q, U, V at mu = 1 for line `line` (index among the lines),
 * out [ncol][nl][4]; B_T, theta, chi [ncol][ndep]. */
int rho_emergent_stokes(rho_ctx *c, int32_t line, double geff, const double *B_T, const double *theta,
                        const double *chi, int64_t nl, const double *lam, double *out)
{
    if (line < 0 || line >= c->at.nline) return fail(c, "line index out of range");
    for (int64_t col = 0; col < c->ncol; ++col)
        emergent_stokes_column(c, col, line, geff, B_T + col * c->ndep, theta + col * c->ndep, chi + col * c->ndep,
                               nl, lam, out + (size_t)col * nl * 4);
    return 0;
}

int rho_two_level_jbar(int N, const double *tau0, int nfreq, double xmax, int nmu, double B,
                       const double *S, double *Jbar, double *Lstar)
{
    if (N < 2 || nfreq < 2 || nmu < 1 || nmu > 16) return 1;
    double mu[16], wmu[16];
    gauss_legendre01(nmu, mu, wmu);
    double *x = malloc(nfreq * 8), *wf = malloc(nfreq * 8), *phi = malloc(nfreq * 8);
    double norm = 0.0;
    for (int f = 0; f < nfreq; ++f) {
        x[f] = -xmax + 2.0 * xmax * f / (nfreq - 1);
        phi[f] = exp(-x[f] * x[f]) / sqrt(PI_D);
        double h = 2.0 * xmax / (nfreq - 1);
        wf[f] = (f == 0 || f == nfreq - 1) ? 0.5 * h : h;
        norm += wf[f] * phi[f];
    }
    for (int f = 0; f < nfreq; ++f) wf[f] /= norm;
    double *dt = malloc(N * 8), *I = malloc(N * 8), *lm = malloc(N * 8);
    for (int k = 0; k < N; ++k) Jbar[k] = Lstar[k] = 0.0;
    double phi0 = 1.0 / sqrt(PI_D);
    for (int f = 0; f < nfreq; ++f)
        for (int m = 0; m < nmu; ++m) {
            for (int k = 0; k < N - 1; ++k) dt[k] = (tau0[k + 1] - tau0[k]) * phi[f] / phi0 / mu[m];
            double wgt = wf[f] * phi[f] * 0.5 * wmu[m];
            rho_sc_sweep(N, dt, S, 0.0, +1, I, lm);
            for (int k = 0; k < N; ++k) { Jbar[k] += wgt * I[k]; Lstar[k] += wgt * lm[k]; }
            double dtv = (tau0[N - 1] - tau0[N - 2]) * phi[f] / phi0;
            (void)dtv;   /* isothermal: dB/dtau = 0, I = B at the bottom */
            rho_sc_sweep(N, dt, S, B, -1, I, lm);
            for (int k = 0; k < N; ++k) { Jbar[k] += wgt * I[k]; Lstar[k] += wgt * lm[k]; }
        }
    free(x); free(wf); free(phi); free(dt); free(I); free(lm);
    return 0;
}

int rho_two_level_solve(int N, const double *tau0, int nfreq, double xmax, int nmu, double eps,
                        double B, int maxiter, double tol, int ng_order, int ng_delay, int ng_period,
                        double *S, int32_t *iters_out)
{
    size_t nv = N;
    double *J = malloc(N * 8), *Ls = malloc(N * 8), *Sn = malloc(N * 8), *hist = malloc(4 * N * 8);
    for (int k = 0; k < N; ++k) S[k] = B;   /* LTE start */
    int hcount = 0, it;
    for (it = 1; it <= maxiter; ++it) {
        if (rho_two_level_jbar(N, tau0, nfreq, xmax, nmu, B, S, J, Ls)) { it = -1; break; }
        double dmax = 0.0;
        for (int k = 0; k < N; ++k) {
            Sn[k] = ((1.0 - eps) * (J[k] - Ls[k] * S[k]) + eps * B) / (1.0 - (1.0 - eps) * Ls[k]);
            double dd = fabs(Sn[k] - S[k]) / Sn[k];
            if (dd > dmax) dmax = dd;
        }
        memmove(hist + nv, hist, 3 * nv * 8);
        memcpy(hist, Sn, nv * 8);
        if (hcount < 4) ++hcount;
        int conv = dmax < tol;
        if (!conv && ng_order == 2 && it >= ng_delay && hcount >= 4 && (it - ng_delay) % ng_period == 0) {
            if (!ng2_w(nv, hist, hist + nv, hist + 2 * nv, hist + 3 * nv, Sn, 0)) {
                memcpy(hist, Sn, nv * 8);
                hcount = 1;
            } else {
                memcpy(Sn, hist, nv * 8);
            }
        }
        memcpy(S, Sn, nv * 8);
        if (conv) break;
    }
    if (iters_out) *iters_out = it > maxiter ? maxiter : it;
    free(J); free(Ls); free(Sn); free(hist);
    return 0;
}
