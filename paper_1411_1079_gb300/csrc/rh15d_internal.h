// rh15d_internal.h -- tables and device math shared by the translation units
// of librh15d_gpu.so (not part of the public ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rh15d.h"

#define RH_MAXLEV 8
#define RH_MAXTR 32
#define RH_KMAX 3          // transitions active in one 32-wavelength tile (union)
#define RH_MAXTILE 96      // 32-wavelength tiles of the grid
#define RH_MAXMU 16
#define RH_MAXMAP 2048
#define RH_NLANEF 7        // per-slot lane fields
#define RH_VT_N 1024       // Voigt coefficient table: intervals in t = 1/(1+|v|)
#define RH_MAXPRD 4        // lines in partial redistribution
#define RH_MAXPRDPT 1024   // wavelength points of all PRD lines together

namespace rh {

// SI constants (CODATA 2018; h, c, k, e exact)
constexpr double kH = 6.62607015e-34;
constexpr double kC = 2.99792458e8;
constexpr double kK = 1.380649e-23;
constexpr double kQ = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kSigmaT = 6.6524587321e-29;
constexpr double kERyd = 13.605693122994 * 1.602176634e-19;
constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.77245385090551602730;

struct DevTrans {
    int l, u, kind, sub;          // kind 0 line (sub = line index), 1 continuum (sub = continuum index)
    double nu0, A, Blu, Bul, alpha0, ln_atop, ln_abot, f;
};

struct DevTile {
    int K;                        // transitions in the union of the tile
    int t[RH_KMAX];
    int acc_off;                  // first accumulator of the tile (per depth)
    int m;                        // accumulators of the tile = K (K + 1)
    int prd_slot;                 // slot j of a PRD line in the union, -1: none
    int pacc_off;                 // first plain-rate accumulator (2 per slot), PRD atoms only
    int phi[RH_KMAX];             // line slot: its row of the profile cache; -1: continuum
};

// Everything the column kernel needs about the atom, passed by value as a
// __grid_constant__ kernel parameter (read through the constant bank).
struct DevAtom {
    int nlev, ntr, nline, ncont, ntile, nmu, macc, nmap;
    double mass, metal_floor;
    double lev_chi[RH_MAXLEV];    // E_continuum - E_i, J (bound levels)
    double lev_g2[RH_MAXLEV];     // g_i / (2 g_continuum)
    double mu[RH_MAXMU], wmu[RH_MAXMU];
    float muf[RH_MAXMU], wm2f[RH_MAXMU];   // mu and w_mu / 2 for the FP32 sweep
    float imuf[RH_MAXMU];                    // 1/mu
    DevTrans tr[RH_MAXTR];
    DevTile tile[RH_MAXTILE];
    int16_t order[RH_MAXTILE];               // tile processing order (most expensive first)
    // accumulator -> rate-matrix entry map: A[row][col] += sign * acc
    int16_t map_acc[RH_MAXMAP];
    int8_t map_row[RH_MAXMAP], map_col[RH_MAXMAP], map_sign[RH_MAXMAP];
    // partial redistribution: PRD lines, their points (offsets into the point
    // arrays, frequency order) and redistribution-kernel blocks (offsets, np^2)
    int nprd, npp, pacc;
    int prd_t[RH_MAXPRD];
    int prd_off[RH_MAXPRD + 1];
    int prd_koff[RH_MAXPRD + 1];
    // profile cache: rows of line slots (tile, slot) whose Voigt profiles for
    // every ray and depth the column kernel keeps per column in global scratch
    int nphi;
    int16_t phi_tile[RH_MAXTILE * RH_KMAX];
    int8_t phi_j[RH_MAXTILE * RH_KMAX];
};

// Lane-table fields (structure of arrays, [field][npad]); per-slot fields are
// [RH_NLANEF * s + f].  Population-proportional quantities are scaled so that
// they stay inside the FP32 range: populations enter the sweep divided by
// n_ref, hence V and U carry a factor n_ref.
//   f = 0 c   : up-rate coefficient  (lines w B_lu; continua 4 pi w alpha / (h nu))
//   f = 1 Vc  : n_ref * V_lu without profile (lines h nu/4pi B_lu; continua alpha)
//   f = 2 Uc  : n_ref * U without profile / depth factor (lines h nu/4pi A;
//               continua 2 h nu^3/c^2 alpha)
//   f = 3 E   : A/B_ul-type constant (lines 2 h nu0^3/c^2; continua 2 h nu^3/c^2)
//   f = 4 q   : Doppler offset c (nu/nu0 - 1) [m/s] (lines)
//   f = 5 pn  : profile normalisation c / (sqrt(pi) nu0) (lines)
//   f = 6 grat: g_l/g_u (lines) -- the continua use G(k) exp(-h nu/kT)
// then four per-lane fields: nu, sigma(H-), (1e15/nu)^3, 2 h nu^3/c^2.
constexpr int kLaneSlotFields = RH_NLANEF;
constexpr int kLaneNu = RH_NLANEF * RH_KMAX;
constexpr int kLaneHm = kLaneNu + 1;
constexpr int kLaneNu3 = kLaneNu + 2;
constexpr int kLaneTw = kLaneNu + 3;
constexpr int kLaneFields = kLaneNu + 4;
constexpr double kNuRef3 = 1e45;   // (1e15 Hz)^3: free-free coefficient scale

// ----------------------------------------------------------------------------
// Voigt function H(a, v), FP64 (FP64 path and table set-up).
// |v| < 6: Taylor expansion of w(v + i a) in the damping a about the real
// axis, w(v) = exp(-v^2) + (2i/sqrt(pi)) F(v) with Dawson's integral F from
// its positive power series F(v) = exp(-v^2) sum v^{2n+1} / (n! (2n+1)), and
// the derivatives from w' = -2 z w + 2i/sqrt(pi), w^{(n+1)} = -2 z w^{(n)} -
// 2 n w^{(n-1)} (order 9; a <= 0.05).  |v| >= 6: w(z) ~ exp(-z^2) +
// (i / (sqrt(pi) z)) sum_k (2k-1)!! / (2 z^2)^k, 36 terms.  ~1e-13 relative.
__host__ __device__ inline double dawson_series(double x)
{
    double s = 0.0, term = x, x2 = x * x;
    for (int n = 0; n < 400; ++n) {
        double t = term / (2 * n + 1);
        s += t;
        if (t <= 1e-17 * s) break;
        term *= x2 / (n + 1);
    }
    return exp(-x2) * s;
}

__host__ __device__ inline double voigt_f64(double a, double v)
{
    double av = fabs(v);
    if (av < 6.0) {
        // w and derivatives at the real point v (complex as re/im pairs)
        double e = exp(-av * av);
        double F = dawson_series(av);
        double wr[10], wi[10];
        wr[0] = e;
        wi[0] = 2.0 / kSqrtPi * F;
        wr[1] = -2.0 * av * wr[0];
        wi[1] = -2.0 * av * wi[0] + 2.0 / kSqrtPi;
        for (int n = 1; n < 9; ++n) {
            wr[n + 1] = -2.0 * (av * wr[n] + n * wr[n - 1]);
            wi[n + 1] = -2.0 * (av * wi[n] + n * wi[n - 1]);
        }
        // sum_n (i a)^n / n! w^{(n)}: real part
        double h = 0.0, pw = 1.0;
        for (int n = 0; n <= 9; ++n) {
            switch (n & 3) {
            case 0: h += pw * wr[n]; break;
            case 1: h -= pw * wi[n]; break;
            case 2: h -= pw * wr[n]; break;
            default: h += pw * wi[n]; break;
            }
            pw *= a / (n + 1);
        }
        return h;
    }
    // asymptotic: z = av + i a; w = exp(-z^2) + (i/(sqrt(pi) z)) S,
    // S = sum t_k, t_{k+1} = t_k (2k+1)/(2 z^2)
    double zr = av, zi = a;
    double z2r = 2.0 * (zr * zr - zi * zi), z2i = 2.0 * (2.0 * zr * zi);
    double d = z2r * z2r + z2i * z2i;
    double ir = z2r / d, ii = -z2i / d;   // 1/(2 z^2)
    double sr = 0.0, si = 0.0, tr = 1.0, ti = 0.0;
    for (int k = 0; k <= 36; ++k) {
        sr += tr;
        si += ti;
        double nr = (tr * ir - ti * ii) * (2 * k + 1), ni = (tr * ii + ti * ir) * (2 * k + 1);
        tr = nr;
        ti = ni;
    }
    // Re[i S conj(z)] / (sqrt(pi)|z|^2) with i S = (-si) + i sr
    double mz = zr * zr + zi * zi;
    return (-si * zr + sr * zi) / (kSqrtPi * mz) + exp(zi * zi - zr * zr) * cos(2.0 * zr * zi);
}

// Faddeeva function w(v + i a) = H + i L, FP64, by the same two branches as
// voigt_f64 (Taylor expansion in a about the real axis for |v| < 6, the
// asymptotic series above); H is even and L odd in v.
__host__ __device__ inline void faddeeva_f64(double a, double v, double &H, double &L)
{
    double av = fabs(v), sg = v < 0.0 ? -1.0 : 1.0;
    if (av < 6.0) {
        double e = exp(-av * av);
        double F = dawson_series(av);
        double wr[10], wi[10];
        wr[0] = e;
        wi[0] = 2.0 / kSqrtPi * F;
        wr[1] = -2.0 * av * wr[0];
        wi[1] = -2.0 * av * wi[0] + 2.0 / kSqrtPi;
        for (int n = 1; n < 9; ++n) {
            wr[n + 1] = -2.0 * (av * wr[n] + n * wr[n - 1]);
            wi[n + 1] = -2.0 * (av * wi[n] + n * wi[n - 1]);
        }
        // sum_n (i a)^n / n! w^{(n)}: real and imaginary parts
        double h = 0.0, l = 0.0, pw = 1.0;
        for (int n = 0; n <= 9; ++n) {
            switch (n & 3) {
            case 0: h += pw * wr[n]; l += pw * wi[n]; break;
            case 1: h -= pw * wi[n]; l += pw * wr[n]; break;
            case 2: h -= pw * wr[n]; l -= pw * wi[n]; break;
            default: h += pw * wi[n]; l -= pw * wr[n]; break;
            }
            pw *= a / (n + 1);
        }
        H = h;
        L = sg * l;
        return;
    }
    double zr = av, zi = a;
    double z2r = 2.0 * (zr * zr - zi * zi), z2i = 2.0 * (2.0 * zr * zi);
    double d = z2r * z2r + z2i * z2i;
    double ir = z2r / d, ii = -z2i / d;
    double sr = 0.0, si = 0.0, tr = 1.0, ti = 0.0;
    for (int k = 0; k <= 36; ++k) {
        sr += tr;
        si += ti;
        double nr = (tr * ir - ti * ii) * (2 * k + 1), ni = (tr * ii + ti * ir) * (2 * k + 1);
        tr = nr;
        ti = ni;
    }
    // w = i S conj(z) / (sqrt(pi)|z|^2) + exp(-z^2)
    double mz = zr * zr + zi * zi, ez = exp(zi * zi - zr * zr);
    H = (-si * zr + sr * zi) / (kSqrtPi * mz) + ez * cos(2.0 * zr * zi);
    L = sg * ((sr * zr + si * zi) / (kSqrtPi * mz) - ez * sin(2.0 * zr * zi));
}

// Coefficients of the expansion of the dispersion function in the damping a
// used by the FP32 path: L(a, v) = L0 - (a^2/2) L2 - 2 a v e^{-v^2}
// + (a^3/6)(8 v^3 - 12 v) e^{-v^2} + O(a^4), L0 = (2/sqrt pi) F(v), L2 = L0''
// (F Dawson's integral: F' = 1 - 2vF, F'' = -2v + (4v^2 - 2)F, F''' = -2 + 8vF +
// (4v^2 - 2)F').  For v >= 8 from the asymptotic series F = sum_k c_k v^{-(2k+1)},
// c_k = (2k-1)!!/2^{k+1}, term by term (no cancellation).  Returns L0, L2 and
// their derivatives in v, for v >= 0.
__host__ inline void dispersion_coeffs(double v, double &l0, double &d0, double &l2, double &d2)
{
    const double k2 = 2.0 / kSqrtPi;
    if (v < 8.0) {
        double F = dawson_series(v), F1 = 1.0 - 2.0 * v * F;
        double F2 = -2.0 * v + (4.0 * v * v - 2.0) * F, F3 = -2.0 + 8.0 * v * F + (4.0 * v * v - 2.0) * F1;
        l0 = k2 * F;
        d0 = k2 * F1;
        l2 = k2 * F2;
        d2 = k2 * F3;
        return;
    }
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0, ck = 0.5, vp = 1.0 / v;   // c_0 v^{-1}
    const double iv2 = 1.0 / (v * v);
    for (int k = 0; k < 30; ++k) {
        const double n = 2.0 * k + 1.0;
        s0 += ck * vp;
        s1 -= n * ck * vp / v;
        s2 += n * (n + 1) * ck * vp * iv2;
        s3 -= n * (n + 1) * (n + 2) * ck * vp * iv2 / v;
        ck *= (2.0 * k + 1.0) / 2.0;
        vp *= iv2;
    }
    l0 = k2 * s0;
    d0 = k2 * s1;
    l2 = k2 * s2;
    d2 = k2 * s3;
}

// Dispersion function, FP32, branch-free: the expansion above with L0, L2
// from a cubic-Hermite table in t = 1/(1+|v|) (tab[i] = {L0, h dL0/dt, L2,
// h dL2/dt} at t_i = i h, h = 1/RH_VT_N); odd in v.
__device__ __forceinline__ float disp_f32(float a, float v, const float4 *__restrict__ tab);

// FP32 reciprocal for the sweep: the hardware approximation (rcp.approx, about
// 1 ulp, denormals flushed; no operand of the sweep is denormal) unless
// RH_RCP_APPROX is 0, then the correctly rounded __frcp_rn.
#ifndef RH_RCP_APPROX
#define RH_RCP_APPROX 1
#endif
__device__ __forceinline__ float rcp_f32(float x)
{
#if RH_RCP_APPROX
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return __frcp_rn(x);
#endif
}

// Coefficients of the expansion of H(a, v) in the damping a used by the FP32
// Voigt function: H = e^{-v^2}[1 + a^2(1 - 2v^2) + a^4(2v^4/3 - 2v^2 + 1/2)]
//                     + a H1(v) + a^3 H3(v),
// H1 = -(2/sqrt pi)(1 - 2vF), H3 = (4/(3 sqrt pi))(v^2 - 1 + vF(3 - 2v^2)),
// F Dawson's integral.  For v >= 8 both come from their asymptotic series
// (no cancellation): with u = 1/(2v^2), c_k = (2k-1)!!,
// H1 = (2/sqrt pi) sum_{k>=1} c_k u^k, H3 = (4/(3 sqrt pi)) sum_{j>=2} (1-j) c_j u^j.
// Returns H1, H3 and their derivatives in v.
__host__ inline void voigt_coeffs(double v, double &h1, double &d1, double &h3, double &d3)
{
    if (v < 8.0) {
        double F = dawson_series(v), Fp = 1.0 - 2.0 * v * F;
        h1 = -(2.0 / kSqrtPi) * Fp;
        d1 = (4.0 / kSqrtPi) * (F + v * Fp);
        h3 = (4.0 / (3.0 * kSqrtPi)) * (v * v - 1.0 + v * F * (3.0 - 2.0 * v * v));
        d3 = (4.0 / (3.0 * kSqrtPi)) * (2.0 * v + (F + v * Fp) * (3.0 - 2.0 * v * v) - 4.0 * v * v * F);
        return;
    }
    double u = 1.0 / (2.0 * v * v), du = -1.0 / (v * v * v);
    double s1 = 0, ds1 = 0, s3 = 0, ds3 = 0, ck = 1.0, uk = 1.0;   // c_0 u^0
    for (int k = 1; k <= 40; ++k) {
        ck *= (2 * k - 1);
        double ukm1 = uk;
        uk *= u;
        s1 += ck * uk;
        ds1 += k * ck * ukm1;
        if (k >= 2) {
            s3 += (1 - k) * ck * uk;
            ds3 += (1 - k) * k * ck * ukm1;
        }
    }
    h1 = (2.0 / kSqrtPi) * s1;
    d1 = (2.0 / kSqrtPi) * ds1 * du;
    h3 = (4.0 / (3.0 * kSqrtPi)) * s3;
    d3 = (4.0 / (3.0 * kSqrtPi)) * ds3 * du;
}

// Voigt function, FP32, branch-free: the expansion above with H1 and H3 from
// a cubic-Hermite table on a uniform grid in t = 1/(1+|v|) in (0, 1]
// (tab[i] = {H1, h dH1/dt, H3, h dH3/dt} at t_i = i h, h = 1/RH_VT_N).
//
// Every rounding step is an explicit intrinsic (fused multiply-adds where they
// are wanted, __f*_rn elsewhere): the compiler may not contract or split them,
// so the result does not depend on the code the function is inlined into.
// Hermite basis: h00 = f^2 (2f - 3) + 1, h01 = f^2 (3 - 2f), h10 = f (f - 1)^2,
// h11 = f^2 (f - 1).
__device__ __forceinline__ float voigt_f32(float a, float v, const float4 *__restrict__ tab)
{
    const float av = fabsf(v);
    const float v2 = __fmul_rn(av, av);
    const float g = __expf(-v2);
    const float t = rcp_f32(__fadd_rn(1.0f, av));
    const float x = __fmul_rn(t, (float)RH_VT_N);
    const int i = min((int)x, RH_VT_N - 1);
    const float f = __fsub_rn(x, (float)i);
    const float4 p0 = tab[i], p1 = tab[i + 1];
    const float f2 = __fmul_rn(f, f), fm1 = __fsub_rn(f, 1.0f);
    const float h00 = __fmaf_rn(f2, __fmaf_rn(2.0f, f, -3.0f), 1.0f);
    const float h01 = __fmul_rn(f2, __fmaf_rn(-2.0f, f, 3.0f));
    const float h10 = __fmul_rn(f, __fmul_rn(fm1, fm1));
    const float h11 = __fmul_rn(f2, fm1);
    const float H1 = __fmaf_rn(h00, p0.x, __fmaf_rn(h10, p0.y, __fmaf_rn(h01, p1.x, __fmul_rn(h11, p1.y))));
    const float H3 = __fmaf_rn(h00, p0.z, __fmaf_rn(h10, p0.w, __fmaf_rn(h01, p1.z, __fmul_rn(h11, p1.w))));
    const float a2 = __fmul_rn(a, a);
    // 1 + a^2 (1 - 2 v^2) + a^4 (2/3 v^4 - 2 v^2 + 1/2)
    const float q4 = __fmaf_rn(v2, __fmaf_rn(0.66666667f, v2, -2.0f), 0.5f);
    const float gpoly = __fmaf_rn(__fmul_rn(a2, a2), q4, __fmaf_rn(a2, __fmaf_rn(-2.0f, v2, 1.0f), 1.0f));
    return __fmaf_rn(g, gpoly, __fmul_rn(a, __fmaf_rn(a2, H3, H1)));
}

__device__ __forceinline__ float disp_f32(float a, float v, const float4 *__restrict__ tab)
{
    float av = fabsf(v);
    float v2 = av * av;
    float g = __expf(-v2);
    float t = rcp_f32(1.0f + av);
    float x = t * (float)RH_VT_N;
    int i = min((int)x, RH_VT_N - 1);
    float f = x - (float)i;
    float4 p0 = tab[i], p1 = tab[i + 1];
    float f2 = f * f, f3 = f2 * f;
    float h00 = 2.0f * f3 - 3.0f * f2 + 1.0f, h10 = f3 - 2.0f * f2 + f, h01 = 3.0f * f2 - 2.0f * f3, h11 = f3 - f2;
    float L0 = h00 * p0.x + h10 * p0.y + h01 * p1.x + h11 * p1.y;
    float L2 = h00 * p0.z + h10 * p0.w + h01 * p1.z + h11 * p1.w;
    float a2 = a * a;
    float l = L0 - 0.5f * a2 * L2 + a * g * av * (-2.0f + a2 * (1.3333333f * v2 - 2.0f));
    return v < 0.0f ? -l : l;
}

// ----------------------------------------------------------------------------
// Angle-averaged redistribution function R_II-A (Hummer 1962) in Doppler
// units, integrated by parts:
//   R(x', x) = (1/2pi) int_{u0}^{u0+6.5} erfc(u) [L(u + xs) + L(u - xb)] du,
//   L(s) = a/(a^2 + s^2), xs = min(x,x'), xb = max(x,x'), u0 = (xb - xs)/2
// (erfc(u0 + 6.5) < 1e-20 erfc(u0)).  Each Lorentzian term: within +-1 of its
// centre c the substitution u = c + a sinh z turns L du into dz/cosh z
// (panels of length ZP in z); elsewhere Gauss-Legendre in u (panels of
// length UP); NG-point rules.  FP64: NG = 8, ZP = 1, UP = 1/2; FP32: NG = 6,
// ZP = 2, UP = 1.
template <typename R> struct R2Rule;
template <> struct R2Rule<double> {
    static constexpr int NG = 8;
    static constexpr double ZP = 1.0, UP = 0.5;
    static constexpr double CUT = 6.0;    // R <= erfc(u0) < 2e-17 beyond
};
template <> struct R2Rule<float> {
    static constexpr int NG = 6;
    static constexpr double ZP = 2.0, UP = 1.0;
    static constexpr double CUT = 5.0;    // R <= erfc(u0) < 2e-12 beyond
};
__host__ __device__ inline void gl_rule(int n, double *x, double *w)
{
    // nodes and weights on [-1, 1] for n = 6 or 8
    if (n == 6) {
        const double xs[3] = {0.2386191860831969086, 0.6612093864662645136, 0.9324695142031520278};
        const double ws[3] = {0.4679139345726910473, 0.3607615730481386076, 0.1713244923791703450};
        for (int i = 0; i < 3; ++i) {
            x[i] = -xs[i]; x[5 - i] = xs[i];
            w[i] = ws[i]; w[5 - i] = ws[i];
        }
    } else {
        const double xs[4] = {0.1834346424956498049, 0.5255324099163289858, 0.7966664774136267396,
                              0.9602898564975362317};
        const double ws[4] = {0.3626837833783619830, 0.3137066458778872873, 0.2223810344533744706,
                              0.1012285362903762592};
        for (int i = 0; i < 4; ++i) {
            x[i] = -xs[i]; x[7 - i] = xs[i];
            w[i] = ws[i]; w[7 - i] = ws[i];
        }
    }
}

template <typename R>
__device__ inline R r2_lorentz(R a, R c, R lo, R hi, const R *gx, const R *gw)
{
    constexpr int NG = R2Rule<R>::NG;
    const R ZP = (R)R2Rule<R>::ZP, UP = (R)R2Rule<R>::UP;
    R s = 0;
    // plain parts [lo, min(hi, c-1)] and [max(lo, c+1), hi]
    for (int side = 0; side < 2; ++side) {
        const R p = side == 0 ? lo : (lo > c + 1 ? lo : c + 1);
        const R q = side == 0 ? (hi < c - 1 ? hi : c - 1) : hi;
        if (!(q > p)) continue;
        const int n = (int)ceil((q - p) / UP);
        const R h = (q - p) / (R)n;
        for (int k = 0; k < n; ++k)
            for (int g = 0; g < NG; ++g) {
                const R u = p + h * ((R)k + gx[g]);
                const R d = u - c;
                s += gw[g] * h * erfc(u) * a / (a * a + d * d);
            }
    }
    // near part in z, u = c + a sinh z
    const R nlo = lo > c - 1 ? lo : c - 1, nhi = hi < c + 1 ? hi : c + 1;
    if (nhi > nlo) {
        const R z0 = asinh((nlo - c) / a), z1 = asinh((nhi - c) / a);
        const int n = (int)ceil((z1 - z0) / ZP);
        const R h = (z1 - z0) / (R)n;
        for (int k = 0; k < n; ++k)
            for (int g = 0; g < NG; ++g) {
                const R z = z0 + h * ((R)k + gx[g]);
                s += gw[g] * h * erfc(c + a * sinh(z)) / cosh(z);
            }
    }
    return s;
}

template <typename R>
__device__ inline R r2a_dev(R a, R xp, R x)
{
    const R xs = xp < x ? xp : x, xb = xp < x ? x : xp;
    const R u0 = (R)0.5 * (xb - xs), U = u0 + (R)6.5;
    if (u0 > (R)R2Rule<R>::CUT) return 0;      // R <= erfc(u0): negligible
    // nodes on [0, 1] and half weights, in the working precision
    double dx[8], dw[8];
    gl_rule(R2Rule<R>::NG, dx, dw);
    R gx[8], gw[8];
    for (int g = 0; g < R2Rule<R>::NG; ++g) {
        gx[g] = (R)(0.5 * (dx[g] + 1.0));
        gw[g] = (R)(0.5 * dw[g]);
    }
    return (r2_lorentz<R>(a, -xs, u0, U, gx, gw) + r2_lorentz<R>(a, xb, u0, U, gx, gw)) / (R)(2.0 * kPi);
}

// FP32 R_II-A: the same integral, but each Lorentzian's neighbourhood
// |u - c| <= 1 (inside [lo, hi]) is split as
//   int erfc(u) L(u - c) du = int P(d) L(d) dd + int [erfc(c + d) - P(d)] L(d) dd,
// P the cubic Taylor polynomial of erfc about c (erfc' = -(2/sqrt pi) e^{-u^2},
// e_n the Taylor coefficients), whose moments against L(d) = a/(a^2 + d^2)
// are closed forms:
//   M0 = atan(d2/a) - atan(d1/a),  M1 = (a/2) ln((a^2 + d2^2)/(a^2 + d1^2)),
//   M2 = a (d2 - d1) - a^2 M0,      M3 = a (d2^2 - d1^2)/2 - a^2 M1,
// and the remainder, O(d^4) L(d), is smooth: Gauss-Legendre on [d1, 0] and
// [0, d2].  Outside the neighbourhood, Gauss-Legendre panels of length 1 as
// in the FP64 rule.  About a third of the FP64 rule's transcendental
// evaluations (no sinh/cosh substitution); the neglected structure of the
// remainder at |d| ~ a is O(a^4) relative.
__host__ __device__ inline float r2_lorentz_win(float a, float c, float lo, float hi, const float *gx,
                                                const float *gw)
{
    constexpr int NG = 6;
    float s = 0.f;
    for (int side = 0; side < 2; ++side) {
        const float p = side == 0 ? lo : fmaxf(lo, c + 1.f);
        const float q = side == 0 ? fminf(hi, c - 1.f) : hi;
        if (!(q > p)) continue;
        const int n = (int)ceilf(q - p);
        const float h = (q - p) / (float)n;
        for (int k = 0; k < n; ++k)
            for (int g = 0; g < NG; ++g) {
                const float u = p + h * ((float)k + gx[g]);
                const float d = u - c;
                s += gw[g] * h * erfcf(u) * a / (a * a + d * d);
            }
    }
    const float wl = fmaxf(lo, c - 1.f), wh = fminf(hi, c + 1.f);
    if (wh > wl) {
        const float d1 = wl - c, d2 = wh - c, a2 = a * a;
        const float e0 = erfcf(c), g0 = 1.1283791670955126f * expf(-c * c);
        const float e1 = -g0, e2 = g0 * c, e3 = g0 * (1.f - 2.f * c * c) * (1.f / 3.f);
        // atan difference without cancellation when d1, d2 have one sign
        const float M0 = (d1 * d2 > 0.f) ? atanf(a * (d2 - d1) / (a2 + d1 * d2)) : atanf(d2 / a) - atanf(d1 / a);
        const float M1 = 0.5f * a * log1pf((d2 - d1) * (d2 + d1) / (a2 + d1 * d1));
        const float M2 = a * (d2 - d1) - a2 * M0;
        const float M3 = 0.5f * a * (d2 - d1) * (d2 + d1) - a2 * M1;
        s += e0 * M0 + e1 * M1 + e2 * M2 + e3 * M3;
        for (int side = 0; side < 2; ++side) {
            const float p = side == 0 ? d1 : fmaxf(d1, 0.f);
            const float q = side == 0 ? fminf(d2, 0.f) : d2;
            if (!(q > p)) continue;
            const float h = q - p;
            for (int g = 0; g < NG; ++g) {
                const float d = p + h * gx[g];
                const float r = erfcf(c + d) - (e0 + d * (e1 + d * (e2 + d * e3)));
                s += gw[g] * h * r * a / (a2 + d * d);
            }
        }
    }
    return s;
}

template <>
__device__ inline float r2a_dev<float>(float a, float xp, float x)
{
    const float xs = xp < x ? xp : x, xb = xp < x ? x : xp;
    const float u0 = 0.5f * (xb - xs), U = u0 + 6.5f;
    if (u0 > (float)R2Rule<float>::CUT) return 0.f;      // R <= erfc(u0): negligible
    // 6-point Gauss-Legendre nodes on [0, 1] and half weights
    const float gx[6] = {0.033765242898423975f, 0.16939530676686776f, 0.38069040695840156f,
                         0.61930959304159844f, 0.83060469323313224f, 0.96623475710157603f};
    const float gw[6] = {0.085662246189585178f, 0.18038078652406930f, 0.23395696728634552f,
                         0.23395696728634552f, 0.18038078652406930f, 0.085662246189585178f};
    return (r2_lorentz_win(a, -xs, u0, U, gx, gw) + r2_lorentz_win(a, xb, u0, U, gx, gw)) *
           (float)(1.0 / (2.0 * kPi));
}

// ----------------------------------------------------------------------------
// Linear short characteristics weights: e0 = 1 - exp(-d), e1 = d - e0,
// w_o = e1/d, w_u = e0 - w_o; also 1 - w_o = e0/d, formed without
// cancellation (it carries the preconditioned rates in optically thick
// layers, where w_o -> 1).
__device__ __forceinline__ void sc_weights(double d, double &one_m_e0, double &wu, double &wo, double &omwo)
{
    double e0 = -expm1(-d);
    if (d < 0.1) {
        // w_o = sum_{n>=2} (-1)^n d^{n-1}/n!  (13 terms: truncation < 1e-20 relative)
        double t = d * 0.5, s = 0.0;
#pragma unroll
        for (int n = 3; n <= 15; ++n) {
            s += t;
            t *= -d / n;
        }
        wo = s;
        wu = e0 - wo;          // ~ d/2: no cancellation
        omwo = 1.0 - wo;
        one_m_e0 = 1.0 - e0;
    } else {
        // 1 - w_o = e0/d and w_u = e0/d - e^{-d}: w_u ~ 1/d at large d is formed
        // without subtracting two numbers close to one
        double ex = exp(-d);
        omwo = e0 / d;
        wo = 1.0 - omwo;
        wu = omwo - ex;
        one_m_e0 = ex;
    }
}

__device__ __forceinline__ void sc_weights(float d, float &one_m_e0, float &wu, float &wo, float &omwo)
{
    if (d < 0.5f) {
        // w_o = sum_{n>=2} (-1)^n d^{n-1}/n!,  e0 = sum_{n>=1} (-1)^{n+1} d^n/n!  (Horner, 9 terms)
        float wo_ = 0.5f + d * (-1.0f / 6 + d * (1.0f / 24 + d * (-1.0f / 120 + d * (1.0f / 720 +
                    d * (-1.0f / 5040 + d * (1.0f / 40320 + d * (-1.0f / 362880)))))));
        wo_ *= d;
        float e0 = d * (1.0f + d * (-0.5f + d * (1.0f / 6 + d * (-1.0f / 24 + d * (1.0f / 120 +
                   d * (-1.0f / 720 + d * (1.0f / 5040 + d * (-1.0f / 40320))))))));
        wo = wo_;
        wu = e0 - wo_;
        omwo = 1.0f - wo_;
        one_m_e0 = 1.0f - e0;
    } else {
        float ex = __expf(-d);
        float inv = rcp_f32(d);
        omwo = (1.0f - ex) * inv;
        wo = 1.0f - omwo;
        wu = omwo - ex;
        one_m_e0 = ex;
    }
}

// Quadratic Bezier short-characteristics step over optical path d (the
// higher-order formal solver option): I_o = I_u ex + wu S_u + wo S_o + wc C
// with C the Bezier control point of the step, and omp = 1 - wo - wc for the
// local operator Psi* = wo + wc.  wu = [2 - e^{-d}(d^2 + 2d + 2)]/d^2,
// wo = [d^2 - 2d + 2 - 2e^{-d}]/d^2, wc = [2d - 4 + (2d + 4)e^{-d}]/d^2,
// omp = 2[1 - e^{-d}(1 + d)]/d^2; below d = 1 their power series in d
// (t_n = (-d)^n/n!: wu = d sum t_n/(n+3), wo = d sum 2t_n/((n+1)(n+2)(n+3)),
// wc = d sum 2t_n/((n+2)(n+3)), omp = sum 2t_n/(n+2)), where the closed
// forms cancel.
__device__ __forceinline__ void bez_weights(double d, double &ex, double &wu, double &wo, double &wc, double &omp)
{
    if (d < 1.0) {
        double t = 1.0, su = 0.0, so = 0.0, sc = 0.0, sp = 0.0;   // 22 terms: truncation < 1e-20
#pragma unroll
        for (int n = 0; n < 22; ++n) {
            if (n > 0) t *= -d * (1.0 / n);
            su += t * (1.0 / (n + 3));
            so += t * (2.0 / ((n + 1) * (n + 2) * (n + 3)));
            sc += t * (2.0 / ((n + 2) * (n + 3)));
            sp += t * (2.0 / (n + 2));
        }
        wu = d * su;
        wo = d * so;
        wc = d * sc;
        omp = sp;
        ex = exp(-d);
    } else {
        const double e = exp(-d), d2 = d * d, id2 = 1.0 / d2;
        ex = e;
        wu = (2.0 - e * (d2 + 2.0 * d + 2.0)) * id2;
        wo = (d2 - 2.0 * d + 2.0 - 2.0 * e) * id2;
        wc = (2.0 * d - 4.0 + (2.0 * d + 4.0) * e) * id2;
        omp = 2.0 * (1.0 - e * (1.0 + d)) * id2;
    }
}

__device__ __forceinline__ void bez_weights(float d, float &ex, float &wu, float &wo, float &wc, float &omp)
{
    if (d < 1.0f) {
        float t = 1.0f, su = 0.0f, so = 0.0f, sc = 0.0f, sp = 0.0f;   // 12 terms: truncation < 3e-9
#pragma unroll
        for (int n = 0; n < 12; ++n) {
            if (n > 0) t *= -d * (1.0f / n);
            su += t * (1.0f / (n + 3));
            so += t * (2.0f / ((n + 1) * (n + 2) * (n + 3)));
            sc += t * (2.0f / ((n + 2) * (n + 3)));
            sp += t * (2.0f / (n + 2));
        }
        wu = d * su;
        wo = d * so;
        wc = d * sc;
        omp = sp;
        ex = __expf(-d);
    } else {
        const float e = __expf(-d), d2 = d * d, id2 = rcp_f32(d2);
        ex = e;
        wu = (2.0f - e * (d2 + 2.0f * d + 2.0f)) * id2;
        wo = (d2 - 2.0f * d + 2.0f - 2.0f * e) * id2;
        wc = (2.0f * d - 4.0f + (2.0f * d + 4.0f) * e) * id2;
        omp = 2.0f * (1.0f - e * (1.0f + d)) * id2;
    }
}

// The Bezier control point of the step u -> o: C = S_o - (d_u/2) S'_o, S'_o
// the weighted harmonic mean of the slopes to the upwind and the downwind
// point (Fritsch & Butland 1984; 0 where they differ in sign), C held
// between S_u and S_o; without a downwind point the midpoint (the linear
// step).
template <typename R>
__device__ __forceinline__ R bez_control(R Su, R So, R Sd, R du, R dd, bool has_d)
{
    if (!has_d) return (R)0.5 * (Su + So);
    const R su = (So - Su) / du, sd = (Sd - So) / dd;
    R der = 0;
    if (su * sd > (R)0) {
        const R a = ((R)1 + dd / (du + dd)) * (R)(1.0 / 3.0);
        der = su * sd / (a * sd + ((R)1 - a) * su);
    }
    const R C = So - (R)0.5 * du * der;
    const R lo = Su < So ? Su : So, hi = Su < So ? So : Su;
    return C < lo ? lo : (C > hi ? hi : C);
}

// spectrum sweeps need no 1 - w_o
template <typename R>
__device__ __forceinline__ void sc_weights(R d, R &one_m_e0, R &wu, R &wo)
{
    R omwo;
    sc_weights(d, one_m_e0, wu, wo, omwo);
}

// e^y E1(y), y > 0: series (y <= 1) or the continued fraction
// E1(y) = e^{-y} / (y + 1 - 1^2/(y + 3 - 2^2/(y + 5 - ...))) evaluated with
// the modified Lentz algorithm.
__host__ __device__ inline double exp_e1(double y)
{
    if (y <= 1.0) {
        const double gam = 0.57721566490153286061;
        double s = 0.0, t = 1.0;
        for (int n = 1; n < 100; ++n) {
            t *= -y / n;
            double a = t / n;
            s += a;
            if (fabs(a) < 1e-18 * fabs(s) + 1e-300) break;
        }
        return exp(y) * (-gam - log(y) - s);
    }
    const double tiny = 1e-300;
    double f = y + 1.0, C = f, D = 0.0;
    for (int n = 1; n < 500; ++n) {
        double an = -(double)n * n, bn = y + 2.0 * n + 1.0;
        D = bn + an * D;
        if (fabs(D) < tiny) D = tiny;
        C = bn + an / C;
        if (fabs(C) < tiny) C = tiny;
        D = 1.0 / D;
        double delta = C * D;
        f *= delta;
        if (fabs(delta - 1.0) < 1e-16) break;
    }
    return 1.0 / f;
}

// H- bound-free cross section (John 1988 fit), m^2; lambda in m.
__host__ __device__ inline double hminus_sigma(double lambda_m)
{
    const double l0 = 1.6419;
    double lum = lambda_m * 1e6;
    if (!(lum < l0)) return 0.0;
    double x = 1.0 / lum - 1.0 / l0, sx = sqrt(x);
    double f = 152.519 + sx * (49.534 + sx * (-118.858 + sx * (92.536 + sx * (-34.194 + sx * 4.982))));
    return 1e-22 * lum * lum * lum * x * sx * f;
}

struct ColumnArrays {
    int64_t ncol;
    int ndep;
    double *z, *T, *nH, *vz, *ne, *np, *nstar, *pops, *Crate, *dmax;
    int32_t *iters;
    uint8_t *status;
};

// launchers (defined in the kernel translation units)
cudaError_t launch_lte_setup(const DevAtom &A, const ColumnArrays &c, int ne_given, cudaStream_t st);
struct IterLaunch {
    int precision = 1, persistent = 1, block_warps = 0, maxiter = 1, ng_order = 0, ng_delay = 0, ng_period = 1,
        start = 0;
    double tol = 0.0, crsw = 1.0;
    int nsm = 1;
    const int *colidx = nullptr;   // columns to iterate (nullptr: all)
    int64_t nwork = 0;             // number of columns to iterate
    const int *nwork_d = nullptr;  // device count of columns to iterate (overrides nwork; set by an
                                   // earlier kernel on the same stream)
    int ctas_per_sm = 0;           // resident column blocks per SM (0: as many as fit)
    // re-run ladder run by the kernel itself for columns that do not converge
    int nrung = 0, rung_maxiter = 1;
    double rung_crsw[RH_MAX_RERUN] = {1.0, 1.0, 1.0, 1.0};
    int rung_ng[RH_MAX_RERUN] = {0, 0, 0, 0};   // Ng order of each rung (0 or the pass's)
    int *rung_cols = nullptr;                 // [nrung] columns entering each rung
    unsigned long long *rung_its = nullptr;   // [1 + nrung] formal solutions per pass / rung
    // partial redistribution (atoms with PRD lines)
    double prd_eps0 = 0.0;                    // PRD switching eps = min(1, eps0 it^2); <= 0: off
    int prd_hybrid = 0;                       // 1: rho in the frame of the moving gas (hybrid PRD)
    int formal = 0;                           // formal solver: 0 linear, 1 quadratic Bezier
    const int *lane_prd = nullptr;            // [npad] PRD point of each lane, -1: none
    const double *prd_nu = nullptr, *prd_w = nullptr;   // [npp] frequency, quadrature weight
    void *prd_scr = nullptr;                  // per-block scratch (mali_prd_bytes_per_block)
    size_t prd_cap = 0;
    // per-block profile cache (mali_phic_bytes_per_block); nullptr: the sweep
    // evaluates the Voigt profiles itself
    void *phic = nullptr;
    size_t phic_cap = 0;
};
cudaError_t launch_mali(const DevAtom &A, const ColumnArrays &c, const void *lane_tab, int npad,
                        const float4 *vtab, double nref, double *nghist, size_t nghist_cap, int *queue,
                        const IterLaunch &o, cudaStream_t st, float *ms_out, int *grid_out, char *err,
                        size_t errn);
size_t mali_nghist_bytes_per_block(const DevAtom &A, int ndep);
int mali_smem_layout(int precision, int L, int N, int ntr, int ncont, int nline, int macc, int ring_warps,
                     size_t *offsets, int noff, size_t *bytes);
int mali_max_ctas_per_sm(const DevAtom &A, int ndep, int precision, int block_warps);
size_t mali_prd_bytes_per_block(const DevAtom &A, int ndep, int precision);
size_t mali_phic_bytes_per_block(const DevAtom &A, int ndep, int precision);
cudaError_t launch_mali_prealloc(const DevAtom &A, const ColumnArrays &c, const void *lane_tab, int npad,
                                 const float4 *vtab, double nref, double *nghist, size_t nghist_cap, int *queue,
                                 const IterLaunch &o, cudaStream_t st, int *grid_out, char *err, size_t errn);
// start populations other than LTE: kind 3 zero radiation, 4 escape
// probability (kStartEscapeIterations solves); sp_* list, per continuum
// transition t, its wavelength points sp_off[t] .. sp_off[t+1]-1 (frequency and
// 4 pi w (2 h nu^3/c^2) alpha / (h nu)); lines have empty ranges
constexpr int kStartEscapeIterations = 3;
cudaError_t launch_start(const DevAtom &A, const ColumnArrays &c, int kind, const int *sp_off, const double *sp_nu,
                         const double *sp_ce, cudaStream_t st);
// depth-grid optimisation: monitor scales and the optional top cut
struct RegridParams {
    double dN, dT, dv, spacing, z_top;
    int use_z_top;
};
cudaError_t launch_regrid(const ColumnArrays &c, int M, const RegridParams &g, double *srow, double *zo, double *To,
                          double *nHo, double *vzo, double *neo, unsigned long long *bad, cudaStream_t st);
// emergent spectrum: per requested wavelength j, up to RH_SPEC_ACT transitions
// with constants spec[(j * RH_SPEC_ACT + s) * RH_SPEC_F + f]
#define RH_SPEC_ACT 8
#define RH_SPEC_F 8
cudaError_t launch_spectrum(const DevAtom &A, const ColumnArrays &c, double mu, int64_t nlam,
                            const double *nu_d, const int *nact_d, const int *act_d, const double *spec_d,
                            double *out, int precision, cudaStream_t st);

// emergent Stokes vector at mu = 1 of transition t0 (a line) with Zeeman
// splitting; B_T, theta, chi [ncol][ndep]; out [ncol][nlam][4]
cudaError_t launch_stokes(const DevAtom &A, const ColumnArrays &c, int t0, double geff, const double *B_T,
                          const double *theta, const double *chi, int64_t nlam, const double *nu_d, const int *nact_d,
                          const int *act_d, const double *spec_d, const float4 *vtab, const float4 *dtab, double *out,
                          int precision, cudaStream_t st);

// learned initial guess (rh15d_mlp.cu)
struct Mlp;
cudaError_t mlp_create(Mlp **out, int nin, int hidden, int nhid, int nout, uint64_t seed);
void mlp_destroy(Mlp *m);
int64_t mlp_nparams(const Mlp *m);
int mlp_nin(const Mlp *m);
int mlp_nlayer(const Mlp *m);
int mlp_nout(const Mlp *m);
int64_t mlp_state_size(const Mlp *m);
cudaError_t mlp_get_state(const Mlp *m, float *h);
cudaError_t mlp_set_state(Mlp *m, const float *h);
cudaError_t mlp_features(const ColumnArrays &c, float *X, cudaStream_t st);
cudaError_t mlp_targets(const ColumnArrays &c, int L, float *Yt, cudaStream_t st);
cudaError_t mlp_set_standardisation(Mlp *m, const float *X, const int *idx, int64_t rows, cudaStream_t st);
cudaError_t mlp_loss_grad(Mlp *m, int64_t rows, const float *X, const float *Yt, const int *idx, double *loss_d,
                          cudaStream_t st);
cudaError_t mlp_adam(Mlp *m, float lr, float b1, float b2, float eps, cudaStream_t st);
const float *mlp_grad(const Mlp *m);
cudaError_t mlp_predict_apply(Mlp *m, const ColumnArrays &c, int L, float *X, float *lnb, int *nfallback_d,
                              cudaStream_t st);
cudaError_t mlp_prepare_predict(Mlp *m, int64_t ncol);   // allocates what mlp_predict_apply needs

}  // namespace rh
