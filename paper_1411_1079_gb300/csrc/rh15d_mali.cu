// rh15d_mali.cu -- column-resident MALI kernel (Sect. 2.1-2.3, 3.1).
//
// One thread block owns one column at a time and runs all of that column's
// MALI iterations with the column's state in shared memory: populations
// (FP64), collisional rates (FP64), per-depth atmosphere scalars, and the
// rate accumulators.  When it takes a column, the block evaluates the line
// profiles of every line slot, ray and depth (they do not depend on the
// populations) into a per-block cache in global memory.  Per iteration:
//   1. warps take 32-wavelength tiles of the grid from a block-local queue;
//      each lane owns one wavelength and, two angles mu at a time, sweeps depth
//      downward and then upward (linear short characteristics, intensity and
//      local operator in registers, profiles read from the cache one depth
//      ahead); at every depth the lane forms its
//      contributions to the preconditioned rate matrix (Rybicki & Hummer
//      1992), the warp reduce-scatters them with shuffles, and one lane per
//      value adds it to the tile's accumulator;
//   2. one thread per depth assembles the rate matrix from the accumulators
//      (FP64) plus collisions and solves the rate equations (FP64, scaled
//      unknowns, partial pivoting);
//   3. the block computes max |dn/n|, applies Ng order-2 acceleration
//      (history in global scratch) and tests convergence (Sect. 2.3).
// Columns come from a device work queue (pool mode, Sect. 3.1) or a static
// split over resident blocks (normal mode).  R is the precision of the
// formal solution and the rate terms (float or double); the rate matrix,
// the solve and Ng are always FP64.
#include <cstdio>
#include <cstring>

#include "rh15d_internal.h"

#ifndef RH_ANGLE_PAIRS
#define RH_ANGLE_PAIRS 1      // two angles per sweep pass (CRD); 0: one
#endif
#ifndef RH_FP32_MINBLOCKS
#define RH_FP32_MINBLOCKS 2   // FP32 sweep: two resident 256-thread blocks per SM (<= 128 registers)
#endif

namespace rh {

namespace {

constexpr int kWarp = 32;
// Profile ring of the FP32 sweep with the profile cache (two angles per
// pass): per warp, its tile's cached line profiles (at most kRingLines line
// slots, the pass's two rays) at kRingSlots depths -- the depth being swept
// and the next two -- copied from the cache by cp.async, so the HBM latency
// of a profile read is covered by two depth steps without holding the values
// in registers.
constexpr int kRingSlots = 3;
constexpr int kRingLines = 3;
constexpr int kRingSlotFloats = 2 * kRingLines * kWarp;
constexpr int kRingFloatsPerWarp = kRingSlots * kRingSlotFloats;
constexpr int kNgLanes = 64;                    // fixed partition of the Ng dot products
constexpr int kRedDoubles = 5 * kNgLanes + 8;   // block reduction scratch

struct KParams {
    int64_t ncol;
    int N, L;
    const double *z, *T, *nH, *vz, *ne, *np, *nstar, *Crate;
    double *pops, *dmax;
    int32_t *iters;
    uint8_t *status;
    const void *lane;
    int npad;
    const float4 *vtab;
    double *nghist;
    int *queue;
    int persistent, maxiter, ng_order, ng_delay, ng_period, start;
    double tol, crsw, inv_nref;
    const int *colidx;         // work item -> column (nullptr: identity)
    int64_t nwork;
    const int *nwork_d;        // device count of work items (overrides nwork when set)
    // re-run ladder inside the kernel (Sect. 2.3): a column not converged
    // after its pass is restarted from LTE with switching factor rung_crsw[r],
    // Ng order rung_ng[r] and rung_maxiter iterations, r = 0 .. nrung-1
    int nrung, rung_maxiter;
    double rung_crsw[RH_MAX_RERUN];
    int rung_ng[RH_MAX_RERUN];
    int *rung_cols;                  // [nrung] columns entering each rung (nullptr: not counted)
    unsigned long long *rung_its;    // [1 + nrung] formal solutions of the pass and of each rung
    // partial redistribution
    double prd_eps0;
    int prd_hybrid;                  // 1: rho in the frame of the moving gas
    int formal;                      // formal solver: 0 linear, 1 quadratic Bezier short characteristics
    const int *lane_prd;
    const double *prd_nu, *prd_w;
    char *prd_scr;
    size_t prd_stride;               // bytes of scratch per block
    // profile cache (nullptr: the sweep evaluates the profiles itself)
    char *phic;
    size_t phic_stride;              // bytes of cache per block
};

// Per-block PRD scratch: in R, the redistribution kernels K [sum np^2][N] (per
// line [k][j][i] = K_ij: transposed, so that the threads of a warp, which own
// consecutive points i, read consecutive addresses), then per PRD point
// [npp][N] the J-bar weights f, the mean intensity J, rho, D = dJ/drho (the
// derivative of J through the line's own emission) and the reduced frequency
// x of the point at each depth, per line [nprd][N] the damping a, then the
// plain-rate accumulators [pacc][N], the intensity of every ray at the PRD
// points [2 nmu][npp][N] (ray 2 m + d) followed by each ray's dI/drho there
// through the line's own emission [2 nmu][npp][N] (the hybrid scheme's
// gas-frame J and D are interpolated from them) and each ray's rho at the
// points [2 nmu][npp][N] (the hybrid scheme's gas-frame rho at the ray's
// gas-frame frequency, filled once per iteration), the hybrid scheme's
// interpolation tables of the column [2 nmu][npp][N] each (they depend on
// its velocities only; brackets as int in R-sized slots): for J_f at point
// i the bracket j and weight t of q_i + mu_z v_z and the weights e0, e1 of
// point i in the ray's rho at points j and j + 1, for the ray's rho at
// point p the bracket and weight of q_p - mu_z v_z; and the points'
// frequencies in velocity units c (nu - nu0) / nu0 [npp].  In FP64 the
// supply fraction F and J-bar per line [nprd][N], then the Ng history of rho
// [4][npp][N] (newest first).
template <typename R>
struct PrdScr {
    R *K, *f, *J, *rho, *D, *x, *a, *plain, *Iray, *ht, *he0, *he1, *rt, *q;
    int *hj, *rj;
    double *F, *Jbar, *hist;
};
template <typename R>
__host__ __device__ inline size_t prd_bytes(const DevAtom &A, int N)
{
    size_t r = sizeof(R) * ((size_t)A.prd_koff[A.nprd] * N + 5 * (size_t)A.npp * N + (size_t)A.nprd * N +
                            (size_t)A.pacc * N + 18 * (size_t)A.nmu * A.npp * N + (size_t)A.npp);
    r = (r + 255) & ~(size_t)255;
    r += sizeof(double) * (2 * (size_t)A.nprd * N + 4 * (size_t)A.npp * N) + 256;
    return (r + 255) & ~(size_t)255;   // every block's scratch 256-byte aligned (float4 loads of K)
}
// Per-block profile cache: the line profile phi (Voigt H(a, v) times its
// normalisation and 1/Doppler width, v including the ray's Doppler shift)
// of every line slot, ray and depth, [nphi][2 nmu][N][32 lanes] in R, ray
// 2 m + d for angle m downward (d = 0) and upward (d = 1).  The profiles do
// not depend on the populations, so a column builds them once and every
// iteration reads them back instead of evaluating the Voigt function.
template <typename R>
__host__ __device__ inline size_t phic_bytes(const DevAtom &A, int N)
{
    const size_t r = sizeof(R) * (size_t)A.nphi * 2 * A.nmu * N * 32;
    return (r + 255) & ~(size_t)255;
}

template <typename R>
__device__ inline PrdScr<R> prd_carve(char *base, const DevAtom &A, int N)
{
    PrdScr<R> q;
    R *r = reinterpret_cast<R *>(base);
    q.K = r;
    r += (size_t)A.prd_koff[A.nprd] * N;
    q.f = r;
    r += (size_t)A.npp * N;
    q.J = r;
    r += (size_t)A.npp * N;
    q.rho = r;
    r += (size_t)A.npp * N;
    q.D = r;
    r += (size_t)A.npp * N;
    q.x = r;
    r += (size_t)A.npp * N;
    q.a = r;
    r += (size_t)A.nprd * N;
    q.plain = r;
    r += (size_t)A.pacc * N;
    q.Iray = r;
    r += 6 * (size_t)A.nmu * A.npp * N;   // intensities, dI/drho, then rho per ray
    const size_t nt = 2 * (size_t)A.nmu * A.npp * N;
    q.hj = reinterpret_cast<int *>(r);
    r += nt;
    q.ht = r;
    r += nt;
    q.he0 = r;
    r += nt;
    q.he1 = r;
    r += nt;
    q.rj = reinterpret_cast<int *>(r);
    r += nt;
    q.rt = r;
    r += nt;
    q.q = r;
    r += (size_t)A.npp;
    size_t off = (reinterpret_cast<size_t>(r) + 255) & ~(size_t)255;
    q.F = reinterpret_cast<double *>(off);
    q.Jbar = q.F + (size_t)A.nprd * N;
    q.hist = q.Jbar + (size_t)A.nprd * N;
    return q;
}

template <typename R>
struct Smem {
    double *n, *nn, *Cr;       // [L*N], [L*N], [N][2*ntr]
    R *slot;                   // [macc][N]
    R *dz, *ivth, *vz;         // [N]
    R *bg;                     // [N][4]: h/kT, free-free, H- density, Thomson (one vector load per depth)
    R *Gc;                     // [ncont][N]
    R *ad;                     // [nline][N] damping
    R *nr;                     // [L][N] populations in R
    float4 *vtab;              // [RH_VT_N + 1] Voigt coefficient table
    double *red;               // reduction scratch [kRedDoubles]
    int *ibuf;                 // [8]
    float *ring;               // [warps][kRingFloatsPerWarp] profile ring (ring kernels only)
};

// Byte offsets of the regions of the block's dynamic shared memory.  The one
// function both sizes the allocation (host) and carves it (device), so the
// two cannot disagree: a layout whose carve ends past the allocated size
// (regions reserved by the carve but dropped from the size) writes outside
// the block's shared memory.
struct SmemLayout {
    size_t n, nn, Cr, red, slot, dz, ivth, vz, bg, Gc, ad, nr, vtab, ibuf, ring, end;
};
// ring_warps: warps whose profile ring the block holds (the launch's warps
// for a ring kernel, else 0)
template <typename R>
__host__ __device__ inline SmemLayout smem_layout(int L, int N, int ntr, int ncont, int nline, int macc,
                                                  int ring_warps)
{
    SmemLayout o;
    size_t b = 0;
    o.n = b;
    b += sizeof(double) * (size_t)L * N;
    o.nn = b;
    b += sizeof(double) * (size_t)L * N;
    o.Cr = b;
    b += sizeof(double) * (size_t)N * 2 * ntr;
    o.red = b;
    b += sizeof(double) * kRedDoubles;
    o.slot = b;
    b += sizeof(R) * (size_t)macc * N;
    size_t *one[3] = {&o.dz, &o.ivth, &o.vz};
    for (int i = 0; i < 3; ++i) {
        *one[i] = b;
        b += sizeof(R) * (size_t)N;
    }
    b = (b + 15) & ~(size_t)15;                    // vector loads of the background block
    o.bg = b;
    b += sizeof(R) * 4 * (size_t)N;
    o.Gc = b;
    b += sizeof(R) * (size_t)ncont * N;
    o.ad = b;
    b += sizeof(R) * (size_t)nline * N;
    o.nr = b;
    b += sizeof(R) * (size_t)L * N;
    b = (b + 15) & ~(size_t)15;                    // float4 table: 16-byte aligned
    o.vtab = b;
    b += sizeof(float4) * (RH_VT_N + 1);
    o.ibuf = b;
    b += sizeof(int) * 8;
    b = (b + 15) & ~(size_t)15;
    o.ring = b;
    b += sizeof(float) * (size_t)kRingFloatsPerWarp * ring_warps;
    o.end = b;
    return o;
}

template <typename R>
__host__ __device__ size_t smem_bytes(int L, int N, int ntr, int ncont, int nline, int macc, int ring_warps)
{
    return smem_layout<R>(L, N, ntr, ncont, nline, macc, ring_warps).end;
}

// kernels whose sweep reads the line profiles through the ring (the
// two-angle passes of the linear solver)
template <typename R, bool PRD, bool CACHE, bool BEZ>
__host__ __device__ constexpr bool uses_ring()
{
    return RH_ANGLE_PAIRS && CACHE && !PRD && !BEZ && sizeof(R) == 4;
}

template <typename R>
__device__ Smem<R> carve(char *base, int L, int N, int ntr, int ncont, int nline, int macc, int ring_warps)
{
    const SmemLayout o = smem_layout<R>(L, N, ntr, ncont, nline, macc, ring_warps);
    Smem<R> s;
    s.n = reinterpret_cast<double *>(base + o.n);
    s.nn = reinterpret_cast<double *>(base + o.nn);
    s.Cr = reinterpret_cast<double *>(base + o.Cr);
    s.red = reinterpret_cast<double *>(base + o.red);
    s.slot = reinterpret_cast<R *>(base + o.slot);
    s.dz = reinterpret_cast<R *>(base + o.dz);
    s.ivth = reinterpret_cast<R *>(base + o.ivth);
    s.vz = reinterpret_cast<R *>(base + o.vz);
    s.bg = reinterpret_cast<R *>(base + o.bg);
    s.Gc = reinterpret_cast<R *>(base + o.Gc);
    s.ad = reinterpret_cast<R *>(base + o.ad);
    s.nr = reinterpret_cast<R *>(base + o.nr);
    s.vtab = reinterpret_cast<float4 *>(base + o.vtab);
    s.ibuf = reinterpret_cast<int *>(base + o.ibuf);
    s.ring = reinterpret_cast<float *>(base + o.ring);
    return s;
}

template <typename R>
__device__ __forceinline__ R voigt(R a, R v, const float4 *tab);
template <>
__device__ __forceinline__ float voigt<float>(float a, float v, const float4 *tab) { return voigt_f32(a, v, tab); }
template <>
__device__ __forceinline__ double voigt<double>(double a, double v, const float4 *) { return voigt_f64(a, v); }

// 4-byte asynchronous global -> shared copy and its group fences (each
// thread waits for its own copies; a thread reads only what it copied)
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Line profile phi(k, ray) of one wavelength: the Doppler shift of the ray,
// the Voigt function and the normalisation, with every rounding step fixed by
// intrinsics.  The cache build and the in-sweep evaluation both call this, and
// the compiler may not fuse or split its operations differently in the two
// places, so cached and uncached sweeps give the same bits.
__device__ __forceinline__ float line_phi(float q, float muz, float vz, float ivth, float a, float pn,
                                          const float4 *tab)
{
    const float v = __fmul_rn(__fmaf_rn(-muz, vz, q), ivth);
    return __fmul_rn(__fmul_rn(voigt<float>(a, v, tab), pn), ivth);
}
__device__ __forceinline__ double line_phi(double q, double muz, double vz, double ivth, double a, double pn,
                                           const float4 *tab)
{
    const double v = __dmul_rn(__fma_rn(-muz, vz, q), ivth);
    return __dmul_rn(__dmul_rn(voigt<double>(a, v, tab), pn), ivth);
}

template <typename R> __device__ __forceinline__ R rcp(R x);
template <> __device__ __forceinline__ float rcp<float>(float x) { return rcp_f32(x); }
template <> __device__ __forceinline__ double rcp<double>(double x) { return 1.0 / x; }

// 1 - exp(-x) for x > 0: FP32 uses 1 - __expf(-x) (x = h nu / kT > 0.1 on every grid here,
// relative error < 1e-6), FP64 expm1
template <typename R> __device__ __forceinline__ R one_m_exp(R x, R ex);
template <> __device__ __forceinline__ float one_m_exp<float>(float x, float ex) { return 1.0f - ex; }
template <> __device__ __forceinline__ double one_m_exp<double>(double x, double ex) { return -expm1(-x); }

template <typename R> __device__ __forceinline__ R rexp(R x);
template <> __device__ __forceinline__ float rexp<float>(float x) { return __expf(x); }
template <> __device__ __forceinline__ double rexp<double>(double x) { return exp(x); }

template <typename R> __device__ __forceinline__ R mu_of(const DevAtom &A, int m);
template <> __device__ __forceinline__ float mu_of<float>(const DevAtom &A, int m) { return A.muf[m]; }
template <> __device__ __forceinline__ double mu_of<double>(const DevAtom &A, int m) { return A.mu[m]; }
template <typename R> __device__ __forceinline__ R imu_of(const DevAtom &A, int m);
template <> __device__ __forceinline__ float imu_of<float>(const DevAtom &A, int m) { return A.imuf[m]; }
template <> __device__ __forceinline__ double imu_of<double>(const DevAtom &A, int m) { return 1.0 / A.mu[m]; }
// a product rounded on its own (never fused into a following addition)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename R> __device__ __forceinline__ R wm2_of(const DevAtom &A, int m);
template <> __device__ __forceinline__ float wm2_of<float>(const DevAtom &A, int m) { return A.wm2f[m]; }
template <> __device__ __forceinline__ double wm2_of<double>(const DevAtom &A, int m) { return 0.5 * A.wmu[m]; }

// four consecutive values of a 16-byte aligned shared array
__device__ __forceinline__ void load4(const float *p, float &a, float &b, float &c, float &d)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void load4(const double *p, double &a, double &b, double &c, double &d)
{
    const double2 u = reinterpret_cast<const double2 *>(p)[0], v = reinterpret_cast<const double2 *>(p)[1];
    a = u.x; b = u.y; c = v.x; d = v.y;
}

// Per-lane constants of one tile with K transitions in its union.
template <typename R, int K>
struct LaneC {
    R c[K], Vc[K], Uc[K], E[K], q[K], pn[K], grat[K];
    int isline[K], lo[K], up[K], sub[K];
    R nu, nu3s, tw, hm;
};

// Depth-dependent, angle-independent quantities of one lane.
template <typename R, int K>
struct DepthC {
    R chibg, etabg, B, etac;
    R Rs[K], Xs[K], nu_[K], chc[K], Uct[K];
    R rf[K];                   // partial redistribution: psi/phi of the slot (1 otherwise)
};

template <typename R, int K, bool PRD = false>
__device__ __forceinline__ void depth_consts(const Smem<R> &s, const LaneC<R, K> &lc, int k, int N, DepthC<R, K> &d,
                                             R rho_k = (R)1, int prd_slot = -1)
{
    R hkT, kff, nhm, thom;
    load4(s.bg + 4 * k, hkT, kff, nhm, thom);
    R x = lc.nu * hkT;
    R ex = rexp<R>(-x);
    R omex = one_m_exp<R>(x, ex);
    d.chibg = (kff * lc.nu3s + nhm * lc.hm) * omex + thom;
    d.B = lc.tw * ex * rcp<R>(omex);
    d.etabg = d.chibg * d.B;
    d.etac = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        R nl = s.nr[lc.lo[j] * N + k];
        d.nu_[j] = s.nr[lc.up[j] * N + k];
        if (lc.isline[j]) {
            d.Rs[j] = lc.grat[j];
            if constexpr (PRD) {
                // psi = rho phi in stimulated and spontaneous emission
                d.rf[j] = j == prd_slot ? rho_k : (R)1;
                d.Rs[j] *= d.rf[j];
            }
            d.chc[j] = 0;
            d.Uct[j] = 0;
        } else {
            if constexpr (PRD) d.rf[j] = 1;
            d.Rs[j] = s.Gc[lc.sub[j] * N + k] * ex;
        }
        d.Xs[j] = nl - d.Rs[j] * d.nu_[j];
        if (!lc.isline[j]) {
            d.chc[j] = lc.Vc[j] * d.Xs[j];
            d.Uct[j] = lc.Uc[j] * d.Rs[j];
            d.etac += d.nu_[j] * d.Uct[j];
        }
    }
}

// Opacity and emissivity for one ray at one depth from the line profiles pc
// of its line slots; per-slot profile phi, opacity chj and emissivity per
// upper-level population U.
template <typename R, int K, bool PRD = false>
__device__ __forceinline__ void angle_vals(const LaneC<R, K> &lc, const DepthC<R, K> &d, const R (&pc)[K], R &chi,
                                           R &eta, R *phi, R *chj, R *U)
{
    chi = d.chibg;
    R ea = d.etac;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (lc.isline[j]) {
            const R ph = pc[j];
            phi[j] = ph;
            chj[j] = lc.Vc[j] * ph * d.Xs[j];
            U[j] = lc.Uc[j] * ph;
            if constexpr (PRD) U[j] *= d.rf[j];
            ea += d.nu_[j] * U[j];
        } else {
            phi[j] = 1;
            chj[j] = d.chc[j];
            U[j] = d.Uct[j];
        }
        chi += chj[j];
    }
    eta = d.etabg + ea;
}

// Warp reduce-scatter of P values (P a power of two): afterwards every lane
// holds the warp total of value index lane >> (5 - log2 P).
template <int P, typename R>
__device__ __forceinline__ R reduce_scatter(R (&v)[P], int lane)
{
    int o = 16;
#pragma unroll
    for (int n = P; n > 1; n >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            R send = upper ? v[i] : v[i + n / 2];
            R keep = upper ? v[i + n / 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
        o >>= 1;
    }
    R r = v[0];
#pragma unroll
    for (; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

template <int M> struct Pow2 { static constexpr int v = M <= 1 ? 1 : (M <= 2 ? 2 : (M <= 4 ? 4 : (M <= 8 ? 8 : (M <= 16 ? 16 : 32)))); };
template <int P> struct Log2 { static constexpr int v = P <= 1 ? 0 : 1 + Log2<P / 2>::v; };
template <> struct Log2<1> { static constexpr int v = 0; };

// Sweep one tile (K transitions in its union) for every angle, downward and
// upward, adding its rate accumulators.  One lane = one wavelength; the
// angle loop runs outside the depth sweep so the lane state is scalar.  At
// each depth the lane forms, without subtracting nearly equal numbers,
//   I_eff = I - Psi* eta_active = I_u e^{-dtau} + w_u S_u + w_o eta_bg/chi,
//   1 - Psi* chi_j = (1 - w_o) + w_o (chi - chi_j)/chi,
// and its contributions (weight w = w_mu/2):
//   up_j = c_j w phi_j I_eff,  down_j = c_j R_j w phi_j (E_j (1 - Psi* chi_j) + I_eff),
//   cross_{j,j'} = c_j X_j w phi_j Psi* U_j';
// the warp sums them over its wavelengths and lane a adds accumulator a.
// PRD: the tile's PRD slot emits with psi = rho phi (rho of the lane's point
// and depth from the block's scratch), PRD lanes accumulate the angle-averaged
// mean intensity J, and every slot also accumulates its plain rates (actual
// intensity) cw I and cw R (E + I), for the PRD update.
// NL >= 0: the tile's first NL slots are lines and the rest continua (the
// host orders the transitions lines first), known at compile time so the
// per-slot kind tests fold away; NL < 0: the kinds are read at run time.
// prd_I (hybrid PRD only, else nullptr): the rays' intensities at the PRD
// points and then their dI/drho, written here, and then the rays' rho,
// read here.
template <typename R, int K, int NL, bool PRD, bool CACHE, bool BEZ>
__device__ void sweep_tile_k(const DevAtom &A, const Smem<R> &s, const KParams &p, int b, int lane, R *prd_rho,
                             R *prd_J, R *prd_D, R *prd_plain, R *prd_I, const R *phc)
{
    const int N = p.N;
    const DevTile &tl = A.tile[b];
    const int nmu = A.nmu;
    const R *lt = reinterpret_cast<const R *>(p.lane);
    const int npad = p.npad;
    const int pi = b * kWarp + lane;
    LaneC<R, K> lc;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const DevTrans &tr = A.tr[tl.t[j]];
        lc.c[j] = lt[(RH_NLANEF * j + 0) * npad + pi];
        lc.Vc[j] = lt[(RH_NLANEF * j + 1) * npad + pi];
        lc.Uc[j] = lt[(RH_NLANEF * j + 2) * npad + pi];
        lc.E[j] = lt[(RH_NLANEF * j + 3) * npad + pi];
        lc.q[j] = lt[(RH_NLANEF * j + 4) * npad + pi];
        lc.pn[j] = lt[(RH_NLANEF * j + 5) * npad + pi];
        lc.grat[j] = lt[(RH_NLANEF * j + 6) * npad + pi];
        lc.isline[j] = NL >= 0 ? j < NL : tr.kind == 0;
        lc.lo[j] = tr.l;
        lc.up[j] = tr.u;
        lc.sub[j] = tr.sub;
    }
    lc.nu = lt[kLaneNu * npad + pi];
    lc.hm = lt[kLaneHm * npad + pi];
    lc.nu3s = lt[kLaneNu3 * npad + pi];
    lc.tw = lt[kLaneTw * npad + pi];
    // line profiles of depth k, ray r (2 m + d) for the tile's line slots (0
    // elsewhere): read from the column's cache (CACHE), or evaluated here (the
    // same arithmetic as the cache's build)
    const int nray = 2 * nmu;
    // lane's element of each line slot's cache row (int: at most 288 rows x
    // 32 rays x 4096 depths x 32 lanes < 2^31)
    int poff[K];
#pragma unroll
    for (int j = 0; j < K; ++j) poff[j] = CACHE && lc.isline[j] ? tl.phi[j] * nray * N * kWarp + lane : 0;
    auto load_ph = [&](int k, int r, R (&o)[K]) {
        const int rk = (r * N + k) * kWarp;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (!lc.isline[j]) {
                o[j] = 0;
            } else if constexpr (CACHE) {
                o[j] = phc[poff[j] + rk];
            } else {
                const R mu = mu_of<R>(A, r >> 1);
                o[j] = line_phi(lc.q[j], (r & 1) ? mu : -mu, s.vz[k], s.ivth[k], s.ad[lc.sub[j] * N + k], lc.pn[j],
                                s.vtab);
            }
        }
    };
    constexpr int M = K * (K + 1);
    constexpr int MP = PRD ? M + 2 * K : M;        // with the plain rates
    constexpr int P = Pow2<MP>::v;
    constexpr int SH = 5 - Log2<P>::v;
    R *slot = s.slot + (size_t)tl.acc_off * N;
    const bool writer = (lane & ((1 << SH) - 1)) == 0;
    const int widx = lane >> SH;
    int pp = -1;                                   // PRD point of the lane
    const R *rho_lane = nullptr;
    R *plain = nullptr;
    constexpr bool bez = BEZ;                      // quadratic Bezier formal solver
    bool hyb = false;                              // hybrid PRD at this lane
    if constexpr (PRD) {
        pp = tl.prd_slot >= 0 ? p.lane_prd[pi] : -1;
        rho_lane = pp >= 0 ? prd_rho + (size_t)pp * N : nullptr;
        plain = prd_plain + (size_t)tl.pacc_off * N;
        hyb = prd_I != nullptr && pp >= 0;
    }

    // rate contributions of one ray at one depth point (add: accumulate into val)
    auto contrib = [&](const DepthC<R, K> &d, const R (&phi)[K], const R (&chj)[K], const R (&U)[K], R ichi, R wo,
                       R omwo, R psi, R Ieff, R wm2, R (&val)[P], bool add) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            R other = d.chibg;
#pragma unroll
            for (int j2 = 0; j2 < K; ++j2)
                if (j2 != j) other += chj[j2];
            const R f = omwo + wo * other * ichi;          // 1 - Psi* chi_j
            const R cw = lc.c[j] * wm2 * phi[j];
            const R v0 = cw * Ieff, v1 = cw * d.Rs[j] * (lc.E[j] * f + Ieff);
            val[j] = add ? val[j] + v0 : v0;
            val[K + j] = add ? val[K + j] + v1 : v1;
            const R cx = cw * d.Xs[j] * psi;
#pragma unroll
            for (int j2 = 0; j2 < K; ++j2)
                if (j2 != j) {
                    const int a = 2 * K + j * (K - 1) + (j2 < j ? j2 : j2 - 1);
                    val[a] = add ? val[a] + cx * U[j2] : cx * U[j2];
                }
        }
    };
    // reduce the warp's contributions and add them to the tile's accumulators
    auto flush = [&](int k, R (&val)[P]) {
#pragma unroll
        for (int a = MP; a < P; ++a) val[a] = 0;
        const R t = reduce_scatter<P>(val, lane);
        if (writer && widx < M) slot[widx * N + k] += t;   // zeroed before the sweep
    };

    // contributions of one depth point to the tile's accumulators
    auto emit = [&](int k, const DepthC<R, K> &d, const R (&phi)[K], const R (&chj)[K], const R (&U)[K], R ichi,
                    R wo, R omwo, R psi, R Ieff, R Ik, R wm2, int ray) {
        R val[P];
        contrib(d, phi, chj, U, ichi, wo, omwo, psi, Ieff, wm2, val, false);
        if constexpr (PRD) {
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const R cw = lc.c[j] * wm2 * phi[j];
                val[M + 2 * j] = cw * Ik;
                val[M + 2 * j + 1] = cw * d.Rs[j] * (lc.E[j] + Ik);
            }
            // fire-and-forget reductions (zeroed before the sweep): one lane per
            // location, adding in program order, so the sum is deterministic;
            // D = dJ/drho through the PRD line's own emission, Psi* n_u U0.
            // Hybrid PRD: the ray's I and dI/drho at the point instead, for
            // the gas-frame J and D of the rho update
            if (pp >= 0) {
                R e0 = 0;
#pragma unroll
                for (int j = 0; j < K; ++j)
                    if (j == tl.prd_slot) e0 = d.nu_[j] * lc.Uc[j] * phi[j];
                if (hyb) {
                    const size_t ri = ((size_t)ray * A.npp + pp) * N + k;
                    prd_I[ri] = Ik;
                    prd_I[ri + 2 * (size_t)A.nmu * A.npp * N] = psi * e0;
                } else {
                    atomicAdd(prd_J + (size_t)pp * N + k, wm2 * Ik);
                    atomicAdd(prd_D + (size_t)pp * N + k, wm2 * (psi * e0));
                }
            }
        }
#pragma unroll
        for (int a = MP; a < P; ++a) val[a] = 0;
        const R t = reduce_scatter<P>(val, lane);
        if (writer && widx < M) slot[widx * N + k] += t;   // zeroed before the sweep
        if constexpr (PRD) {
            if (writer && widx >= M && widx < MP) atomicAdd(plain + (widx - M) * N + k, t);
        }
    };

#if RH_ANGLE_PAIRS
    if constexpr (!PRD && !BEZ) {
        // two angles per pass: the depth terms once per depth, the angles'
        // contributions summed in registers, one warp reduction per depth
        for (int m0 = 0; m0 < nmu; m0 += 2) {
            const bool two = m0 + 1 < nmu;
            const int m1 = two ? m0 + 1 : m0;
            const R mu0 = mu_of<R>(A, m0), imu0 = imu_of<R>(A, m0), wa = wm2_of<R>(A, m0);
            const R mu1 = mu_of<R>(A, m1), imu1 = imu_of<R>(A, m1), wb = wm2_of<R>(A, m1);
            for (int dir = 0; dir < 2; ++dir) {
                const R z0 = dir == 0 ? -mu0 : mu0, z1 = dir == 0 ? -mu1 : mu1;
                const int ra = 2 * m0 + dir, rb = 2 * m1 + dir;
                R Ia, chipa = 0, Spa, Ib = 0, chipb = 0, Spb = 0;
                {
                    const int k0 = dir == 0 ? 0 : N - 1;
                    R B2 = 0;
                    R pc[K];
                    if (dir == 1) {
                        DepthC<R, K> d2;
                        depth_consts<R, K>(s, lc, N - 2, N, d2);
                        B2 = d2.B;
                        R phi[K], chj[K], U[K], eta;
                        load_ph(N - 2, ra, pc);
                        angle_vals<R, K>(lc, d2, pc, chipa, eta, phi, chj, U);
                        if (two) {
                            load_ph(N - 2, rb, pc);
                            angle_vals<R, K>(lc, d2, pc, chipb, eta, phi, chj, U);
                        }
                    }
                    DepthC<R, K> d;
                    depth_consts<R, K>(s, lc, k0, N, d);
                    R val[P];
                    {
                        R chi, eta, phi[K], chj[K], U[K];
                        load_ph(k0, ra, pc);
                        angle_vals<R, K>(lc, d, pc, chi, eta, phi, chj, U);
                        const R ichi = rcp<R>(chi);
                        Ia = dir == 0 ? (R)0 : d.B + mu0 * (d.B - B2) * rcp<R>((R)0.5 * (chi + chipa) * s.dz[N - 2]);
                        chipa = chi;
                        Spa = eta * ichi;
                        contrib(d, phi, chj, U, ichi, (R)0, (R)1, (R)0, Ia, wa, val, false);
                    }
                    if (two) {
                        R chi, eta, phi[K], chj[K], U[K];
                        load_ph(k0, rb, pc);
                        angle_vals<R, K>(lc, d, pc, chi, eta, phi, chj, U);
                        const R ichi = rcp<R>(chi);
                        Ib = dir == 0 ? (R)0 : d.B + mu1 * (d.B - B2) * rcp<R>((R)0.5 * (chi + chipb) * s.dz[N - 2]);
                        chipb = chi;
                        Spb = eta * ichi;
                        contrib(d, phi, chj, U, ichi, (R)0, (R)1, (R)0, Ib, wb, val, true);
                    }
                    flush(k0, val);
                }
                // profiles of the depth being swept: through the warp's ring
                // (copies issued two steps ahead), else loaded one step ahead
                constexpr bool RING = uses_ring<R, PRD, CACHE, BEZ>() && NL > 0;
                R pa[K], pb[K];
                float *rw = nullptr;   // the lane's element of the warp's ring
                int rs = 1;            // ring slot of the current step
                // issue the copies of step st's depth into ring slot sl (one
                // commit group per step, empty past the last step)
                auto ring_fill = [&](int st, int sl) {
                    if constexpr (RING) {
                        if (st < N) {
                            const int kk = dir == 0 ? st : N - 1 - st;
                            float *dst = rw + sl * kRingSlotFloats;
#pragma unroll
                            for (int j = 0; j < NL; ++j) {
                                cp_async4(dst + j * kWarp, phc + poff[j] + (ra * N + kk) * kWarp);
                                if (two) cp_async4(dst + (kRingLines + j) * kWarp, phc + poff[j] + (rb * N + kk) * kWarp);
                            }
                        }
                        cp_async_commit();
                    }
                };
                if constexpr (RING) {
                    rw = s.ring + (size_t)(threadIdx.x >> 5) * kRingFloatsPerWarp + lane;
                    ring_fill(1, 1);
                    ring_fill(2, 2);
                } else {
                    load_ph(dir == 0 ? 1 : N - 2, ra, pa);
                    if (two) load_ph(dir == 0 ? 1 : N - 2, rb, pb);
                }
                for (int step = 1; step < N; ++step) {
                    const int k = dir == 0 ? step : N - 1 - step;
                    R na[K], nb[K];
                    if constexpr (RING) {
                        cp_async_wait<1>();                 // this step's copies have landed
                        const float *sl = rw + rs * kRingSlotFloats;
#pragma unroll
                        for (int j = 0; j < K; ++j) {
                            pa[j] = j < NL ? sl[j * kWarp] : (R)0;
                            pb[j] = (j < NL && two) ? sl[(kRingLines + j) * kWarp] : (R)0;
                        }
                        // refill the slot read one step ago with step + 2
                        const int sf = rs == 0 ? kRingSlots - 1 : rs - 1;
                        ring_fill(step + 2, sf);
                        rs = rs == kRingSlots - 1 ? 0 : rs + 1;
                    } else {
                        const int kn = step + 1 < N ? (dir == 0 ? k + 1 : k - 1) : k;
                        load_ph(kn, ra, na);
                        if (two) load_ph(kn, rb, nb);
                    }
                    DepthC<R, K> d;
                    depth_consts<R, K>(s, lc, k, N, d);
                    const R dzk = dir == 0 ? s.dz[k - 1] : s.dz[k];
                    R val[P];
                    {
                        R chi, eta, phi[K], chj[K], U[K];
                        angle_vals<R, K>(lc, d, pa, chi, eta, phi, chj, U);
                        const R ichi = rcp<R>(chi);
                        const R S = eta * ichi;
                        R ome, wu, wo, omwo;
                        sc_weights((R)0.5 * (chi + chipa) * dzk * imu0, ome, wu, wo, omwo);
                        const R base = Ia * ome + wu * Spa;
                        Ia = base + wo * S;
                        chipa = chi;
                        Spa = S;
                        contrib(d, phi, chj, U, ichi, wo, omwo, wo * ichi, base + wo * (d.etabg * ichi), wa, val,
                                false);
                    }
                    if (two) {
                        R chi, eta, phi[K], chj[K], U[K];
                        angle_vals<R, K>(lc, d, pb, chi, eta, phi, chj, U);
                        const R ichi = rcp<R>(chi);
                        const R S = eta * ichi;
                        R ome, wu, wo, omwo;
                        sc_weights((R)0.5 * (chi + chipb) * dzk * imu1, ome, wu, wo, omwo);
                        const R base = Ib * ome + wu * Spb;
                        Ib = base + wo * S;
                        chipb = chi;
                        Spb = S;
                        contrib(d, phi, chj, U, ichi, wo, omwo, wo * ichi, base + wo * (d.etabg * ichi), wb, val,
                                true);
                    }
                    flush(k, val);
                    if constexpr (!RING) {
#pragma unroll
                        for (int j = 0; j < K; ++j) {
                            pa[j] = na[j];
                            pb[j] = nb[j];
                        }
                    }
                }
            }
        }
        return;
    }
#endif
    for (int m = 0; m < nmu; ++m) {
        const R mu = mu_of<R>(A, m), imu = imu_of<R>(A, m), wm2 = wm2_of<R>(A, m);
        for (int dir = 0; dir < 2; ++dir) {
            const R muz = dir == 0 ? -mu : mu;
            const int ray = 2 * m + dir;
            R I, chip = 0, Sp;
            // rho of the lane's PRD point: the static-frame ratio, or (hybrid)
            // this ray's interpolated gas-frame ratio
            const R *rl = hyb ? prd_I + ((4 * (size_t)A.nmu + ray) * A.npp + pp) * N : rho_lane;
            {
                R pc[K];
                // boundary point: I = 0 at the top; at the bottom the diffusion
                // condition, which needs chi and B one point up
                const int k0 = dir == 0 ? 0 : N - 1;
                R B2 = 0;
                if (dir == 1) {
                    DepthC<R, K> d2;
                    depth_consts<R, K, PRD>(s, lc, N - 2, N, d2, rl ? rl[N - 2] : (R)1, tl.prd_slot);
                    B2 = d2.B;
                    R phi[K], chj[K], U[K], eta;
                    load_ph(N - 2, ray, pc);
                    angle_vals<R, K, PRD>(lc, d2, pc, chip, eta, phi, chj, U);
                }
                DepthC<R, K> d;
                depth_consts<R, K, PRD>(s, lc, k0, N, d, rl ? rl[k0] : (R)1, tl.prd_slot);
                R chi, eta, phi[K], chj[K], U[K];
                load_ph(k0, ray, pc);
                angle_vals<R, K, PRD>(lc, d, pc, chi, eta, phi, chj, U);
                const R ichi = rcp<R>(chi);
                if (dir == 0) {
                    I = 0;
                } else {
                    R dtv = (R)0.5 * (chi + chip) * s.dz[N - 2];
                    I = d.B + mu * (d.B - B2) * rcp<R>(dtv);
                }
                chip = chi;
                Sp = eta * ichi;
                emit(k0, d, phi, chj, U, ichi, (R)0, (R)1, (R)0, I, I, wm2, ray);
            }
            // rho of the lane's PRD point (global scratch) loaded one depth step ahead
            R rho_nx = (PRD && rl) ? rl[dir == 0 ? 1 : N - 2] : (R)1;
            // cached profiles, like rho, loaded one depth step ahead
            R pa[K];
            load_ph(dir == 0 ? 1 : N - 2, ray, pa);
            for (int step = 1; step < N; ++step) {
                const int k = dir == 0 ? step : N - 1 - step;
                const bool has_d = step + 1 < N;   // a downwind point
                const R rho_k = rho_nx;
                if (PRD && rl && has_d) rho_nx = rl[dir == 0 ? step + 1 : N - 2 - step];
                R na[K];
                load_ph(has_d ? (dir == 0 ? k + 1 : k - 1) : k, ray, na);
                // quadratic Bezier step: the downwind point's opacity and source
                // function first (its profiles and rho are the ones loaded for
                // the next step), so that its depth terms are dead before the
                // point's own are formed
                R chid = 0, Sd = 0;
                if (bez && has_d) {   // BEZ kernels only
                    DepthC<R, K> dd;
                    depth_consts<R, K, PRD>(s, lc, dir == 0 ? k + 1 : k - 1, N, dd, rho_nx, tl.prd_slot);
                    R etad, phid[K], chjd[K], Ud[K];
                    angle_vals<R, K, PRD>(lc, dd, na, chid, etad, phid, chjd, Ud);
                    Sd = etad * rcp<R>(chid);
                }
                DepthC<R, K> d;
                depth_consts<R, K, PRD>(s, lc, k, N, d, rho_k, tl.prd_slot);
                R chi, eta, phi[K], chj[K], U[K];
                angle_vals<R, K, PRD>(lc, d, pa, chi, eta, phi, chj, U);
                const R ichi = rcp<R>(chi);
                const R S = eta * ichi;
                const R dzk = dir == 0 ? s.dz[k - 1] : s.dz[k];
                const R dtau = (R)0.5 * (chi + chip) * dzk * imu;
                R Ieff, psi, wo, omwo;
                if (bez) {
                    const R dtd = has_d ? (R)0.5 * (chid + chi) * (dir == 0 ? s.dz[k] : s.dz[k - 1]) * imu : (R)1;
                    R ex, wu, wob, wc, omp;
                    bez_weights(dtau, ex, wu, wob, wc, omp);
                    const R C = bez_control<R>(Sp, S, Sd, dtau, dtd, has_d);
                    const R base = I * ex + wu * Sp + wc * (C - S);
                    wo = wob + wc;                 // Psi* = w_o + w_c
                    omwo = omp;
                    I = base + wo * S;
                    Ieff = base + wo * (d.etabg * ichi);
                } else {
                    R ome, wu;
                    sc_weights(dtau, ome, wu, wo, omwo);
                    const R base = I * ome + wu * Sp;
                    I = base + wo * S;
                    Ieff = base + wo * (d.etabg * ichi);
                }
                psi = wo * ichi;
#pragma unroll
                for (int j = 0; j < K; ++j) pa[j] = na[j];
                chip = chi;
                Sp = S;
                emit(k, d, phi, chj, U, ichi, wo, omwo, psi, Ieff, I, wm2, ray);
            }
        }
    }
}

template <typename R, bool PRD, bool CACHE, bool BEZ>
__device__ __forceinline__ void sweep_tile(const DevAtom &A, const Smem<R> &s, const KParams &p, int b, int lane,
                                           R *prd_rho, R *prd_J, R *prd_D, R *prd_plain, R *prd_I,
                                           const R *phc)
{
    const DevTile &tl = A.tile[b];
    if constexpr (sizeof(R) == 4 && !PRD && !BEZ) {
        // the FP32 CRD instantiations (with and without the profile cache, so
        // that the two keep the same arithmetic): one tile kernel per
        // (transitions, lines)
        int nl = 0;
        for (int j = 0; j < tl.K; ++j) nl += A.tr[tl.t[j]].kind == 0;
#define RH_TILE(K_, NL_) \
    sweep_tile_k<R, K_, NL_, PRD, CACHE, BEZ>(A, s, p, b, lane, prd_rho, prd_J, prd_D, prd_plain, prd_I, phc)
        switch (tl.K * 4 + nl) {
        case 4: RH_TILE(1, 0); break;
        case 5: RH_TILE(1, 1); break;
        case 8: RH_TILE(2, 0); break;
        case 9: RH_TILE(2, 1); break;
        case 10: RH_TILE(2, 2); break;
        case 12: RH_TILE(3, 0); break;
        case 13: RH_TILE(3, 1); break;
        case 14: RH_TILE(3, 2); break;
        default: RH_TILE(3, 3); break;
        }
#undef RH_TILE
    } else {
        switch (tl.K) {
        case 1: sweep_tile_k<R, 1, -1, PRD, CACHE, BEZ>(A, s, p, b, lane, prd_rho, prd_J, prd_D, prd_plain, prd_I, phc); break;
        case 2: sweep_tile_k<R, 2, -1, PRD, CACHE, BEZ>(A, s, p, b, lane, prd_rho, prd_J, prd_D, prd_plain, prd_I, phc); break;
        default: sweep_tile_k<R, 3, -1, PRD, CACHE, BEZ>(A, s, p, b, lane, prd_rho, prd_J, prd_D, prd_plain, prd_I, phc); break;
        }
    }
}

// Hybrid PRD tables.  Interpolation over PRD line [off, last] (points sorted
// by frequency q, velocity units) at x: the bracket j in [off, last - 1] and
// weight t on point j + 1, value (1 - t) v_j + t v_{j+1}; beyond the ends
// the end value, (off, 0) or (last - 1, 1).
template <typename R>
__device__ __forceinline__ void prd_bracket(const R *qv, int off, int last, R x, int &j, R &t)
{
    if (x <= qv[off]) {
        j = off;
        t = 0;
    } else if (x >= qv[last]) {
        j = last - 1;
        t = 1;
    } else {
        int lo = off, hi = last;                   // qv[lo] <= x < qv[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (qv[mid] <= x) lo = mid;
            else hi = mid;
        }
        j = lo;
        t = (x - qv[lo]) / (qv[lo + 1] - qv[lo]);
    }
}

// weight of point i in the interpolation at x
template <typename R>
__device__ __forceinline__ R prd_weight(const R *qv, int off, int last, int i, R x)
{
    int j;
    R t;
    prd_bracket<R>(qv, off, last, x, j, t);
    return (j == i ? (R)1 - t : (R)0) + (j + 1 == i ? t : (R)0);
}

// the column's tables: threads take (ray, point, depth)
template <typename R>
__device__ void build_hybrid_tables(const DevAtom &A, const Smem<R> &s, const PrdScr<R> &ps, int N)
{
    const int nw = 2 * A.nmu * A.npp * N;
    for (int e = threadIdx.x; e < nw; e += blockDim.x) {
        const int k = e % N, rp = e / N, pt = rp % A.npp, ray = rp / A.npp;
        int q = 0;
        while (pt >= A.prd_off[q + 1]) ++q;
        const int off = A.prd_off[q], last = A.prd_off[q + 1] - 1;
        const R mu = mu_of<R>(A, ray >> 1), muz = (ray & 1) ? mu : -mu, sh = muz * s.vz[k];
        int j;
        R t;
        prd_bracket<R>(ps.q, off, last, ps.q[pt] + sh, j, t);
        ps.hj[e] = j;
        ps.ht[e] = t;
        ps.he0[e] = prd_weight<R>(ps.q, off, last, pt, ps.q[j] - sh);
        ps.he1[e] = prd_weight<R>(ps.q, off, last, pt, ps.q[j + 1] - sh);
        prd_bracket<R>(ps.q, off, last, ps.q[pt] - sh, j, t);
        ps.rj[e] = j;
        ps.rt[e] = t;
    }
}

// Hybrid PRD: each ray's rho at the PRD points, the gas-frame rho_f at the
// ray's gas-frame frequency q_p - mu_z v_z, for the sweep to read like the
// static-frame rho; threads take (ray, point, depth)
template <typename R>
__device__ void fill_rho_ray(const DevAtom &A, const PrdScr<R> &ps, int N)
{
    const int nw = 2 * A.nmu * A.npp * N;
    R *out = ps.Iray + 4 * (size_t)A.nmu * A.npp * N;
    for (int e = threadIdx.x; e < nw; e += blockDim.x) {
        const int k = e % N, j = ps.rj[e];
        const R t = ps.rt[e];
        out[e] = ((R)1 - t) * ps.rho[(size_t)j * N + k] + t * ps.rho[(size_t)(j + 1) * N + k];
    }
}

// Hybrid PRD: the gas-frame mean intensity and its local derivative at every
// PRD point and depth (threads take (point, depth)),
//   J_f(i) = sum over rays (w_mu/2) [(1 - t) I_j + t I_{j+1}],
//   D_f(i) = sum over rays (w_mu/2) [(1 - t) dI_j e0 + t dI_{j+1} e1],
// rays in the order the sweep adds the static-frame J, each product rounded
// before its sum as the sweep's accumulation does
template <typename R>
__device__ void hybrid_JD(const DevAtom &A, const PrdScr<R> &ps, int N)
{
    const size_t nt = (size_t)A.npp * N, nr = 2 * (size_t)A.nmu;
    for (int e = threadIdx.x; e < (int)nt; e += blockDim.x) {
        const int k = e % N;
        R J = 0, D = 0;
        for (int ray = 0; ray < (int)nr; ++ray) {
            const R w = wm2_of<R>(A, ray >> 1);
            const size_t x = (size_t)ray * nt + e;
            const int j = ps.hj[x];
            const R t = ps.ht[x];
            const R *Ir = ps.Iray + (size_t)ray * nt + k, *Dr = Ir + nr * nt;
            const R v = ((R)1 - t) * Ir[(size_t)j * N] + t * Ir[(size_t)(j + 1) * N];
            const R dv = ((R)1 - t) * Dr[(size_t)j * N] * ps.he0[x] + t * Dr[(size_t)(j + 1) * N] * ps.he1[x];
            J += mul_rn(w, v);
            D += mul_rn(w, dv);
        }
        ps.J[e] = J;
        ps.D[e] = D;
    }
}

// Fill the column's profile cache: warps take (row, ray) pairs, lanes their
// wavelengths, and walk the depths (the same arithmetic as the uncached sweep).
template <typename R>
__device__ void build_profiles(const DevAtom &A, const Smem<R> &s, const KParams &p, R *phc)
{
    const int N = p.N, nray = 2 * A.nmu;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const R *lt = reinterpret_cast<const R *>(p.lane);
    for (int w = threadIdx.x >> 5; w < A.nphi * nray; w += nw) {
        const int row = w / nray, r = w - row * nray;
        const int b = A.phi_tile[row], j = A.phi_j[row];
        const int pi = b * kWarp + lane;
        const R q = lt[(RH_NLANEF * j + 4) * p.npad + pi];
        const R pn = lt[(RH_NLANEF * j + 5) * p.npad + pi];
        const R mu = mu_of<R>(A, r >> 1);
        const R muz = (r & 1) ? mu : -mu;
        const R *ad = s.ad + (size_t)A.tr[A.tile[b].t[j]].sub * N;
        R *o = phc + (size_t)w * N * kWarp + lane;
        for (int k = 0; k < N; ++k) o[(size_t)k * kWarp] = line_phi(q, muz, s.vz[k], s.ivth[k], ad[k], pn, s.vtab);
    }
}

__device__ __forceinline__ double block_max(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = -1.0e308;
    for (int i = 0; i < nw; ++i) t = fmax(t, red[i]);
    __syncthreads();
    return t;
}

// Rate matrix of depth k from the accumulators and collisions; scaled LU
// solve for the new populations.  Returns 0 on success.
__device__ int solve_depth(const DevAtom &A, const double *slotd, const float *slotf, int N, int k,
                           const double *Cr, double fcr, const double *n, const double *nH, double *nn)
{
    const int L = A.nlev;
    double G[RH_MAXLEV * RH_MAXLEV];
    for (int i = 0; i < L * L; ++i) G[i] = 0.0;
    for (int e = 0; e < A.nmap; ++e) {
        const int a = A.map_acc[e];
        const double v = slotd ? slotd[a * N + k] : (double)slotf[a * N + k];
        G[A.map_row[e] * L + A.map_col[e]] += A.map_sign[e] > 0 ? v : -v;   // signs are +-1
    }
    const double *Ck = Cr + (size_t)k * 2 * A.ntr;
    for (int t = 0; t < A.ntr; ++t) {
        int l = A.tr[t].l, u = A.tr[t].u;
        G[u * L + l] += Ck[2 * t] * fcr;
        G[l * L + u] += Ck[2 * t + 1] * fcr;
    }
    for (int q = 0; q < L; ++q) {
        double s = 0.0;
        for (int pp = 0; pp < L; ++pp)
            if (pp != q) s += G[pp * L + q];
        G[q * L + q] = -s;
    }
    double sc[RH_MAXLEV], b[RH_MAXLEV];
    int r = 0;
    for (int l = 0; l < L; ++l) {
        sc[l] = n[l * N + k];
        if (sc[l] > sc[r]) r = l;
        b[l] = 0.0;
    }
    for (int q = 0; q < L; ++q) G[r * L + q] = 1.0;
    b[r] = nH[k];
    for (int pp = 0; pp < L; ++pp) {
        double mx = 0.0;
        for (int q = 0; q < L; ++q) {
            G[pp * L + q] *= sc[q];
            mx = fmax(mx, fabs(G[pp * L + q]));
        }
        if (!(mx > 0.0)) return 1;
        double im = 1.0 / mx;
        for (int q = 0; q < L; ++q) G[pp * L + q] *= im;
        b[pp] *= im;
    }
    for (int c = 0; c < L; ++c) {
        int piv = c;
        for (int rr = c + 1; rr < L; ++rr)
            if (fabs(G[rr * L + c]) > fabs(G[piv * L + c])) piv = rr;
        if (G[piv * L + c] == 0.0) return 1;
        if (piv != c) {
            for (int q = 0; q < L; ++q) {
                double t = G[c * L + q];
                G[c * L + q] = G[piv * L + q];
                G[piv * L + q] = t;
            }
            double t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        // one reciprocal per pivot (kept for the back substitution)
        const double ip = 1.0 / G[c * L + c];
        G[c * L + c] = ip;
        for (int rr = c + 1; rr < L; ++rr) {
            const double f = G[rr * L + c] * ip;
            for (int q = c + 1; q < L; ++q) G[rr * L + q] -= f * G[c * L + q];
            b[rr] -= f * b[c];
        }
    }
    for (int c = L - 1; c >= 0; --c) {
        double s = b[c];
        for (int q = c + 1; q < L; ++q) s -= G[c * L + q] * b[q];
        b[c] = s * G[c * L + c];
    }
    for (int l = 0; l < L; ++l) nn[l * N + k] = b[l] * sc[l];
    return 0;
}

// CACHE: line profiles from the per-block cache (p.phic, nullptr only for an
// atom without lines); otherwise evaluated in the sweep.  BEZ: the quadratic
// Bezier formal solver (its own instantiations, so that the linear kernels
// keep their registers)
template <typename R, bool PRD, bool CACHE, bool BEZ>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? RH_FP32_MINBLOCKS : 1) mali_kernel(const __grid_constant__ DevAtom A, const KParams p)
{
    extern __shared__ __align__(16) char smem_raw[];
    const int N = p.N, L = A.nlev;
    Smem<R> s = carve<R>(smem_raw, L, N, A.ntr, A.ncont, A.nline, A.macc,
                         uses_ring<R, PRD, CACHE, BEZ>() ? (int)(blockDim.x >> 5) : 0);
    const int tid = threadIdx.x, lane = tid & 31;
    const int LN = L * N;
    double *hist = p.nghist + (size_t)blockIdx.x * 4 * LN;

    for (int i = tid; i <= RH_VT_N; i += blockDim.x) s.vtab[i] = p.vtab[i];
    const int64_t nwork = p.nwork_d ? (int64_t)*p.nwork_d : p.nwork;
    PrdScr<R> ps{};
    if constexpr (PRD) ps = prd_carve<R>(p.prd_scr + (size_t)blockIdx.x * p.prd_stride, A, N);
    R *phc = (CACHE && p.phic) ? reinterpret_cast<R *>(p.phic + (size_t)blockIdx.x * p.phic_stride) : nullptr;
    int64_t done = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            int64_t q;
            if (p.persistent) q = atomicAdd(p.queue, 1);
            else q = (int64_t)blockIdx.x + done * gridDim.x;
            s.ibuf[0] = q < nwork ? (p.colidx ? p.colidx[q] : (int)q) : -1;
        }
        __syncthreads();
        const int col = s.ibuf[0];
        if (col < 0) break;
        ++done;
        const size_t cN = (size_t)col * N;
        // ---- load the column
        for (int k = tid; k < N; k += blockDim.x) {
            double T = p.T[cN + k];
            double ne = p.ne[cN + k];
            s.dz[k] = (R)(k < N - 1 ? fabs(p.z[cN + k] - p.z[cN + k + 1]) : 0.0);
            double vth = sqrt(2.0 * kK * T / A.mass);
            s.ivth[k] = (R)(1.0 / vth);
            s.vz[k] = (R)p.vz[cN + k];
            s.bg[4 * k + 0] = (R)(kH / (kK * T));
            double e2 = kQ * kQ / (4.0 * kPi * kEps0);
            double Cff = e2 * e2 * e2 * 4.0 / (3.0 * kMe * kH * kC) * sqrt(2.0 * kPi / (3.0 * kK * kMe));
            s.bg[4 * k + 1] = (R)(Cff * ne * p.np[cN + k] / sqrt(T) / kNuRef3);
            double n1 = p.nstar[((size_t)col * L + 0) * N + k];
            double lam3 = pow(kH * kH / (2.0 * kPi * kMe * kK * T), 1.5);
            s.bg[4 * k + 2] = (R)(0.25 * n1 * ne * lam3 * exp(0.754 * kQ / (kK * T)));
            s.bg[4 * k + 3] = (R)(kSigmaT * ne);
            double sk = N > 1 ? (double)k / (N - 1) : 0.0;
            for (int t = 0; t < A.ntr; ++t) {
                const DevTrans &tr = A.tr[t];
                if (tr.kind == 0) {
                    s.ad[tr.sub * N + k] = (R)exp((1.0 - sk) * tr.ln_atop + sk * tr.ln_abot);
                } else {
                    s.Gc[tr.sub * N + k] = (R)(p.nstar[((size_t)col * L + tr.l) * N + k] /
                                               p.nstar[((size_t)col * L + tr.u) * N + k]);
                }
            }
        }
        for (int i = tid; i < N * 2 * A.ntr; i += blockDim.x) s.Cr[i] = p.Crate[(size_t)col * N * 2 * A.ntr + i];
        if (phc) {
            __syncthreads();   // the column's Doppler widths, velocities and damping
            build_profiles<R>(A, s, p, phc);
        }
        if constexpr (PRD) {
            // redistribution kernels of the column: K_ij = R(x_j, x_i) w_j / sum_j (.),
            // x in Doppler units of the depth (static frame), and the J-bar weights
            // f_j = H(a, x_j) w_j / sum_j (.); x and a per point and depth first
            for (int e = tid; e < A.npp * N; e += blockDim.x) {
                const int pp = e / N, k = e % N;
                int q = 0;
                while (pp >= A.prd_off[q + 1]) ++q;
                const DevTrans &tr = A.tr[A.prd_t[q]];
                const double dnuD = tr.nu0 / kC * sqrt(2.0 * kK * p.T[cN + k] / A.mass);
                ps.x[e] = (R)((p.prd_nu[pp] - tr.nu0) / dnuD);
            }
            for (int pp = tid; pp < A.npp; pp += blockDim.x) {
                int q = 0;
                while (pp >= A.prd_off[q + 1]) ++q;
                const double nu0 = A.tr[A.prd_t[q]].nu0;
                ps.q[pp] = (R)(kC * (p.prd_nu[pp] - nu0) / nu0);
            }
            for (int e = tid; e < A.nprd * N; e += blockDim.x) {
                const int q = e / N, k = e % N;
                const DevTrans &tr = A.tr[A.prd_t[q]];
                const double sk = N > 1 ? (double)k / (N - 1) : 0.0;
                ps.a[e] = (R)exp((1.0 - sk) * tr.ln_atop + sk * tr.ln_abot);
            }
            __syncthreads();
            if (p.prd_hybrid) build_hybrid_tables<R>(A, s, ps, N);   // read after later barriers
            for (int q = 0; q < A.nprd; ++q) {
                const int off = A.prd_off[q], np = A.prd_off[q + 1] - off, npair = np * (np + 1) / 2;
                R *Kq = ps.K + (size_t)A.prd_koff[q] * N;
                // R is symmetric: one evaluation per unordered pair (i <= j), pairs
                // numbered row by row, p = i np - i (i - 1) / 2 + (j - i)
                for (int e = tid; e < npair * N; e += blockDim.x) {
                    const int k = e / npair, pr = e % npair;
                    int i = (int)((2.0f * np + 1.0f - sqrtf((2.0f * np + 1.0f) * (2.0f * np + 1.0f) - 8.0f * pr)) * 0.5f);
                    while (i > 0 && i * np - i * (i - 1) / 2 > pr) --i;
                    while ((i + 1) * np - (i + 1) * i / 2 <= pr) ++i;
                    const int j = i + pr - (i * np - i * (i - 1) / 2);
                    const R ak = ps.a[q * N + k];
                    const R rv = r2a_dev<R>(ak, ps.x[(size_t)(off + j) * N + k], ps.x[(size_t)(off + i) * N + k]);
                    Kq[((size_t)k * np + j) * np + i] = rv * (R)p.prd_w[off + j];     // K_ij
                    Kq[((size_t)k * np + i) * np + j] = rv * (R)p.prd_w[off + i];     // K_ji
                }
            }
            __syncthreads();
            for (int q = 0; q < A.nprd; ++q) {
                const int off = A.prd_off[q], np = A.prd_off[q + 1] - off;
                R *Kq = ps.K + (size_t)A.prd_koff[q] * N;
                for (int e = tid; e < np * N; e += blockDim.x) {
                    const int k = e / np, i = e % np;
                    R *col = Kq + (size_t)k * np * np + i;                    // K_ij at col[j np]
                    R sr = 0;
                    for (int j = 0; j < np; ++j) sr += col[(size_t)j * np];
                    const R inv = (R)1 / sr;
                    for (int j = 0; j < np; ++j) col[(size_t)j * np] *= inv;
                }
                for (int k = tid; k < N; k += blockDim.x) {
                    const R ak = ps.a[q * N + k];
                    R fs = 0;
                    for (int j = 0; j < np; ++j) {
                        const R v = voigt<R>(ak, ps.x[(size_t)(off + j) * N + k], s.vtab) * (R)p.prd_w[off + j];
                        ps.f[(size_t)(off + j) * N + k] = v;
                        fs += v;
                    }
                    const R inv = (R)1 / fs;
                    for (int j = 0; j < np; ++j) ps.f[(size_t)(off + j) * N + k] *= inv;
                }
            }
        }
        int start = p.start, ng_order = p.ng_order, maxiter = p.maxiter, rung = 0;
        double crsw = p.crsw;
        int it = 0, status = RH_COL_MAXITER;
        double dmax = 1e300;
      restart:
        if constexpr (PRD) {
            for (int i = tid; i < A.npp * N; i += blockDim.x) ps.rho[i] = 1;   // PRD starts as CRD
            if (p.prd_hybrid) {
                __syncthreads();
                fill_rho_ray<R>(A, ps, N);
            }
        }
        for (int i = tid; i < LN; i += blockDim.x) {
            double v = start == 0 ? p.nstar[(size_t)col * LN + i] : p.pops[(size_t)col * LN + i];
            s.n[i] = v;
        }
        int hcount = 0, hpos = 0, rcount = 0, rpos = 0;
        status = RH_COL_MAXITER;
        dmax = 1e300;
        for (it = 1; it <= maxiter; ++it) {
            double fcr = crsw > 1.0 ? fmax(1.0, crsw * pow(10.0, -(double)(it - 1))) : 1.0;
            for (int i = tid; i < LN; i += blockDim.x) s.nr[i] = (R)(s.n[i] * p.inv_nref);
            for (int i = tid; i < A.macc * N; i += blockDim.x) s.slot[i] = 0;
            if constexpr (PRD) {
                for (int i = tid; i < A.npp * N; i += blockDim.x) {
                    ps.J[i] = 0;
                    ps.D[i] = 0;
                }
                for (int i = tid; i < A.pacc * N; i += blockDim.x) ps.plain[i] = 0;
            }
            if (tid == 0) s.ibuf[1] = 0;
            __syncthreads();
            // ---- formal solution and rate accumulation: warps take tiles from a
            // block-local queue, most expensive tiles first
            for (;;) {
                int q = 0;
                if (lane == 0) q = atomicAdd(&s.ibuf[1], 1);
                q = __shfl_sync(0xffffffffu, q, 0);
                if (q >= A.ntile) break;
                sweep_tile<R, PRD, CACHE, BEZ>(A, s, p, A.order[q], lane, ps.rho, ps.J, ps.D, ps.plain,
                                          p.prd_hybrid ? ps.Iray : nullptr, phc);
            }
            __syncthreads();
            // ---- rate equations, one thread per depth
            int bad = 0;
            double dloc = 0.0;
            for (int k = tid; k < N; k += blockDim.x) {
                int e = solve_depth(A, sizeof(R) == 8 ? reinterpret_cast<const double *>(s.slot) : nullptr,
                                    sizeof(R) == 4 ? reinterpret_cast<const float *>(s.slot) : nullptr, N, k,
                                    s.Cr, fcr, s.n, p.nH + cN, s.nn);
                if (e) bad = 2;
                for (int l = 0; l < L && !e; ++l) {
                    double a = s.nn[l * N + k];
                    if (!(isfinite(a) && a > 0.0)) {
                        bad = bad ? bad : 1;
                        break;
                    }
                    dloc = fmax(dloc, fabs(a - s.n[l * N + k]) / a);
                }
            }
            double badg = block_max((double)bad, s.red);
            dmax = block_max(dloc, s.red);
            if (badg > 0) {
                status = badg > 1.5 ? RH_COL_SINGULAR : RH_COL_NONFINITE;
                break;
            }
            const bool conv = dmax < p.tol && fcr == 1.0;
            // ---- Ng history (newest first, ring of 4)
            hpos = (hpos + 3) & 3;
            for (int i = tid; i < LN; i += blockDim.x) hist[(size_t)hpos * LN + i] = s.nn[i];
            __syncthreads();
            if (hcount < 4) ++hcount;
            if (!conv && ng_order == 2 && it >= p.ng_delay && hcount >= 4 &&
                (it - p.ng_delay) % p.ng_period == 0) {
                const double *x0 = hist + (size_t)hpos * LN, *x1 = hist + (size_t)((hpos + 1) & 3) * LN,
                             *x2 = hist + (size_t)((hpos + 2) & 3) * LN, *x3 = hist + (size_t)((hpos + 3) & 3) * LN;
                // dot products over a fixed partition of kNgLanes partial sums,
                // added in a fixed order: the result does not depend on the
                // block size
                for (int v = tid; v < kNgLanes; v += blockDim.x) {
                    double q[5] = {0, 0, 0, 0, 0};
                    for (int i = v; i < LN; i += kNgLanes) {
                        double d0 = x0[i] - x1[i], d1 = x1[i] - x2[i], d2 = x2[i] - x3[i];
                        double pp = d0 - d1, qq = d0 - d2;
                        q[0] += pp * pp;
                        q[1] += pp * qq;
                        q[2] += qq * qq;
                        q[3] += d0 * pp;
                        q[4] += d0 * qq;
                    }
                    for (int j = 0; j < 5; ++j) s.red[j * kNgLanes + v] = q[j];
                }
                __syncthreads();
                if (tid < 5) {
                    double t = 0.0;
                    for (int i = 0; i < kNgLanes; ++i) t += s.red[tid * kNgLanes + i];
                    s.red[5 * kNgLanes + tid] = t;
                }
                __syncthreads();
                const double a11 = s.red[5 * kNgLanes + 0], a12 = s.red[5 * kNgLanes + 1],
                             a22 = s.red[5 * kNgLanes + 2], b1 = s.red[5 * kNgLanes + 3],
                             b2 = s.red[5 * kNgLanes + 4];
                __syncthreads();
                double det = a11 * a22 - a12 * a12;
                if (fabs(det) > 0.0 && isfinite(det)) {
                    double ca = (b1 * a22 - b2 * a12) / det, cb = (a11 * b2 - a12 * b1) / det;
                    int okl = 1;
                    for (int i = tid; i < LN; i += blockDim.x) {
                        double v = (1.0 - ca - cb) * x0[i] + ca * x1[i] + cb * x2[i];
                        if (!(isfinite(v) && v > 0.0)) okl = 0;
                    }
                    double ok = -block_max(-(double)okl, s.red);
                    if (ok > 0.5) {
                        for (int i = tid; i < LN; i += blockDim.x) {
                            double v = (1.0 - ca - cb) * x0[i] + ca * x1[i] + cb * x2[i];
                            s.nn[i] = v;
                        }
                        __syncthreads();
                        for (int i = tid; i < LN; i += blockDim.x) hist[(size_t)hpos * LN + i] = s.nn[i];
                        hcount = 1;
                    }
                }
            }
            __syncthreads();
            for (int i = tid; i < LN; i += blockDim.x) s.n[i] = s.nn[i];
            __syncthreads();
            if (conv) {
                status = RH_COL_CONVERGED;
                break;
            }
            if constexpr (PRD) {
                // rho for the next iteration (Uitenbroek 2001, Eq. 14, angle-averaged,
                // gamma = 1): r = 1 + F (sum_j K_ij J_j / Jbar - 1), F = n_l R_lu /
                // (supply of the upper level) with the plain rates of this formal
                // solution and the collisions, n the next iteration's populations;
                // PRD switching (Eq. 1) r' = eps r + (1 - eps), eps = min(1, eps0
                // it^2) of the iteration that uses it
                const double eps =
                    p.prd_eps0 > 0.0 ? fmin(1.0, p.prd_eps0 * (double)(it + 1) * (double)(it + 1)) : 1.0;
                if (p.prd_hybrid) {
                    hybrid_JD<R>(A, ps, N);   // the gas-frame J and D in place of the sweep's
                    __syncthreads();
                }
                for (int e = tid; e < A.nprd * N; e += blockDim.x) {
                    const int q = e / N, k = e % N, tq = A.prd_t[q];
                    const int u = A.tr[tq].u, l = A.tr[tq].l;
                    double in = 0.0, up_line = 0.0;
                    for (int b = 0; b < A.ntile; ++b) {
                        const DevTile &tb = A.tile[b];
                        for (int j = 0; j < tb.K; ++j) {
                            const DevTrans &t2 = A.tr[tb.t[j]];
                            const double pu = (double)ps.plain[(size_t)(tb.pacc_off + 2 * j) * N + k];
                            const double pd = (double)ps.plain[(size_t)(tb.pacc_off + 2 * j + 1) * N + k];
                            if (t2.u == u) in += s.n[t2.l * N + k] * pu;
                            if (t2.l == u) in += s.n[t2.u * N + k] * pd;
                            if (tb.t[j] == tq) up_line += pu;
                        }
                    }
                    const double *Ck = s.Cr + (size_t)k * 2 * A.ntr;
                    for (int t = 0; t < A.ntr; ++t) {
                        if (A.tr[t].u == u) in += s.n[A.tr[t].l * N + k] * Ck[2 * t] * fcr;
                        if (A.tr[t].l == u) in += s.n[A.tr[t].u * N + k] * Ck[2 * t + 1] * fcr;
                    }
                    ps.F[e] = s.n[l * N + k] * up_line / in;
                    const int off = A.prd_off[q], np = A.prd_off[q + 1] - off;
                    R jb = 0;
                    for (int j = 0; j < np; ++j) jb += ps.f[(size_t)(off + j) * N + k] * ps.J[(size_t)(off + j) * N + k];
                    ps.Jbar[e] = (double)jb;
                }
                __syncthreads();
                // with Ng: one Jacobi step rho += (r' - rho) / max(1 - eps g_ii, 0.02),
                // g_ii = dr_i/drho_i = F D_i (K_ii - f_i sum_j K_ij J_j / Jbar) / Jbar,
                // and Ng on the rho sequence; without Ng: rho = (rho + r') / 2
                const bool jac = ng_order == 2;
                rpos = (rpos + 3) & 3;
                double *rh0 = ps.hist + (size_t)rpos * A.npp * N;
                // threads own (depth, point) with the point fastest: K_ij of
                // consecutive points i at consecutive addresses, J_j shared.  In
                // FP32, with np a multiple of 4, a thread owns four consecutive
                // points and streams K as float4 with eight rows in flight (the
                // sum is memory-latency-bound otherwise); the sums run over j in
                // the same order either way.
                for (int q = 0; q < A.nprd; ++q) {
                    const int off = A.prd_off[q], np = A.prd_off[q + 1] - off;
                    const R *Kq = ps.K + (size_t)A.prd_koff[q] * N;
                    const bool vec = sizeof(R) == 4 && (np & 3) == 0 && (A.prd_koff[q] & 3) == 0;
                    const int G = vec ? 4 : 1, ng = np / G;
                    for (int e = tid; e < ng * N; e += blockDim.x) {
                        const int k = e / ng, i0 = (e % ng) * G;
                        const R *col = Kq + (size_t)k * np * np + i0;
                        const R *Jk = ps.J + (size_t)off * N + k;
                        R sr[4] = {0, 0, 0, 0};
                        if constexpr (sizeof(R) == 4) {
                            if (vec) {
                                float4 acc[2] = {make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0)};
                                int j = 0;
                                for (; j + 8 <= np; j += 8) {
                                    float4 kv[8];
                                    float jv[8];
#pragma unroll
                                    for (int u = 0; u < 8; ++u) {
                                        kv[u] = *reinterpret_cast<const float4 *>(col + (size_t)(j + u) * np);
                                        jv[u] = Jk[(size_t)(j + u) * N];
                                    }
#pragma unroll
                                    for (int u = 0; u < 8; ++u) {
                                        float4 &a4 = acc[u & 1];
                                        a4.x += kv[u].x * jv[u];
                                        a4.y += kv[u].y * jv[u];
                                        a4.z += kv[u].z * jv[u];
                                        a4.w += kv[u].w * jv[u];
                                    }
                                }
                                for (; j < np; ++j) {
                                    const float4 kv = *reinterpret_cast<const float4 *>(col + (size_t)j * np);
                                    const float jv = Jk[(size_t)j * N];
                                    acc[0].x += kv.x * jv;
                                    acc[0].y += kv.y * jv;
                                    acc[0].z += kv.z * jv;
                                    acc[0].w += kv.w * jv;
                                }
                                sr[0] = acc[0].x + acc[1].x;
                                sr[1] = acc[0].y + acc[1].y;
                                sr[2] = acc[0].z + acc[1].z;
                                sr[3] = acc[0].w + acc[1].w;
                            }
                        }
                        if (!vec) {
                            // eight independent partial sums, added in a fixed order
                            R part[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                            int j = 0;
                            for (; j + 8 <= np; j += 8) {
#pragma unroll
                                for (int u = 0; u < 8; ++u)
                                    part[u] += col[(size_t)(j + u) * np] * Jk[(size_t)(j + u) * N];
                            }
                            for (; j < np; ++j) part[0] += col[(size_t)j * np] * Jk[(size_t)j * N];
                            sr[0] = ((part[0] + part[1]) + (part[2] + part[3])) + ((part[4] + part[5]) + (part[6] + part[7]));
                        }
                        const R jb = (R)ps.Jbar[q * N + k], F = (R)ps.F[q * N + k], ep = (R)eps;
#pragma unroll
                        for (int g = 0; g < 4; ++g) {
                            if (g >= G) break;
                            const int i = i0 + g, pe = (off + i) * N + k;
                            const R r = (R)1 + F * (sr[g] / jb - (R)1);
                            R den = 2;
                            if (jac) {
                                const R gi = F * (Kq[((size_t)k * np + i) * np + i] - ps.f[pe] * sr[g] / jb) * ps.D[pe] / jb;
                                den = (R)1 - ep * gi;
                                den = den > (R)0.02 ? den : (R)0.02;
                            }
                            ps.rho[pe] += ((ep * r + ((R)1 - ep)) - ps.rho[pe]) / den;
                            rh0[pe] = (double)ps.rho[pe];
                        }
                    }
                }
                __syncthreads();
                if (rcount < 4) ++rcount;
                if (jac && it >= p.ng_delay && rcount >= 4 && (it - p.ng_delay) % p.ng_period == 0) {
                    const int RV = A.npp * N;
                    const double *x0 = rh0, *x1 = ps.hist + (size_t)((rpos + 1) & 3) * RV,
                                 *x2 = ps.hist + (size_t)((rpos + 2) & 3) * RV,
                                 *x3 = ps.hist + (size_t)((rpos + 3) & 3) * RV;
                    for (int v = tid; v < kNgLanes; v += blockDim.x) {
                        double q5[5] = {0, 0, 0, 0, 0};
                        for (int i = v; i < RV; i += kNgLanes) {
                            double d0 = x0[i] - x1[i], d1 = x1[i] - x2[i], d2 = x2[i] - x3[i];
                            double pq = d0 - d1, qq = d0 - d2;
                            q5[0] += pq * pq;
                            q5[1] += pq * qq;
                            q5[2] += qq * qq;
                            q5[3] += d0 * pq;
                            q5[4] += d0 * qq;
                        }
                        for (int j = 0; j < 5; ++j) s.red[j * kNgLanes + v] = q5[j];
                    }
                    __syncthreads();
                    if (tid < 5) {
                        double t = 0.0;
                        for (int i = 0; i < kNgLanes; ++i) t += s.red[tid * kNgLanes + i];
                        s.red[5 * kNgLanes + tid] = t;
                    }
                    __syncthreads();
                    const double a11 = s.red[5 * kNgLanes + 0], a12 = s.red[5 * kNgLanes + 1],
                                 a22 = s.red[5 * kNgLanes + 2], b1 = s.red[5 * kNgLanes + 3],
                                 b2 = s.red[5 * kNgLanes + 4];
                    __syncthreads();
                    const double det = a11 * a22 - a12 * a12;
                    if (fabs(det) > 0.0 && isfinite(det)) {
                        const double ca = (b1 * a22 - b2 * a12) / det, cb = (a11 * b2 - a12 * b1) / det;
                        int okl = 1;
                        for (int i = tid; i < RV; i += blockDim.x) {
                            const double v = (1.0 - ca - cb) * x0[i] + ca * x1[i] + cb * x2[i];
                            if (!(isfinite(v) && v >= 0.0)) okl = 0;
                        }
                        const double ok = -block_max(-(double)okl, s.red);
                        if (ok > 0.5) {
                            for (int i = tid; i < RV; i += blockDim.x) {
                                const double v = (1.0 - ca - cb) * x0[i] + ca * x1[i] + cb * x2[i];
                                ps.rho[i] = (R)v;
                                rh0[i] = (double)ps.rho[i];
                            }
                            rcount = 1;
                        }
                    }
                }
                __syncthreads();
                if (p.prd_hybrid) fill_rho_ray<R>(A, ps, N);   // read after the next barrier
            }
        }
        if (it > maxiter) it = maxiter;
        if (tid == 0 && p.rung_its) atomicAdd(&p.rung_its[rung], (unsigned long long)it);
        if (status != RH_COL_CONVERGED && rung < p.nrung) {
            // next rung of the re-run ladder: from LTE, its own switching and Ng
            start = 0;
            ng_order = p.rung_ng[rung];
            crsw = p.rung_crsw[rung];
            maxiter = p.rung_maxiter;
            ++rung;
            if (tid == 0 && p.rung_cols) atomicAdd(&p.rung_cols[rung - 1], 1);
            __syncthreads();
            goto restart;
        }
        for (int i = tid; i < LN; i += blockDim.x) p.pops[(size_t)col * LN + i] = s.n[i];
        if (tid == 0) {
            p.iters[col] = it;
            p.status[col] = (uint8_t)status;
            p.dmax[col] = dmax;
        }
    }
}

}  // namespace

size_t mali_nghist_bytes_per_block(const DevAtom &A, int ndep) { return sizeof(double) * 4 * A.nlev * ndep; }

// the column kernel's shared-memory layout for the given sizes: its byte
// offsets in carve order and the allocated size (host computation only)
int mali_smem_layout(int precision, int L, int N, int ntr, int ncont, int nline, int macc, int ring_warps,
                     size_t *offsets, int noff, size_t *bytes)
{
    const SmemLayout o = precision == 1 ? smem_layout<float>(L, N, ntr, ncont, nline, macc, ring_warps)
                                        : smem_layout<double>(L, N, ntr, ncont, nline, macc, ring_warps);
    const size_t v[16] = {o.n,  o.nn, o.Cr, o.red,  o.slot, o.dz,   o.ivth, o.vz,
                          o.bg, o.Gc, o.ad, o.nr,   o.vtab, o.ibuf, o.ring, o.end};
    for (int i = 0; i < noff && i < 16; ++i) offsets[i] = v[i];
    *bytes = precision == 1 ? smem_bytes<float>(L, N, ntr, ncont, nline, macc, ring_warps)
                            : smem_bytes<double>(L, N, ntr, ncont, nline, macc, ring_warps);
    return 16;
}

size_t mali_phic_bytes_per_block(const DevAtom &A, int ndep, int precision)
{
    return precision == 1 ? phic_bytes<float>(A, ndep) : phic_bytes<double>(A, ndep);
}

size_t mali_prd_bytes_per_block(const DevAtom &A, int ndep, int precision)
{
    if (!A.nprd) return 0;
    return precision == 1 ? prd_bytes<float>(A, ndep) : prd_bytes<double>(A, ndep);
}

// the column kernel for (PRD lines, profile cache, Bezier solver); the
// Bezier kernels exist with the profile cache only (nullptr otherwise)
template <typename R>
static void (*pick_kernel(bool prd, bool cache, bool bez))(DevAtom, KParams)
{
    if (prd) return bez ? mali_kernel<R, true, true, true> : mali_kernel<R, true, true, false>;
    if (cache) return bez ? mali_kernel<R, false, true, true> : mali_kernel<R, false, true, false>;
    return bez ? nullptr : mali_kernel<R, false, false, false>;
}

// resident blocks per SM of the linear solver's kernel (a launch with the
// Bezier solver takes its own kernel's occupancy)
int mali_max_ctas_per_sm(const DevAtom &A, int ndep, int precision, int block_warps)
{
    size_t sm;
    const void *fn;
    if (precision == 1) {
        sm = smem_bytes<float>(A.nlev, ndep, A.ntr, A.ncont, A.nline, A.macc,
                               A.nprd ? 0 : (uses_ring<float, false, true, false>() ? block_warps : 0));
        fn = (const void *)pick_kernel<float>(A.nprd > 0, true, false);
    } else {
        sm = smem_bytes<double>(A.nlev, ndep, A.ntr, A.ncont, A.nline, A.macc, 0);
        fn = (const void *)pick_kernel<double>(A.nprd > 0, true, false);
    }
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block_warps * 32, sm) != cudaSuccess) return 0;
    return per_sm;
}

template <typename R>
static cudaError_t launch_t(const DevAtom &A, const KParams &p, int block_warps, int ctas_per_sm, int nsm, size_t cap,
                            size_t prd_cap, size_t phic_cap, cudaStream_t st, float *ms, char *err, size_t errn,
                            int *grid_out)
{
    const bool bez = p.formal == 1;
    const int ring_warps = !A.nprd && !bez && uses_ring<R, false, true, false>() ? block_warps : 0;
    size_t sm = smem_bytes<R>(A.nlev, p.N, A.ntr, A.ncont, A.nline, A.macc, ring_warps);
    if (A.nphi && !p.phic) {
        snprintf(err, errn, "no profile cache");
        return cudaErrorInvalidValue;
    }
    auto kern = pick_kernel<R>(A.nprd > 0, true, bez);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int threads = block_warps * 32;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) {
        snprintf(err, errn, "column kernel does not fit: %zu B shared memory, %d threads", sm, threads);
        return cudaErrorInvalidConfiguration;
    }
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    int64_t grid = (int64_t)per_sm * nsm;
    if (!p.nwork_d && grid > p.nwork) grid = p.nwork;
    size_t per_block = mali_nghist_bytes_per_block(A, p.N);
    if ((size_t)grid * per_block > cap) grid = (int64_t)(cap / per_block);
    if (A.nprd && (size_t)grid * p.prd_stride > prd_cap) grid = (int64_t)(prd_cap / p.prd_stride);
    if (p.phic && (size_t)grid * p.phic_stride > phic_cap) grid = (int64_t)(phic_cap / p.phic_stride);
    if (grid < 1) {
        snprintf(err, errn, "no scratch for the Ng history");
        return cudaErrorMemoryAllocation;
    }
    *grid_out = (int)grid;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    kern<<<(unsigned)grid, threads, sm, st>>>(A, p);
    e = cudaGetLastError();
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess && ms) cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

cudaError_t launch_mali(const DevAtom &A, const ColumnArrays &c, const void *lane_tab, int npad, const float4 *vtab,
                        double nref, double *nghist, size_t nghist_cap, int *queue, const IterLaunch &o,
                        cudaStream_t st, float *ms_out, int *grid_out, char *err, size_t errn)
{
    KParams p;
    p.ncol = c.ncol;
    p.N = c.ndep;
    p.L = A.nlev;
    p.z = c.z;
    p.T = c.T;
    p.nH = c.nH;
    p.vz = c.vz;
    p.ne = c.ne;
    p.np = c.np;
    p.nstar = c.nstar;
    p.Crate = c.Crate;
    p.pops = c.pops;
    p.dmax = c.dmax;
    p.iters = c.iters;
    p.status = c.status;
    p.lane = lane_tab;
    p.npad = npad;
    p.vtab = vtab;
    p.nghist = nghist;
    p.queue = queue;
    p.persistent = o.persistent;
    p.maxiter = o.maxiter;
    p.ng_order = o.ng_order;
    p.ng_delay = o.ng_delay;
    p.ng_period = o.ng_period;
    p.start = o.start;
    p.tol = o.tol;
    p.crsw = o.crsw;
    p.inv_nref = 1.0 / nref;
    p.colidx = o.colidx;
    p.nwork = o.nwork;
    p.nwork_d = o.nwork_d;
    p.nrung = o.nrung;
    p.rung_maxiter = o.rung_maxiter;
    for (int r = 0; r < RH_MAX_RERUN; ++r) {
        p.rung_crsw[r] = o.rung_crsw[r];
        p.rung_ng[r] = o.rung_ng[r];
    }
    p.rung_cols = o.rung_cols;
    p.rung_its = o.rung_its;
    p.prd_eps0 = o.prd_eps0;
    p.prd_hybrid = o.prd_hybrid;
    p.formal = o.formal;
    p.lane_prd = o.lane_prd;
    p.prd_nu = o.prd_nu;
    p.prd_w = o.prd_w;
    p.prd_scr = reinterpret_cast<char *>(o.prd_scr);
    p.prd_stride = A.nprd ? (o.precision == 1 ? prd_bytes<float>(A, c.ndep) : prd_bytes<double>(A, c.ndep)) : 0;
    p.phic_stride = o.precision == 1 ? phic_bytes<float>(A, c.ndep) : phic_bytes<double>(A, c.ndep);
    p.phic = (o.phic && p.phic_stride && p.phic_stride <= o.phic_cap) ? reinterpret_cast<char *>(o.phic) : nullptr;
    int bw = o.block_warps > 0 ? o.block_warps : (o.precision ? 8 : 4);
    if (o.persistent) {
        cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
    }
    if (o.precision == 1)
        return launch_t<float>(A, p, bw, o.ctas_per_sm, o.nsm, nghist_cap, o.prd_cap, o.phic_cap, st, ms_out, err,
                               errn, grid_out);
    return launch_t<double>(A, p, bw, o.ctas_per_sm, o.nsm, nghist_cap, o.prd_cap, o.phic_cap, st, ms_out, err, errn,
                            grid_out);
}

}  // namespace rh

// ----------------------------------------------------------------------------
// Launcher for callers that must not allocate: the same kernel, no timing
// events (event objects are driver allocations), scratch pointers supplied
// by the caller.  Grid size is clamped to the Ng-history capacity.
namespace rh {

cudaError_t launch_mali_prealloc(const DevAtom &A, const ColumnArrays &c, const void *lane_tab, int npad,
                                 const float4 *vtab, double nref, double *nghist, size_t nghist_cap, int *queue,
                                 const IterLaunch &o, cudaStream_t st, int *grid_out, char *err, size_t errn)
{
    KParams p;
    p.ncol = c.ncol;
    p.N = c.ndep;
    p.L = A.nlev;
    p.z = c.z;
    p.T = c.T;
    p.nH = c.nH;
    p.vz = c.vz;
    p.ne = c.ne;
    p.np = c.np;
    p.nstar = c.nstar;
    p.Crate = c.Crate;
    p.pops = c.pops;
    p.dmax = c.dmax;
    p.iters = c.iters;
    p.status = c.status;
    p.lane = lane_tab;
    p.npad = npad;
    p.vtab = vtab;
    p.nghist = nghist;
    p.queue = queue;
    p.persistent = o.persistent;
    p.maxiter = o.maxiter;
    p.ng_order = o.ng_order;
    p.ng_delay = o.ng_delay;
    p.ng_period = o.ng_period;
    p.start = o.start;
    p.tol = o.tol;
    p.crsw = o.crsw;
    p.inv_nref = 1.0 / nref;
    p.colidx = o.colidx;
    p.nwork = o.nwork;
    p.nwork_d = o.nwork_d;
    p.nrung = o.nrung;
    p.rung_maxiter = o.rung_maxiter;
    for (int r = 0; r < RH_MAX_RERUN; ++r) {
        p.rung_crsw[r] = o.rung_crsw[r];
        p.rung_ng[r] = o.rung_ng[r];
    }
    p.rung_cols = o.rung_cols;
    p.rung_its = o.rung_its;
    p.prd_eps0 = o.prd_eps0;
    p.prd_hybrid = o.prd_hybrid;
    p.formal = o.formal;
    p.lane_prd = o.lane_prd;
    p.prd_nu = o.prd_nu;
    p.prd_w = o.prd_w;
    p.prd_scr = reinterpret_cast<char *>(o.prd_scr);
    p.prd_stride = A.nprd ? (o.precision == 1 ? prd_bytes<float>(A, c.ndep) : prd_bytes<double>(A, c.ndep)) : 0;
    p.phic_stride = o.precision == 1 ? phic_bytes<float>(A, c.ndep) : phic_bytes<double>(A, c.ndep);
    p.phic = (o.phic && p.phic_stride && p.phic_stride <= o.phic_cap) ? reinterpret_cast<char *>(o.phic) : nullptr;
    const int bw = o.block_warps > 0 ? o.block_warps : (o.precision ? 8 : 4);
    const int threads = bw * 32;
    size_t sm;
    const void *fn;
    // without a profile cache (callers that cannot allocate) the sweep
    // evaluates the profiles; partial redistribution always has the cache
    const bool cache = p.phic || !A.nphi;
    if (!cache && A.nprd) {
        snprintf(err, errn, "the partial-redistribution kernel needs the profile cache");
        return cudaErrorInvalidValue;
    }
    const bool bez = o.formal == 1;
    if (bez && !cache) {
        snprintf(err, errn, "the Bezier formal solver needs the profile cache (an earlier rh_iterate or rh_solve)");
        return cudaErrorInvalidValue;
    }
    if (o.precision == 1) {
        sm = smem_bytes<float>(A.nlev, p.N, A.ntr, A.ncont, A.nline, A.macc,
                               (!A.nprd && cache && !bez && uses_ring<float, false, true, false>()) ? bw : 0);
        fn = (const void *)pick_kernel<float>(A.nprd > 0, cache, bez);
    } else {
        sm = smem_bytes<double>(A.nlev, p.N, A.ntr, A.ncont, A.nline, A.macc, 0);
        fn = (const void *)pick_kernel<double>(A.nprd > 0, cache, bez);
    }
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) {
        snprintf(err, errn, "column kernel does not fit: %zu B shared memory, %d threads", sm, threads);
        return cudaErrorInvalidConfiguration;
    }
    if (o.ctas_per_sm > 0 && o.ctas_per_sm < per_sm) per_sm = o.ctas_per_sm;
    int64_t grid = (int64_t)per_sm * o.nsm;
    if (!p.nwork_d && grid > p.nwork) grid = p.nwork;
    const size_t per_block = mali_nghist_bytes_per_block(A, p.N);
    if ((size_t)grid * per_block > nghist_cap) grid = (int64_t)(nghist_cap / per_block);
    if (A.nprd && (size_t)grid * p.prd_stride > o.prd_cap) grid = (int64_t)(o.prd_cap / p.prd_stride);
    if (p.phic && (size_t)grid * p.phic_stride > o.phic_cap) grid = (int64_t)(o.phic_cap / p.phic_stride);
    if (grid < 1) {
        snprintf(err, errn, "Ng history of one column (%zu B) exceeds the scratch capacity (%zu B)", per_block,
                 nghist_cap);
        return cudaErrorInvalidValue;
    }
    *grid_out = (int)grid;
    if (o.persistent) {
        e = cudaMemsetAsync(queue, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
    }
    void *args[] = {(void *)&A, (void *)&p};
    e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(threads), args, sm, st);
    return e;
}

}  // namespace rh
