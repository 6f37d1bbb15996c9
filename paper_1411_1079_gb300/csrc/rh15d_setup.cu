// rh15d_setup.cu -- per-depth set-up (LTE start, Sect. 2.3) and the emergent
// spectrum (Sect. 2.2) kernels.
#include "rh15d_internal.h"

namespace rh {

namespace {

// One thread per (column, depth): electron density (hydrogen Saha with a
// metal electron floor, unless given), LTE populations (Saha-Boltzmann of the
// model atom), LTE start populations, and collisional rates:
//   bound-bound van Regemorter: C_lu = n_e K Omega / (g_l sqrt T) e^{-y},
//     K = h^2 / ((2 pi m_e)^{3/2} sqrt k), Omega = (8 pi / sqrt 3)(E_H/dE) g_l f P(y),
//     P = max(0.2, 0.276 e^y E1(y));
//   bound-free Seaton: C_lc = 1.55e11 n_e alpha0 0.1 e^{-u} / (u sqrt T) (SI);
//   downward rates by detailed balance with the LTE populations.
__global__ void lte_setup_kernel(const __grid_constant__ DevAtom A, ColumnArrays c, int ne_given)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int N = c.ndep, L = A.nlev;
    if (idx >= c.ncol * N) return;
    const int64_t col = idx / N;
    const int k = (int)(idx % N);
    const double T = c.T[idx], nH = c.nH[idx];
    const double kT = kK * T;
    const double lam3 = pow(kH * kH / (2.0 * kPi * kMe * kT), 1.5);
    const int ic = L - 1;
    double phi[RH_MAXLEV];
    double Phi = 0.0;
    for (int i = 0; i < ic; ++i) {
        phi[i] = A.lev_g2[i] * lam3 * exp(A.lev_chi[i] / kT);
        Phi += phi[i];
    }
    double ne;
    if (ne_given) {
        ne = c.ne[idx];
    } else {
        double b = 1.0 + A.metal_floor * nH * Phi;
        double npr = 2.0 * nH / (b + sqrt(b * b + 4.0 * Phi * nH));
        ne = npr + A.metal_floor * nH;
        c.ne[idx] = ne;
    }
    double nc = nH / (1.0 + ne * Phi);
    double ns[RH_MAXLEV];
    for (int i = 0; i < ic; ++i) ns[i] = nc * ne * phi[i];
    ns[ic] = nc;
    c.np[idx] = nc;
    for (int i = 0; i < L; ++i) {
        c.nstar[((size_t)col * L + i) * N + k] = ns[i];
        c.pops[((size_t)col * L + i) * N + k] = ns[i];
    }
    const double Kc = kH * kH / (pow(2.0 * kPi * kMe, 1.5) * sqrt(kK));
    double *Cr = c.Crate + ((size_t)col * N + k) * 2 * A.ntr;
    for (int t = 0; t < A.ntr; ++t) {
        const DevTrans &tr = A.tr[t];
        double up;
        if (tr.kind == 0) {
            double dE = kH * tr.nu0;
            double y = dE / kT;
            double P = fmax(0.2, 0.276 * exp_e1(y));
            double Omega = 8.0 * kPi / sqrt(3.0) * (kERyd / dE) * tr.f * P;   // g_l cancels with 1/g_l
            up = ne * Kc * Omega / sqrt(T) * exp(-y);
        } else {
            double u = kH * tr.nu0 / kT;
            up = 1.55e11 * ne * tr.alpha0 * 0.1 * exp(-u) / (u * sqrt(T));
        }
        Cr[2 * t] = up;
        Cr[2 * t + 1] = up * ns[tr.l] / ns[tr.u];
    }
}

// Emergent intensity: one thread per (column, requested wavelength), upward
// linear short-characteristics sweep at direction cosine mu from the
// diffusion condition at the bottom.
template <typename R>
__global__ void spectrum_kernel(const __grid_constant__ DevAtom A, ColumnArrays c, double mu, int64_t nlam,
                                const double *nu_d, const int *nact_d, const int *act_d, const double *spec,
                                double *out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= c.ncol * nlam) return;
    const int64_t col = idx / nlam, j = idx % nlam;
    const int N = c.ndep, L = A.nlev;
    const double nu = nu_d[j];
    const int na = nact_d[j];
    const double e2 = kQ * kQ / (4.0 * kPi * kEps0);
    const double Cff = e2 * e2 * e2 * 4.0 / (3.0 * kMe * kH * kC) * sqrt(2.0 * kPi / (3.0 * kK * kMe));
    const double hm = hminus_sigma(kC / nu);
    const double tw = 2.0 * kH * nu * nu * nu / (kC * kC);
    const size_t cN = (size_t)col * N;
    R I = 0, chip = 0, Sp = 0;
    R Bp = 0;
    for (int step = 0; step < N; ++step) {
        const int k = N - 1 - step;
        const double T = c.T[cN + k];
        const double ne = c.ne[cN + k];
        const double x = kH * nu / (kK * T);
        const double lam3 = pow(kH * kH / (2.0 * kPi * kMe * kK * T), 1.5);
        const double nhm = 0.25 * c.nstar[((size_t)col * L + 0) * N + k] * ne * lam3 * exp(0.754 * kQ / (kK * T));
        const double omex = -expm1(-x);
        double chi = (Cff * ne * c.np[cN + k] / sqrt(T) / (nu * nu * nu) + nhm * hm) * omex + kSigmaT * ne;
        const double B = tw * exp(-x) / omex;
        double eta = chi * B;
        const double vth = sqrt(2.0 * kK * T / A.mass);
        const double sk = N > 1 ? (double)k / (N - 1) : 0.0;
        for (int s = 0; s < na; ++s) {
            const int t = act_d[j * RH_SPEC_ACT + s];
            const DevTrans &tr = A.tr[t];
            const double *f = spec + ((size_t)j * RH_SPEC_ACT + s) * RH_SPEC_F;
            const double nl = c.pops[((size_t)col * L + tr.l) * N + k];
            const double nu_ = c.pops[((size_t)col * L + tr.u) * N + k];
            double Vlu, Vul, U;
            if (tr.kind == 0) {
                const double a = exp((1.0 - sk) * tr.ln_atop + sk * tr.ln_abot);
                const double v = (f[3] - mu * c.vz[cN + k]) / vth;
                const double ph = (R)voigt_f64(a, v) * f[4] / vth;
                Vlu = f[0] * ph;
                Vul = f[2] * Vlu;
                U = f[1] * ph;
            } else {
                const double G = c.nstar[((size_t)col * L + tr.l) * N + k] / c.nstar[((size_t)col * L + tr.u) * N + k];
                Vlu = f[0];
                Vul = G * exp(-x) * f[0];
                U = f[1] * G * exp(-x);
            }
            chi += nl * Vlu - nu_ * Vul;
            eta += nu_ * U;
        }
        const R chiR = (R)chi, S = (R)(eta / chi);
        if (step == 0) {
            chip = chiR;
            Sp = S;
            Bp = (R)B;
            // diffusion condition needs chi and B one point up: computed next step
            continue;
        }
        if (step == 1) {
            // I at the bottom point from the diffusion approximation
            const R dtv = (R)0.5 * (chiR + chip) * (R)fabs(c.z[cN + N - 2] - c.z[cN + N - 1]);
            I = Bp + (R)mu * (Bp - (R)B) / dtv;
        }
        const R dtau = (R)0.5 * (chiR + chip) * (R)fabs(c.z[cN + k] - c.z[cN + k + 1]) / (R)mu;
        R ome, wu, wo;
        sc_weights(dtau, ome, wu, wo);
        I = I * ome + wu * Sp + wo * S;
        chip = chiR;
        Sp = S;
    }
    out[idx] = (double)I;
}

// ----------------------------------------------------------------------------
// Start populations other than LTE (Sect. 2.3: zero radiation, escape
// probability iterations).  One block per column, FP64.  The radiative rates
// keep only spontaneous emission -- A_ul for a line; for a continuum the
// recombination sum_j ce_j e^{-h nu_j/kT} (n*_l/n*_c) over the continuum's
// wavelength points, ce_j = 4 pi w_j (2 h nu_j^3/c^2) alpha(nu_j)/(h nu_j) --
// times, for the escape-probability start, the probability of escape through
// the top p = beta(tau)/2, beta(tau) = (1 - e^{-tau})/tau, tau the line-centre
// (Doppler core) or edge optical depth from the top by the trapezoid rule at
// the current populations (opacity clipped at zero).  Each solve: the rate
// matrix with collisions, the row of the most populated level (current
// populations) replaced by particle conservation, unknowns scaled by the
// current populations, rows equilibrated, partial pivoting.  A column whose
// solve fails keeps its LTE populations and gets status SINGULAR.
__device__ int start_solve_depth(const DevAtom &A, const double *R, const double *esc, const double *Cr, int N,
                                 int k, const double *n, double nH, double *nn)
{
    const int L = A.nlev;
    double G[RH_MAXLEV * RH_MAXLEV];
    for (int i = 0; i < L * L; ++i) G[i] = 0.0;
    for (int t = 0; t < A.ntr; ++t) {
        const int l = A.tr[t].l, u = A.tr[t].u;
        G[l * L + u] += R[t * N + k] * esc[t * N + k] + Cr[2 * t + 1];
        G[u * L + l] += Cr[2 * t];
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
    b[r] = nH;
    for (int pp = 0; pp < L; ++pp) {
        double mx = 0.0;
        for (int q = 0; q < L; ++q) {
            G[pp * L + q] *= sc[q];
            mx = fmax(mx, fabs(G[pp * L + q]));
        }
        if (!(mx > 0.0)) return 1;
        for (int q = 0; q < L; ++q) G[pp * L + q] /= mx;
        b[pp] /= mx;
    }
    for (int cc = 0; cc < L; ++cc) {
        int piv = cc;
        for (int rr = cc + 1; rr < L; ++rr)
            if (fabs(G[rr * L + cc]) > fabs(G[piv * L + cc])) piv = rr;
        if (G[piv * L + cc] == 0.0) return 1;
        if (piv != cc) {
            for (int q = 0; q < L; ++q) {
                double tmp = G[cc * L + q];
                G[cc * L + q] = G[piv * L + q];
                G[piv * L + q] = tmp;
            }
            double tmp = b[cc];
            b[cc] = b[piv];
            b[piv] = tmp;
        }
        for (int rr = cc + 1; rr < L; ++rr) {
            double f = G[rr * L + cc] / G[cc * L + cc];
            for (int q = cc; q < L; ++q) G[rr * L + q] -= f * G[cc * L + q];
            b[rr] -= f * b[cc];
        }
    }
    for (int cc = L - 1; cc >= 0; --cc) {
        double s = b[cc];
        for (int q = cc + 1; q < L; ++q) s -= G[cc * L + q] * b[q];
        b[cc] = s / G[cc * L + cc];
    }
    for (int l = 0; l < L; ++l) {
        const double v = b[l] * sc[l];
        if (!(isfinite(v) && v > 0.0)) return 1;
        nn[l * N + k] = v;
    }
    return 0;
}

__global__ void start_kernel(const __grid_constant__ DevAtom A, ColumnArrays c, int kind, int nit, const int *sp_off,
                             const double *sp_nu, const double *sp_ce)
{
    extern __shared__ double sm[];
    const int N = c.ndep, L = A.nlev, NT = A.ntr, LN = L * N;
    double *n = sm, *nn = n + LN, *R = nn + LN, *esc = R + NT * N;
    __shared__ int bad;
    const int64_t col = blockIdx.x;
    const int tid = threadIdx.x;
    const size_t cN = (size_t)col * N;
    const double *nstar = c.nstar + (size_t)col * LN;
    if (tid == 0) bad = 0;
    for (int i = tid; i < LN; i += blockDim.x) n[i] = nstar[i];
    for (int i = tid; i < NT * N; i += blockDim.x) {
        const int t = i / N, k = i % N;
        const DevTrans &tr = A.tr[t];
        double r;
        if (tr.kind == 0) {
            r = tr.A;
        } else {
            const double kT = kK * c.T[cN + k], G = nstar[tr.l * N + k] / nstar[tr.u * N + k];
            double s = 0.0;
            for (int j = sp_off[t]; j < sp_off[t + 1]; ++j) s += sp_ce[j] * exp(-kH * sp_nu[j] / kT);
            r = s * G;
        }
        R[i] = r;
        esc[i] = 1.0;
    }
    __syncthreads();
    const double *Crc = c.Crate + cN * 2 * NT;
    for (int it = 0; it < nit; ++it) {
        if (kind == 4) {
            for (int t = tid; t < NT; t += blockDim.x) {
                const DevTrans &tr = A.tr[t];
                double tau = 0.0, chip = 0.0;
                for (int k = 0; k < N; ++k) {
                    const double T = c.T[cN + k];
                    double chi;
                    if (tr.kind == 0) {
                        const double dnuD = tr.nu0 / kC * sqrt(2.0 * kK * T / A.mass);
                        chi = (n[tr.l * N + k] - n[tr.u * N + k] * (tr.Bul / tr.Blu)) * (kH * tr.nu0 / (4.0 * kPi)) *
                              tr.Blu / (kSqrtPi * dnuD);
                    } else {
                        const double G = nstar[tr.l * N + k] / nstar[tr.u * N + k];
                        chi = (n[tr.l * N + k] - n[tr.u * N + k] * G * exp(-kH * tr.nu0 / (kK * T))) * tr.alpha0;
                    }
                    chi = fmax(chi, 0.0);
                    if (k > 0) tau += 0.5 * (chi + chip) * fabs(c.z[cN + k - 1] - c.z[cN + k]);
                    chip = chi;
                    esc[t * N + k] = 0.5 * (tau > 0.0 ? -expm1(-tau) / tau : 1.0);
                }
            }
            __syncthreads();
        }
        for (int k = tid; k < N; k += blockDim.x)
            if (start_solve_depth(A, R, esc, Crc + (size_t)k * 2 * NT, N, k, n, c.nH[cN + k], nn)) bad = 1;
        __syncthreads();
        if (bad) break;
        for (int i = tid; i < LN; i += blockDim.x) n[i] = nn[i];
        __syncthreads();
    }
    double *pops = c.pops + (size_t)col * LN;
    for (int i = tid; i < LN; i += blockDim.x) pops[i] = bad ? nstar[i] : n[i];
    if (tid == 0) c.status[col] = (uint8_t)(bad ? RH_COL_SINGULAR : RH_COL_NOTRUN);
}

// ----------------------------------------------------------------------------
// Emergent Stokes vector at mu = 1 of one line with Zeeman splitting (normal
// triplet, effective Lande factor geff), one thread per (column, requested
// wavelength).  Opacities of the background and of the other transitions as
// in spectrum_kernel (unpolarised); the polarised line's propagation matrix
// in the convention
//   K = [[eI, eQ, eU, eV], [eQ, eI, rV, -rU], [eU, -rV, eI, rQ], [eV, rU, -rQ, eI]],
//   eI_l = (k/2)[p sin^2 th + (b + r)(1 + cos^2 th)/2], eQ = (k/2)[p - (b+r)/2] sin^2 th cos 2chi,
//   eU = ... sin 2chi, eV = (k/2)(r - b) cos th, rQ/rU/rV likewise with the
//   dispersion profiles; b, p, r at v - v_B, v, v + v_B; v_B = geff e B/(4 pi m_e)/dnu_D;
// emission: the background and other transitions unpolarised, the line
// S_l (eI_l, eQ, eU, eV).  DELO-linear along the ray (Rees, Durrant & Murphy
// 1989): (1 + w_o K'_o) I_o = e^{-dtau} I_u + w_u (S_u - K'_u I_u) + w_o S_o with
// K' = K/eI - 1 and S the emission / eI; 4 x 4 solve with partial pivoting.
// Bottom: I = B + dB/dtau (diffusion), Q = U = V = 0.
template <typename R>
__device__ __forceinline__ void zeeman_profiles(R a, R v, R vB, const float4 *vtab, const float4 *dtab, R *H, R *L);
template <>
__device__ __forceinline__ void zeeman_profiles<double>(double a, double v, double vB, const float4 *,
                                                        const float4 *, double *H, double *L)
{
    faddeeva_f64(a, v - vB, H[0], L[0]);
    faddeeva_f64(a, v, H[1], L[1]);
    faddeeva_f64(a, v + vB, H[2], L[2]);
}
template <>
__device__ __forceinline__ void zeeman_profiles<float>(float a, float v, float vB, const float4 *vtab,
                                                       const float4 *dtab, float *H, float *L)
{
    const float vs[3] = {v - vB, v, v + vB};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        H[i] = voigt_f32(a, vs[i], vtab);
        L[i] = disp_f32(a, vs[i], dtab);
    }
}

template <typename R>
__device__ void delo_step(R ex, R wu, R wo, const R *Ku, const R *Ko, const R *Su, const R *So, R *I)
{
    // K'(k) from (eQ, eU, eV, rQ, rU, rV)/eI
    auto kp = [](const R *k, R M[4][4]) {
        M[0][0] = 0; M[0][1] = k[0]; M[0][2] = k[1]; M[0][3] = k[2];
        M[1][0] = k[0]; M[1][1] = 0; M[1][2] = k[5]; M[1][3] = -k[4];
        M[2][0] = k[1]; M[2][1] = -k[5]; M[2][2] = 0; M[2][3] = k[3];
        M[3][0] = k[2]; M[3][1] = k[4]; M[3][2] = -k[3]; M[3][3] = 0;
    };
    R Mu[4][4], A[4][4], b[4];
    kp(Ku, Mu);
    kp(Ko, A);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        R kI = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) kI += Mu[i][j] * I[j];
        b[i] = ex * I[i] + wu * (Su[i] - kI) + wo * So[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) A[i][j] = (i == j ? (R)1 : (R)0) + wo * A[i][j];
    }
    // Gaussian elimination with partial pivoting (fixed size, unrolled)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int piv = c;
#pragma unroll
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (r == piv && piv != c) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    R tq = A[c][q];
                    A[c][q] = A[r][q];
                    A[r][q] = tq;
                }
                R tb = b[c];
                b[c] = b[r];
                b[r] = tb;
            }
        const R ip = (R)1 / A[c][c];
#pragma unroll
        for (int r = c + 1; r < 4; ++r) {
            const R f = A[r][c] * ip;
#pragma unroll
            for (int q = c; q < 4; ++q) A[r][q] -= f * A[c][q];
            b[r] -= f * b[c];
        }
    }
#pragma unroll
    for (int c = 3; c >= 0; --c) {
        R s = b[c];
#pragma unroll
        for (int q = c + 1; q < 4; ++q) s -= A[c][q] * b[q];
        b[c] = s / A[c][c];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) I[i] = b[i];
}

template <typename R>
__global__ void stokes_kernel(const __grid_constant__ DevAtom A, ColumnArrays c, int t0, double geff, const double *Bf,
                              const double *thf, const double *azf, int64_t nlam, const double *nu_d,
                              const int *nact_d, const int *act_d, const double *spec, const float4 *vtab_g,
                              const float4 *dtab_g, double *out)
{
    __shared__ float4 tabs[sizeof(R) == 4 ? 2 * (RH_VT_N + 1) : 1];
    const float4 *vtab = tabs, *dtab = tabs + (RH_VT_N + 1);
    if (sizeof(R) == 4) {
        for (int i = threadIdx.x; i <= RH_VT_N; i += blockDim.x) {
            tabs[i] = vtab_g[i];
            tabs[RH_VT_N + 1 + i] = dtab_g[i];
        }
        __syncthreads();
    }
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= c.ncol * nlam) return;
    const int64_t col = idx / nlam, j = idx % nlam;
    const int N = c.ndep, L = A.nlev;
    const double nu = nu_d[j];
    const int na = nact_d[j];
    const double e2 = kQ * kQ / (4.0 * kPi * kEps0);
    const double Cff = e2 * e2 * e2 * 4.0 / (3.0 * kMe * kH * kC) * sqrt(2.0 * kPi / (3.0 * kK * kMe));
    const double hm = hminus_sigma(kC / nu);
    const double tw = 2.0 * kH * nu * nu * nu / (kC * kC);
    const size_t cN = (size_t)col * N;
    const DevTrans &tr0 = A.tr[t0];
    const double h4 = kH * nu / (4.0 * kPi);
    const double nuB = geff * kQ / (4.0 * kPi * kMe);   // Zeeman splitting per tesla, Hz
    R I[4] = {0, 0, 0, 0}, Ku[6], Su[4], eIu = 0, Bu = 0;
    for (int step = 0; step < N; ++step) {
        const int k = N - 1 - step;
        const double T = c.T[cN + k];
        const double ne = c.ne[cN + k];
        const double x = kH * nu / (kK * T);
        const double lam3 = pow(kH * kH / (2.0 * kPi * kMe * kK * T), 1.5);
        const double nhm = 0.25 * c.nstar[((size_t)col * L + 0) * N + k] * ne * lam3 * exp(0.754 * kQ / (kK * T));
        const double omex = -expm1(-x);
        double chi = (Cff * ne * c.np[cN + k] / sqrt(T) / (nu * nu * nu) + nhm * hm) * omex + kSigmaT * ne;
        const double B = tw * exp(-x) / omex;
        double eta = chi * B;
        const double vth = sqrt(2.0 * kK * T / A.mass);
        const double sk = N > 1 ? (double)k / (N - 1) : 0.0;
        for (int s2 = 0; s2 < na; ++s2) {
            const int t = act_d[j * RH_SPEC_ACT + s2];
            if (t == t0) continue;
            const DevTrans &tr = A.tr[t];
            const double *f = spec + ((size_t)j * RH_SPEC_ACT + s2) * RH_SPEC_F;
            const double nl = c.pops[((size_t)col * L + tr.l) * N + k];
            const double nu_ = c.pops[((size_t)col * L + tr.u) * N + k];
            double Vlu, Vul, U;
            if (tr.kind == 0) {
                const double a = exp((1.0 - sk) * tr.ln_atop + sk * tr.ln_abot);
                const double v = (f[3] - c.vz[cN + k]) / vth;
                const double ph = voigt_f64(a, v) * f[4] / vth;
                Vlu = f[0] * ph;
                Vul = f[2] * Vlu;
                U = f[1] * ph;
            } else {
                const double G = c.nstar[((size_t)col * L + tr.l) * N + k] / c.nstar[((size_t)col * L + tr.u) * N + k];
                Vlu = f[0];
                Vul = G * exp(-x) * f[0];
                U = f[1] * G * exp(-x);
            }
            chi += nl * Vlu - nu_ * Vul;
            eta += nu_ * U;
        }
        // the polarised line
        const double dnuD = tr0.nu0 * vth / kC;
        const double nl0 = c.pops[((size_t)col * L + tr0.l) * N + k];
        const double nu0 = c.pops[((size_t)col * L + tr0.u) * N + k];
        const double kl = (nl0 * tr0.Blu - nu0 * tr0.Bul) * h4 / (kSqrtPi * dnuD);
        const double Sl = nu0 * tr0.A / (nl0 * tr0.Blu - nu0 * tr0.Bul);
        const double a0 = exp((1.0 - sk) * tr0.ln_atop + sk * tr0.ln_abot);
        const R v = (R)(kC * ((nu - tr0.nu0) / tr0.nu0) / vth - c.vz[cN + k] / vth);
        const R vB = (R)(nuB * Bf[cN + k] / dnuD);
        R Hz[3], Lz[3];
        zeeman_profiles<R>((R)a0, v, vB, vtab, dtab, Hz, Lz);
        const double th = thf[cN + k], az = azf[cN + k];
        const R s2 = (R)(sin(th) * sin(th)), ct = (R)cos(th), c2 = (R)cos(2.0 * az), sn2 = (R)sin(2.0 * az);
        const R hk = (R)(0.5 * kl);
        const R lI = hk * (Hz[1] * s2 + (R)0.5 * (Hz[0] + Hz[2]) * ((R)1 + ct * ct));
        const R lq = hk * (Hz[1] - (R)0.5 * (Hz[0] + Hz[2])) * s2;
        const R lV = hk * (Hz[2] - Hz[0]) * ct;
        const R rq = hk * (Lz[1] - (R)0.5 * (Lz[0] + Lz[2])) * s2;
        const R rV = hk * (Lz[2] - Lz[0]) * ct;
        const R eI = (R)chi + lI;
        const R ie = (R)1 / eI;
        const R e6[6] = {lq * c2, lq * sn2, lV, rq * c2, rq * sn2, rV};
        R Ko[6], So[4];
#pragma unroll
        for (int i = 0; i < 6; ++i) Ko[i] = e6[i] * ie;
        So[0] = ((R)eta + (R)Sl * lI) * ie;
        So[1] = (R)Sl * e6[0] * ie;
        So[2] = (R)Sl * e6[1] * ie;
        So[3] = (R)Sl * e6[2] * ie;
        if (step == 0) {
            eIu = eI;
            Bu = (R)B;
        } else {
            if (step == 1) {
                // diffusion condition at the bottom point (vertical optical depth)
                const R dtv = (R)0.5 * (eI + eIu) * (R)fabs(c.z[cN + N - 2] - c.z[cN + N - 1]);
                I[0] = Bu + (Bu - (R)B) / dtv;
            }
            const R dtau = (R)0.5 * (eI + eIu) * (R)fabs(c.z[cN + k] - c.z[cN + k + 1]);
            R ome, wu, wo;
            sc_weights(dtau, ome, wu, wo);
            delo_step<R>(ome, wu, wo, Ku, Ko, Su, So, I);
            eIu = eI;
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) Ku[i] = Ko[i];
#pragma unroll
        for (int i = 0; i < 4; ++i) Su[i] = So[i];
    }
    double *o = out + (size_t)idx * 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = (double)I[i];
}

// FP32 Zeeman Stokes spectrum, one block per column (grid-stride): the
// quantities that depend on depth only -- background coefficients, Doppler
// widths, populations (divided by kStokesNref so that every product stays in
// FP32 range), continuum LTE ratios, the polarised line's opacity factor,
// source function, damping, Zeeman splitting and field geometry -- are formed
// once per depth in FP64 and stored in shared memory in FP32; then every
// thread sweeps its wavelengths with FP32 opacities, profiles and the same
// DELO-linear step as stokes_kernel.  Layout of the shared arrays: kSF fields
// [field][N], then the populations [L][N] and continuum ratios [ncont][N].
constexpr double kStokesNref = 1e20;
constexpr int kSF = 16;
enum { SF_HKT, SF_KFF, SF_NHM, SF_THOM, SF_IVTH, SF_VZ, SF_DZ, SF_SK, SF_KL, SF_SL, SF_A0, SF_VB, SF_S2, SF_CT, SF_C2,
       SF_SN2 };
__global__ void __launch_bounds__(128) stokes32_kernel(const __grid_constant__ DevAtom A, ColumnArrays c, int t0,
                                                       double geff, const double *Bf, const double *thf,
                                                       const double *azf, int64_t nlam, const double *nu_d,
                                                       const int *nact_d, const int *act_d, const double *spec,
                                                       const float4 *vtab_g, const float4 *dtab_g, double *out)
{
    extern __shared__ __align__(16) float sf[];
    __shared__ float4 tabs[2 * (RH_VT_N + 1)];
    const float4 *vtab = tabs, *dtab = tabs + (RH_VT_N + 1);
    for (int i = threadIdx.x; i <= RH_VT_N; i += blockDim.x) {
        tabs[i] = vtab_g[i];
        tabs[RH_VT_N + 1 + i] = dtab_g[i];
    }
    const int N = c.ndep, L = A.nlev;
    float *pop = sf + (size_t)kSF * N;            // [L][N] populations / kStokesNref
    float *gc = pop + (size_t)L * N;              // [ncont][N] n*_l / n*_u
    const DevTrans &tr0 = A.tr[t0];
    const double e2 = kQ * kQ / (4.0 * kPi * kEps0);
    const double Cff = e2 * e2 * e2 * 4.0 / (3.0 * kMe * kH * kC) * sqrt(2.0 * kPi / (3.0 * kK * kMe));
    const double nuB = geff * kQ / (4.0 * kPi * kMe);
    const double h40 = kH * tr0.nu0 / (4.0 * kPi);
    for (int64_t col = blockIdx.x; col < c.ncol; col += gridDim.x) {
        __syncthreads();
        const size_t cN = (size_t)col * N;
        for (int k = threadIdx.x; k < N; k += blockDim.x) {
            const double T = c.T[cN + k], ne = c.ne[cN + k];
            const double vth = sqrt(2.0 * kK * T / A.mass);
            const double lam3 = pow(kH * kH / (2.0 * kPi * kMe * kK * T), 1.5);
            const double sk = N > 1 ? (double)k / (N - 1) : 0.0;
            sf[SF_HKT * N + k] = (float)(kH / (kK * T));
            sf[SF_KFF * N + k] = (float)(Cff * ne * c.np[cN + k] / sqrt(T) / kNuRef3);
            sf[SF_NHM * N + k] = (float)(0.25 * c.nstar[((size_t)col * L + 0) * N + k] * ne * lam3 *
                                         exp(0.754 * kQ / (kK * T)));
            sf[SF_THOM * N + k] = (float)(kSigmaT * ne);
            sf[SF_IVTH * N + k] = (float)(1.0 / vth);
            sf[SF_VZ * N + k] = (float)c.vz[cN + k];
            sf[SF_DZ * N + k] = (float)(k < N - 1 ? fabs(c.z[cN + k] - c.z[cN + k + 1]) : 0.0);
            sf[SF_SK * N + k] = (float)sk;
            const double nl0 = c.pops[((size_t)col * L + tr0.l) * N + k];
            const double nu0 = c.pops[((size_t)col * L + tr0.u) * N + k];
            const double dnuD = tr0.nu0 * vth / kC;
            sf[SF_KL * N + k] = (float)((nl0 * tr0.Blu - nu0 * tr0.Bul) * h40 / (kSqrtPi * dnuD));
            sf[SF_SL * N + k] = (float)(nu0 * tr0.A / (nl0 * tr0.Blu - nu0 * tr0.Bul));
            sf[SF_A0 * N + k] = (float)exp((1.0 - sk) * tr0.ln_atop + sk * tr0.ln_abot);
            sf[SF_VB * N + k] = (float)(nuB * Bf[cN + k] / dnuD);
            const double th = thf[cN + k], az = azf[cN + k];
            sf[SF_S2 * N + k] = (float)(sin(th) * sin(th));
            sf[SF_CT * N + k] = (float)cos(th);
            sf[SF_C2 * N + k] = (float)cos(2.0 * az);
            sf[SF_SN2 * N + k] = (float)sin(2.0 * az);
            for (int l = 0; l < L; ++l)
                pop[l * N + k] = (float)(c.pops[((size_t)col * L + l) * N + k] / kStokesNref);
            for (int t = 0; t < A.ntr; ++t) {
                const DevTrans &tr = A.tr[t];
                if (tr.kind != 0)
                    gc[tr.sub * N + k] = (float)(c.nstar[((size_t)col * L + tr.l) * N + k] /
                                                 c.nstar[((size_t)col * L + tr.u) * N + k]);
            }
        }
        __syncthreads();
        for (int64_t j = threadIdx.x; j < nlam; j += blockDim.x) {
            const double nud = nu_d[j];
            const float nu = (float)nud;
            const int na = nact_d[j];
            const float hm = (float)hminus_sigma(kC / nud);
            const float tw = (float)(2.0 * kH * nud * nud * nud / (kC * kC));
            const float nu3s = (float)(kNuRef3 / (nud * nud * nud));
            const float q0 = (float)(kC * ((nud - tr0.nu0) / tr0.nu0));
            const float hr = (float)(nud / tr0.nu0);             // h4(nu) / h4(nu0)
            float I[4] = {0, 0, 0, 0}, Ku[6], Su[4], eIu = 0, Bu = 0;
            for (int step = 0; step < N; ++step) {
                const int k = N - 1 - step;
                const float x = nu * sf[SF_HKT * N + k];
                const float ex = __expf(-x), omex = 1.0f - ex;
                float chi = (sf[SF_KFF * N + k] * nu3s + sf[SF_NHM * N + k] * hm) * omex + sf[SF_THOM * N + k];
                const float B = tw * ex / omex;
                float eta = chi * B;
                const float ivth = sf[SF_IVTH * N + k], vz = sf[SF_VZ * N + k], sk = sf[SF_SK * N + k];
                for (int s2i = 0; s2i < na; ++s2i) {
                    const int t = act_d[j * RH_SPEC_ACT + s2i];
                    if (t == t0) continue;
                    const DevTrans &tr = A.tr[t];
                    const double *f = spec + ((size_t)j * RH_SPEC_ACT + s2i) * RH_SPEC_F;
                    const float nl = pop[tr.l * N + k], nuu = pop[tr.u * N + k];
                    if (tr.kind == 0) {
                        const float a = __expf((1.0f - sk) * (float)tr.ln_atop + sk * (float)tr.ln_abot);
                        const float v = ((float)f[3] - vz) * ivth;
                        const float ph = voigt_f32(a, v, vtab) * (float)(f[4] * kStokesNref) * ivth;
                        const float Vlu = (float)f[0] * ph;
                        chi += nl * Vlu - nuu * ((float)f[2] * Vlu);
                        eta += nuu * ((float)f[1] * ph);
                    } else {
                        const float G = gc[tr.sub * N + k] * ex;
                        const float al = (float)(f[0] * kStokesNref);
                        chi += nl * al - nuu * G * al;
                        eta += nuu * G * (float)(f[1] * kStokesNref);
                    }
                }
                const float v = (q0 - vz) * ivth;
                float Hz[3], Lz[3];
                zeeman_profiles<float>(sf[SF_A0 * N + k], v, sf[SF_VB * N + k], vtab, dtab, Hz, Lz);
                const float s2 = sf[SF_S2 * N + k], ct = sf[SF_CT * N + k];
                const float c2 = sf[SF_C2 * N + k], sn2 = sf[SF_SN2 * N + k];
                const float hk = 0.5f * sf[SF_KL * N + k] * hr, Sl = sf[SF_SL * N + k];
                const float lI = hk * (Hz[1] * s2 + 0.5f * (Hz[0] + Hz[2]) * (1.0f + ct * ct));
                const float lq = hk * (Hz[1] - 0.5f * (Hz[0] + Hz[2])) * s2;
                const float lV = hk * (Hz[2] - Hz[0]) * ct;
                const float rq = hk * (Lz[1] - 0.5f * (Lz[0] + Lz[2])) * s2;
                const float rV = hk * (Lz[2] - Lz[0]) * ct;
                const float eI = chi + lI;
                const float ie = 1.0f / eI;
                const float e6[6] = {lq * c2, lq * sn2, lV, rq * c2, rq * sn2, rV};
                float Ko[6], So[4];
#pragma unroll
                for (int i = 0; i < 6; ++i) Ko[i] = e6[i] * ie;
                So[0] = (eta + Sl * lI) * ie;
                So[1] = Sl * e6[0] * ie;
                So[2] = Sl * e6[1] * ie;
                So[3] = Sl * e6[2] * ie;
                if (step == 0) {
                    eIu = eI;
                    Bu = B;
                } else {
                    if (step == 1) {
                        // diffusion condition at the bottom point (vertical optical depth)
                        const float dtv = 0.5f * (eI + eIu) * sf[SF_DZ * N + N - 2];
                        I[0] = Bu + (Bu - B) / dtv;
                    }
                    const float dtau = 0.5f * (eI + eIu) * sf[SF_DZ * N + k];
                    float ome, wu, wo;
                    sc_weights(dtau, ome, wu, wo);
                    delo_step<float>(ome, wu, wo, Ku, Ko, Su, So, I);
                    eIu = eI;
                }
#pragma unroll
                for (int i = 0; i < 6; ++i) Ku[i] = Ko[i];
#pragma unroll
                for (int i = 0; i < 4; ++i) Su[i] = So[i];
            }
            double *o = out + ((size_t)col * nlam + j) * 4;
#pragma unroll
            for (int i = 0; i < 4; ++i) o[i] = (double)I[i];
        }
    }
}

// Depth-grid optimisation (Sect. 2.3), one thread per column, FP64.  The
// column -- after the optional cut at z_top, whose new top point is
// interpolated (T, v_z linearly, n_H and n_e logarithmically in height) -- is
// walked twice: first the monitor s (cumulative, into the scratch row of the
// column), whose step between neighbours is the root sum of squares of the
// step in log10 of the hydrogen column density over dN, in ln T over dT, in
// v_z over dv and in height over spacing x (height / (M - 1)); the column
// density above each point is n_H H at the top (H the scale height of the
// top two points) plus the exact integral of an exponential n_H between
// points.  Then M points at equal steps of s from the top to the bottom,
// each interpolated on its segment of the old grid.
__global__ void regrid_kernel(int64_t ncol, int N, int M, const double *z, const double *T, const double *nH,
                              const double *vz, const double *ne, RegridParams g, double *srow, double *zo,
                              double *To, double *nHo, double *vzo, double *neo, unsigned long long *bad)
{
    const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const double *cz = z + col * N, *cT = T + col * N, *cn = nH + col * N, *cv = vz + col * N, *ce = ne + col * N;
    double *sc = srow + col * N;
    // the kept column: an optional interpolated top point, then old points k0..N-1
    int k0 = 0;
    bool top = false;
    double tz = 0, tT = 0, tln = 0, tv = 0, tle = 0;
    if (g.use_z_top && g.z_top < cz[0]) {
        if (!(g.z_top > cz[N - 1])) {
            atomicMin(bad, (unsigned long long)col);
            return;
        }
        while (cz[k0] > g.z_top) ++k0;
        if (cz[k0] < g.z_top) {
            const double f = (g.z_top - cz[k0 - 1]) / (cz[k0] - cz[k0 - 1]);
            top = true;
            tz = g.z_top;
            tT = cT[k0 - 1] + f * (cT[k0] - cT[k0 - 1]);
            tln = log(cn[k0 - 1]) + f * (log(cn[k0]) - log(cn[k0 - 1]));
            tv = cv[k0 - 1] + f * (cv[k0] - cv[k0 - 1]);
            tle = log(ce[k0 - 1]) + f * (log(ce[k0]) - log(ce[k0 - 1]));
        }
    }
    const int n = N - k0 + (top ? 1 : 0);
    auto at = [&](int i, double &zz, double &tt, double &ln, double &vv, double &le) {
        if (top && i == 0) {
            zz = tz; tt = tT; ln = tln; vv = tv; le = tle;
            return;
        }
        const int k = k0 + i - (top ? 1 : 0);
        zz = cz[k]; tt = cT[k]; ln = log(cn[k]); vv = cv[k]; le = log(ce[k]);
    };
    double z0, T0, l0, v0, e0, z1, T1, l1, v1, e1;
    at(0, z0, T0, l0, v0, e0);
    at(1, z1, T1, l1, v1, e1);
    double zb, Tb, lb, vb, eb;
    at(n - 1, zb, Tb, lb, vb, eb);
    const double dzs = g.spacing * (z0 - zb) / (M - 1);
    // monitor
    double Ncol = exp(l0) * ((l1 - l0) > 1e-12 ? (z0 - z1) / (l1 - l0) : (z0 - z1));
    sc[0] = 0.0;
    for (int i = 0; i + 1 < n; ++i) {
        if (i > 0) {
            z0 = z1; T0 = T1; l0 = l1; v0 = v1;
            at(i + 1, z1, T1, l1, v1, e1);
        }
        const double dz = z0 - z1, dl = l1 - l0;
        const double seg = fabs(dl) > 1e-12 ? dz * (exp(l1) - exp(l0)) / dl : dz * exp(l0);
        const double N1 = Ncol + seg;
        const double q1 = log10(N1 / Ncol) / g.dN, q2 = log(T1 / T0) / g.dT, q3 = (v1 - v0) / g.dv, q4 = dz / dzs;
        sc[i + 1] = sc[i] + sqrt(q1 * q1 + q2 * q2 + q3 * q3 + q4 * q4);
        Ncol = N1;
    }
    // new points
    const double stot = sc[n - 1];
    int i = 0;
    double za, Ta, la, va, ea, zc, Tc, lc, vc, ec;
    at(0, za, Ta, la, va, ea);
    at(1, zc, Tc, lc, vc, ec);
    for (int j = 0; j < M; ++j) {
        const int64_t o = col * M + j;
        if (j == M - 1) {
            zo[o] = zb; To[o] = Tb; nHo[o] = exp(lb); vzo[o] = vb; neo[o] = exp(eb);
            break;
        }
        const double sj = stot * j / (M - 1);
        while (i + 2 < n && sc[i + 1] < sj) {
            ++i;
            za = zc; Ta = Tc; la = lc; va = vc; ea = ec;
            at(i + 1, zc, Tc, lc, vc, ec);
        }
        const double f = (sj - sc[i]) / (sc[i + 1] - sc[i]);
        zo[o] = za + f * (zc - za);
        To[o] = Ta + f * (Tc - Ta);
        nHo[o] = exp(la + f * (lc - la));
        vzo[o] = va + f * (vc - va);
        neo[o] = exp(ea + f * (ec - ea));
    }
}

}  // namespace

cudaError_t launch_lte_setup(const DevAtom &A, const ColumnArrays &c, int ne_given, cudaStream_t st)
{
    int64_t n = c.ncol * c.ndep;
    if (n == 0) return cudaSuccess;
    int threads = 128;
    int64_t blocks = (n + threads - 1) / threads;
    lte_setup_kernel<<<(unsigned)blocks, threads, 0, st>>>(A, c, ne_given);
    return cudaGetLastError();
}

cudaError_t launch_start(const DevAtom &A, const ColumnArrays &c, int kind, const int *sp_off, const double *sp_nu,
                         const double *sp_ce, cudaStream_t st)
{
    if (c.ncol == 0) return cudaSuccess;
    const size_t sm = sizeof(double) * (2 * (size_t)A.nlev * c.ndep + 2 * (size_t)A.ntr * c.ndep);
    cudaError_t e = cudaFuncSetAttribute(start_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    start_kernel<<<(unsigned)c.ncol, 128, sm, st>>>(A, c, kind, kind == 4 ? kStartEscapeIterations : 1, sp_off, sp_nu,
                                                    sp_ce);
    return cudaGetLastError();
}

cudaError_t launch_stokes(const DevAtom &A, const ColumnArrays &c, int t0, double geff, const double *B_T,
                          const double *theta, const double *chi, int64_t nlam, const double *nu_d, const int *nact_d,
                          const int *act_d, const double *spec_d, const float4 *vtab, const float4 *dtab, double *out,
                          int precision, cudaStream_t st)
{
    int64_t n = c.ncol * nlam;
    if (n == 0) return cudaSuccess;
    int threads = 128;
    int64_t blocks = (n + threads - 1) / threads;
    // FP32: depth-only quantities once per column in shared memory (fits for
    // every depth count up to the limit below; larger columns use the
    // per-wavelength kernel)
    const size_t sm32 = sizeof(float) * (size_t)c.ndep * (kSF + A.nlev + A.ncont);
    if (precision == 1 && sm32 <= 160 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(stokes32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm32);
        if (e != cudaSuccess) return e;
        int dev = 0, nsm = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, stokes32_kernel, 128, sm32);
        if (e != cudaSuccess) return e;
        int64_t g = (int64_t)(per > 0 ? per : 1) * nsm;
        if (g > c.ncol) g = c.ncol;
        stokes32_kernel<<<(unsigned)g, 128, sm32, st>>>(A, c, t0, geff, B_T, theta, chi, nlam, nu_d, nact_d, act_d,
                                                        spec_d, vtab, dtab, out);
    } else if (precision == 1)
        stokes_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(A, c, t0, geff, B_T, theta, chi, nlam, nu_d, nact_d,
                                                                 act_d, spec_d, vtab, dtab, out);
    else
        stokes_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(A, c, t0, geff, B_T, theta, chi, nlam, nu_d,
                                                                  nact_d, act_d, spec_d, vtab, dtab, out);
    return cudaGetLastError();
}

cudaError_t launch_spectrum(const DevAtom &A, const ColumnArrays &c, double mu, int64_t nlam, const double *nu_d,
                            const int *nact_d, const int *act_d, const double *spec_d, double *out, int precision,
                            cudaStream_t st)
{
    int64_t n = c.ncol * nlam;
    if (n == 0) return cudaSuccess;
    int threads = 128;
    int64_t blocks = (n + threads - 1) / threads;
    if (precision == 1)
        spectrum_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(A, c, mu, nlam, nu_d, nact_d, act_d, spec_d, out);
    else
        spectrum_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(A, c, mu, nlam, nu_d, nact_d, act_d, spec_d, out);
    return cudaGetLastError();
}

cudaError_t launch_regrid(const ColumnArrays &c, int M, const RegridParams &g, double *srow, double *zo, double *To,
                          double *nHo, double *vzo, double *neo, unsigned long long *bad, cudaStream_t st)
{
    regrid_kernel<<<(unsigned)((c.ncol + 127) / 128), 128, 0, st>>>(c.ncol, c.ndep, M, c.z, c.T, c.nH, c.vz, c.ne, g,
                                                                   srow, zo, To, nHo, vzo, neo, bad);
    return cudaGetLastError();
}

}  // namespace rh
