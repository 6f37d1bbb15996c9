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

}  // namespace rh
