// rh15d_mlp.cu -- learned initial guess for MALI: an MLP that maps a
// column's atmosphere (T, log10 n_e, log10 n_H, v_z at every depth) to the
// log departure coefficients ln(n_i / n*_i) at every depth, trained on the
// GPU on columns that MALI converged, evaluated to start MALI closer to its
// fixed point (the paper's start solutions, Sect. 2.3, decide the iteration
// count; this start is an addition, MALI still iterates to the same
// criterion and the LTE start stays the fallback).
//
// Network: nin -> hidden -> ... -> nout, GELU (erf form) on hidden layers.
// BF16 weights and activations, FP32 accumulation on the tensor cores
// (hand-written mma.sync m16n8k16), FP32 master weights and Adam moments.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "rh15d_internal.h"

namespace rh {

namespace {

typedef __nv_bfloat16 bf16;

enum Epi { EPI_BIAS_GELU = 0, EPI_BIAS = 1, EPI_F32 = 2, EPI_GELU_BACK = 3 };

constexpr int TM = 64, TN = 64, TK = 32, TKP = TK + 8;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

__device__ __forceinline__ void mma_bf16(float *c, const uint32_t *a, const uint32_t *b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C(m,n) = sum_k A(m,k) B(k,n), A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn]
// (BF16, any strides; out-of-range elements read as zero), FP32 accumulation
// on tensor cores, 64x64 block tile, 4 warps of 32x32.  Epilogues:
//   EPI_BIAS_GELU: Z = C + bias (FP32, ldz), Y = bf16(GELU(Z)) (ldy)
//   EPI_BIAS:      O = C + bias (FP32, ldo)
//   EPI_F32:       O = C (FP32, ldo)
//   EPI_GELU_BACK: Y = bf16(C * GELU'(Z)) (ldy), Z read (ldz)
template <int EPI>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(int M, int N, int K, const bf16 *__restrict__ A, int64_t sam,
                                                        int64_t sak, const bf16 *__restrict__ B, int64_t sbk,
                                                        int64_t sbn, const float *__restrict__ bias, float *Z,
                                                        int64_t ldz, bf16 *Y, int64_t ldy, float *O, int64_t ldo)
{
    __shared__ __align__(16) bf16 As[TM][TKP];
    __shared__ __align__(16) bf16 Bs[TN][TKP];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int g = lane >> 2, tg = lane & 3;
    const int64_t m0 = (int64_t)blockIdx.y * TM, n0 = (int64_t)blockIdx.x * TN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += TK) {
        for (int e = tid; e < TM * TK; e += 128) {
            int r = e / TK, kk = e % TK;
            int64_t m = m0 + r;
            int k = k0 + kk;
            As[r][kk] = (m < M && k < K) ? A[m * sam + (int64_t)k * sak] : zero;
            int64_t n = n0 + r;
            Bs[r][kk] = (n < N && k < K) ? B[(int64_t)k * sbk + n * sbn] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < TK; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                int r0 = wm * 32 + i * 16;
                af[i][0] = *reinterpret_cast<const uint32_t *>(&As[r0 + g][ks + 2 * tg]);
                af[i][1] = *reinterpret_cast<const uint32_t *>(&As[r0 + g + 8][ks + 2 * tg]);
                af[i][2] = *reinterpret_cast<const uint32_t *>(&As[r0 + g][ks + 8 + 2 * tg]);
                af[i][3] = *reinterpret_cast<const uint32_t *>(&As[r0 + g + 8][ks + 8 + 2 * tg]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int c0 = wn * 32 + j * 8;
                bfr[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[c0 + g][ks + 2 * tg]);
                bfr[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[c0 + g][ks + 8 + 2 * tg]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                int64_t m = m0 + wm * 32 + i * 16 + g + (r >= 2 ? 8 : 0);
                int64_t n = n0 + wn * 32 + j * 8 + 2 * tg + (r & 1);
                if (m >= M || n >= N) continue;
                float v = acc[i][j][r];
                if (EPI == EPI_BIAS_GELU) {
                    float z = v + bias[n];
                    Z[m * ldz + n] = z;
                    Y[m * ldy + n] = __float2bfloat16_rn(gelu(z));
                } else if (EPI == EPI_BIAS) {
                    O[m * ldo + n] = v + bias[n];
                } else if (EPI == EPI_F32) {
                    O[m * ldo + n] = v;
                } else {
                    Y[m * ldy + n] = __float2bfloat16_rn(v * gelu_grad(Z[m * ldz + n]));
                }
            }
}

template <int EPI>
cudaError_t gemm(cudaStream_t st, int M, int N, int K, const bf16 *A, int64_t sam, int64_t sak, const bf16 *B,
                 int64_t sbk, int64_t sbn, const float *bias, float *Z, int64_t ldz, bf16 *Y, int64_t ldy, float *O,
                 int64_t ldo)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((N + TN - 1) / TN), (unsigned)((M + TM - 1) / TM));
    gemm_bf16_kernel<EPI><<<grid, 128, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, bias, Z, ldz, Y, ldy, O, ldo);
    return cudaGetLastError();
}

// raw input features per column: [T | log10 n_e | log10 n_H | v_z] x ndep
__global__ void features_kernel(ColumnArrays c, float *X)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int N = c.ndep;
    if (i >= c.ncol * N) return;
    int64_t col = i / N;
    int k = (int)(i % N);
    float *x = X + col * 4 * N;
    x[k] = (float)c.T[i];
    x[N + k] = (float)log10(c.ne[i]);
    x[2 * N + k] = (float)log10(c.nH[i]);
    x[3 * N + k] = (float)c.vz[i];
}

// standardise with the stored mean / std and convert to BF16; rows listed by idx (or all)
__global__ void standardise_kernel(int64_t nrow, int nin, const float *X, const int *idx, const float *mean,
                                   const float *istd, bf16 *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrow * nin) return;
    int64_t r = i / nin;
    int f = (int)(i % nin);
    int64_t src = idx ? idx[r] : r;
    out[i] = __float2bfloat16_rn((X[src * nin + f] - mean[f]) * istd[f]);
}

// per-feature mean and inverse standard deviation over the listed rows (two passes, FP64)
__global__ void feature_stats_kernel(int64_t nrow, int nin, const float *X, const int *idx, float *mean, float *istd)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nin) return;
    double s = 0.0;
    for (int64_t r = 0; r < nrow; ++r) s += X[(int64_t)idx[r] * nin + f];
    double mu = s / nrow, v = 0.0;
    for (int64_t r = 0; r < nrow; ++r) {
        double d = X[(int64_t)idx[r] * nin + f] - mu;
        v += d * d;
    }
    double sd = sqrt(v / nrow);
    mean[f] = (float)mu;
    istd[f] = (float)(sd > 1e-12 * (fabs(mu) + 1.0) ? 1.0 / sd : 1.0);
}

// targets ln(n / n*) [col][level][depth] flattened level-major per column
__global__ void targets_kernel(int64_t ncol, int nout, const double *pops, const double *nstar, float *Yt)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncol * nout) return;
    Yt[i] = (float)log(pops[i] / nstar[i]);
}

// MSE loss over a batch (gathered rows) and its gradient dL/dpred (BF16):
// L = mean over rows and outputs of (pred - target)^2
__global__ void mse_kernel(int64_t nrow, int nout, const float *pred, const float *Yt, const int *idx, bf16 *dpred,
                           double *loss)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < nrow * nout) {
        int64_t r = i / nout;
        int o = (int)(i % nout);
        float t = Yt[(int64_t)(idx ? idx[r] : r) * nout + o];
        float d = pred[i] - t;
        l = (double)d * d;
        dpred[i] = __float2bfloat16_rn(2.0f * d / (float)(nrow * nout));
    }
    // block reduction then one atomic per block
    __shared__ double red[256];
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / (double)(nrow * nout));
}

// db[n] = sum_m dZ[m][n]  (dZ BF16), FP32 result
__global__ void colsum_kernel(int64_t M, int N, const bf16 *dZ, float *db)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int64_t m = 0; m < M; ++m) s += __bfloat162float(dZ[m * N + n]);
    db[n] = s;
}

// Adam step on FP32 master parameters, then BF16 copies of the weights
__global__ void adam_kernel(int64_t n, float *w, const float *gw, float *m1, float *m2, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float g = gw[i];
    float a = b1 * m1[i] + (1.f - b1) * g, b = b2 * m2[i] + (1.f - b2) * g * g;
    m1[i] = a;
    m2[i] = b;
    w[i] -= lr * (a * c1) / (sqrtf(b * c2) + eps);
}

__global__ void to_bf16_kernel(int64_t n, const float *w, bf16 *o)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = __float2bfloat16_rn(w[i]);
}

// start populations from the predicted ln b: n_i = b_i n*_i, renormalised so
// that sum_i n_i = n_H at each depth; non-finite predictions -> LTE
__global__ void apply_guess_kernel(int64_t ncol, int L, int N, const float *lnb, const double *nstar, const double *nH,
                                   double *pops, int *nfallback)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncol * N) return;
    int64_t col = i / N;
    int k = (int)(i % N);
    double n[RH_MAXLEV], s = 0.0;
    bool ok = true;
    for (int l = 0; l < L; ++l) {
        size_t q = ((size_t)col * L + l) * N + k;
        float x = lnb[q];
        double v = nstar[q] * exp((double)fminf(fmaxf(x, -80.f), 80.f));
        ok = ok && isfinite(x) && isfinite(v) && v > 0.0;
        n[l] = v;
        s += v;
    }
    if (!ok || !(s > 0.0)) {
        atomicAdd(nfallback, 1);
        for (int l = 0; l < L; ++l) pops[((size_t)col * L + l) * N + k] = nstar[((size_t)col * L + l) * N + k];
        return;
    }
    double f = nH[i] / s;
    for (int l = 0; l < L; ++l) pops[((size_t)col * L + l) * N + k] = n[l] * f;
}

}  // namespace

// ---------------------------------------------------------------------------
struct Mlp {
    int nin = 0, hidden = 0, nhid = 0, nout = 0, nlayer = 0;
    std::vector<int> din, dout;          // per layer
    std::vector<int64_t> woff, boff;     // offsets into the parameter vector
    int64_t nparam = 0;
    float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;   // FP32 master, grad, Adam
    bf16 *wb = nullptr;                  // BF16 weights (same offsets)
    float *mean = nullptr, *istd = nullptr;
    int64_t adam_t = 0;
    // work buffers sized for the largest batch seen
    int64_t cap = 0;
    bf16 *act = nullptr;                 // [nlayer][cap][maxdim] layer inputs (BF16)
    float *zbuf = nullptr;               // [nlayer][cap][maxdim] pre-activations
    bf16 *dz = nullptr, *dx = nullptr;   // [cap][maxdim]
    float *pred = nullptr;               // [cap][nout]
    int maxdim = 0;
};

static void mlp_free_work(Mlp *m)
{
    cudaFree(m->act);
    cudaFree(m->zbuf);
    cudaFree(m->dz);
    cudaFree(m->dx);
    cudaFree(m->pred);
    m->act = nullptr;
    m->zbuf = nullptr;
    m->dz = m->dx = nullptr;
    m->pred = nullptr;
    m->cap = 0;
}

void mlp_destroy(Mlp *m)
{
    if (!m) return;
    mlp_free_work(m);
    cudaFree(m->w);
    cudaFree(m->g);
    cudaFree(m->m1);
    cudaFree(m->m2);
    cudaFree(m->wb);
    cudaFree(m->mean);
    cudaFree(m->istd);
    delete m;
}

int64_t mlp_nparams(const Mlp *m) { return m ? m->nparam : 0; }
int mlp_nin(const Mlp *m) { return m ? m->nin : 0; }
int mlp_nlayer(const Mlp *m) { return m ? m->nlayer : 0; }
int mlp_nout(const Mlp *m) { return m ? m->nout : 0; }

// He-normal initialisation (seeded), zero biases, identity standardisation
cudaError_t mlp_create(Mlp **out, int nin, int hidden, int nhid, int nout, uint64_t seed)
{
    Mlp *m = new Mlp();
    m->nin = nin;
    m->hidden = hidden;
    m->nhid = nhid;
    m->nout = nout;
    m->nlayer = nhid + 1;
    int64_t off = 0;
    m->maxdim = std::max(std::max(nin, hidden), nout);
    for (int l = 0; l < m->nlayer; ++l) {
        int di = l == 0 ? nin : hidden, dn = l == nhid ? nout : hidden;
        m->din.push_back(di);
        m->dout.push_back(dn);
        m->woff.push_back(off);
        off += (int64_t)di * dn;
        m->boff.push_back(off);
        off += dn;
    }
    m->nparam = off;
    std::vector<float> h(off, 0.f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    for (int l = 0; l < m->nlayer; ++l) {
        double s = std::sqrt(2.0 / m->din[l]);
        for (int64_t i = 0; i < (int64_t)m->din[l] * m->dout[l]; ++i) h[m->woff[l] + i] = (float)(s * nd(rng));
    }
    cudaError_t e = cudaMalloc(&m->w, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->g, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->m1, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->m2, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->wb, off * 2);
    if (e == cudaSuccess) e = cudaMalloc(&m->mean, nin * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->istd, nin * 4);
    if (e == cudaSuccess) e = cudaMemcpy(m->w, h.data(), off * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m1, 0, off * 4);
    if (e == cudaSuccess) e = cudaMemset(m->m2, 0, off * 4);
    if (e == cudaSuccess) {
        std::vector<float> z(nin, 0.f), o(nin, 1.f);
        e = cudaMemcpy(m->mean, z.data(), nin * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(m->istd, o.data(), nin * 4, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        to_bf16_kernel<<<(unsigned)((off + 255) / 256), 256>>>(off, m->w, m->wb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        mlp_destroy(m);
        return e;
    }
    *out = m;
    return cudaSuccess;
}

static cudaError_t mlp_ensure_work(Mlp *m, int64_t rows)
{
    if (rows <= m->cap) return cudaSuccess;
    mlp_free_work(m);
    size_t per = (size_t)rows * m->maxdim;
    cudaError_t e = cudaMalloc(&m->act, per * m->nlayer * 2);
    if (e == cudaSuccess) e = cudaMalloc(&m->zbuf, per * m->nlayer * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->dz, per * 2);
    if (e == cudaSuccess) e = cudaMalloc(&m->dx, per * 2);
    if (e == cudaSuccess) e = cudaMalloc(&m->pred, (size_t)rows * m->nout * 4);
    if (e == cudaSuccess) m->cap = rows;
    return e;
}

// parameter vector layout on the host: weights and biases as on the device,
// then mean[nin], istd[nin]
int64_t mlp_state_size(const Mlp *m) { return m->nparam + 2 * m->nin; }

cudaError_t mlp_get_state(const Mlp *m, float *h)
{
    cudaError_t e = cudaMemcpy(h, m->w, m->nparam * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(h + m->nparam, m->mean, m->nin * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(h + m->nparam + m->nin, m->istd, m->nin * 4, cudaMemcpyDeviceToHost);
    return e;
}

cudaError_t mlp_set_state(Mlp *m, const float *h)
{
    cudaError_t e = cudaMemcpy(m->w, h, m->nparam * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->mean, h + m->nparam, m->nin * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->istd, h + m->nparam + m->nin, m->nin * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        to_bf16_kernel<<<(unsigned)((m->nparam + 255) / 256), 256>>>(m->nparam, m->w, m->wb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemset(m->m1, 0, m->nparam * 4);
    if (e == cudaSuccess) e = cudaMemset(m->m2, 0, m->nparam * 4);
    m->adam_t = 0;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e;
}

// forward pass of `rows` standardised inputs (BF16 [rows][nin] in m->act layer 0)
static cudaError_t mlp_forward(Mlp *m, int64_t rows, cudaStream_t st)
{
    const size_t per = (size_t)m->cap * m->maxdim;
    for (int l = 0; l < m->nlayer; ++l) {
        const bf16 *X = m->act + per * l;
        const bf16 *W = m->wb + m->woff[l];
        const float *b = m->w + m->boff[l];
        const int di = m->din[l], dn = m->dout[l];
        // C(m,n) = sum_k X(m,k) W(n,k): A = X (sam = di, sak = 1), B(k,n) = W[n*di + k]
        cudaError_t e;
        if (l < m->nlayer - 1)
            e = gemm<EPI_BIAS_GELU>(st, (int)rows, dn, di, X, di, 1, W, 1, di, b, m->zbuf + per * l, dn,
                                    m->act + per * (l + 1), dn, nullptr, 0);
        else
            e = gemm<EPI_BIAS>(st, (int)rows, dn, di, X, di, 1, W, 1, di, b, nullptr, 0, nullptr, 0, m->pred, dn);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// backward pass from dpred (BF16 [rows][nout] in m->dz): gradients into m->g
static cudaError_t mlp_backward(Mlp *m, int64_t rows, cudaStream_t st)
{
    const size_t per = (size_t)m->cap * m->maxdim;
    bf16 *dZ = m->dz, *dX = m->dx;
    for (int l = m->nlayer - 1; l >= 0; --l) {
        const int di = m->din[l], dn = m->dout[l];
        const bf16 *X = m->act + per * l;
        // dW(n,k) = sum_m dZ(m,n) X(m,k): A(n,m) = dZ[m*dn + n] (sam = 1, sak = dn), B(m,k) = X[m*di + k]
        cudaError_t e = gemm<EPI_F32>(st, dn, di, (int)rows, dZ, 1, dn, X, di, 1, nullptr, nullptr, 0, nullptr, 0,
                                      m->g + m->woff[l], di);
        if (e != cudaSuccess) return e;
        colsum_kernel<<<(dn + 127) / 128, 128, 0, st>>>(rows, dn, dZ, m->g + m->boff[l]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (l == 0) break;
        // dX(m,k) = sum_n dZ(m,n) W(n,k), times GELU'(Z_{l-1}): A = dZ (sam = dn, sak = 1), B(n,k) = W[n*di + k]
        const bf16 *W = m->wb + m->woff[l];
        e = gemm<EPI_GELU_BACK>(st, (int)rows, di, dn, dZ, dn, 1, W, di, 1, nullptr, m->zbuf + per * (l - 1), di, dX,
                                di, nullptr, 0);
        if (e != cudaSuccess) return e;
        std::swap(dZ, dX);
    }
    return cudaSuccess;
}

cudaError_t mlp_features(const ColumnArrays &c, float *X, cudaStream_t st)
{
    int64_t n = c.ncol * c.ndep;
    features_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c, X);
    return cudaGetLastError();
}

// loss and gradient for rows idx (device) of X (raw features) / Yt (targets)
cudaError_t mlp_loss_grad(Mlp *m, int64_t rows, const float *X, const float *Yt, const int *idx, double *loss_d,
                          cudaStream_t st)
{
    cudaError_t e = mlp_ensure_work(m, rows);
    if (e != cudaSuccess) return e;
    int64_t n = rows * m->nin;
    standardise_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rows, m->nin, X, idx, m->mean, m->istd, m->act);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = mlp_forward(m, rows, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(loss_d, 0, sizeof(double), st)) != cudaSuccess) return e;
    int64_t no = rows * m->nout;
    mse_kernel<<<(unsigned)((no + 255) / 256), 256, 0, st>>>(rows, m->nout, m->pred, Yt, idx, m->dz, loss_d);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return mlp_backward(m, rows, st);
}

cudaError_t mlp_adam(Mlp *m, float lr, float b1, float b2, float eps, cudaStream_t st)
{
    m->adam_t++;
    float c1 = 1.f / (1.f - std::pow(b1, (float)m->adam_t)), c2 = 1.f / (1.f - std::pow(b2, (float)m->adam_t));
    adam_kernel<<<(unsigned)((m->nparam + 255) / 256), 256, 0, st>>>(m->nparam, m->w, m->g, m->m1, m->m2, lr, b1, b2,
                                                                      eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    to_bf16_kernel<<<(unsigned)((m->nparam + 255) / 256), 256, 0, st>>>(m->nparam, m->w, m->wb);
    return cudaGetLastError();
}

cudaError_t mlp_set_standardisation(Mlp *m, const float *X, const int *idx, int64_t rows, cudaStream_t st)
{
    feature_stats_kernel<<<(m->nin + 127) / 128, 128, 0, st>>>(rows, m->nin, X, idx, m->mean, m->istd);
    return cudaGetLastError();
}

cudaError_t mlp_targets(const ColumnArrays &c, int L, float *Yt, cudaStream_t st)
{
    int64_t n = c.ncol * (int64_t)L * c.ndep;
    targets_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c.ncol, L * c.ndep, c.pops, c.nstar, Yt);
    return cudaGetLastError();
}

const float *mlp_grad(const Mlp *m) { return m->g; }

// predictions for every loaded column, in chunks, applied as start populations
cudaError_t mlp_prepare_predict(Mlp *m, int64_t ncol) { return mlp_ensure_work(m, std::min<int64_t>(16384, ncol)); }

cudaError_t mlp_predict_apply(Mlp *m, const ColumnArrays &c, int L, float *X, float *lnb, int *nfallback_d,
                              cudaStream_t st)
{
    cudaError_t e = mlp_features(c, X, st);
    if (e != cudaSuccess) return e;
    const int64_t chunk = 16384;
    if ((e = mlp_ensure_work(m, std::min<int64_t>(chunk, c.ncol))) != cudaSuccess) return e;
    for (int64_t r0 = 0; r0 < c.ncol; r0 += m->cap) {
        int64_t rows = std::min<int64_t>(m->cap, c.ncol - r0);
        int64_t n = rows * m->nin;
        standardise_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rows, m->nin, X + r0 * m->nin, nullptr,
                                                                         m->mean, m->istd, m->act);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = mlp_forward(m, rows, st)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(lnb + r0 * m->nout, m->pred, rows * m->nout * 4, cudaMemcpyDeviceToDevice, st)) !=
            cudaSuccess)
            return e;
    }
    if ((e = cudaMemsetAsync(nfallback_d, 0, sizeof(int), st)) != cudaSuccess) return e;
    int64_t n = c.ncol * c.ndep;
    apply_guess_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c.ncol, L, c.ndep, lnb, c.nstar, c.nH, c.pops,
                                                                     nfallback_d);
    return cudaGetLastError();
}

}  // namespace rh
