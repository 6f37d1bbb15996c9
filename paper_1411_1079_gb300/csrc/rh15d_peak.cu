// rh15d_peak.cu -- measured fused multiply-add rate of the device (FP32 or
// FP64), the denominator of the column kernel's roofline.  Every thread runs
// kChains independent dependent chains x <- x * a + b (kUnroll chains deep per
// loop trip), enough independent work per warp scheduler to keep the FMA pipe
// issuing every cycle; the kernel is timed with CUDA events.
#include <cuda_runtime.h>

#include <cstdio>

#include "rh15d_internal.h"

namespace rh {
namespace {

constexpr int kChains = 16;
constexpr int kUnroll = 4;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(T *sink, long long trips, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (long long i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    // a store the compiler cannot prove dead, never taken for the inputs used
    if (s == (T)-1.2345e-7) sink[threadIdx.x] = s;
}

template <typename T>
cudaError_t run(int nsm, long long trips, T *sink, cudaStream_t st, float *ms)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    cudaEventRecord(e0, st);
    // a, b keep every chain bounded (|a| < 1): x converges to b / (1 - a)
    fma_chain_kernel<T><<<nsm * kBlocksPerSm, kThreads, 0, st>>>(sink, trips, (T)0.999, (T)1e-4);
    e = cudaGetLastError();
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

template <typename T>
cudaError_t measure(double seconds, double *flop_s, double *secs_out)
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    T *sink = nullptr;
    e = cudaMalloc(&sink, kThreads * sizeof(T));
    if (e != cudaSuccess) return e;
    cudaStream_t st;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaFree(sink);
        return e;
    }
    // calibrate the trip count on a short launch, then time one launch of
    // about `seconds`
    long long trips = 256;
    float ms = 0.f;
    for (int k = 0; k < 12 && e == cudaSuccess; ++k) {
        e = run<T>(nsm, trips, sink, st, &ms);
        if (ms > 20.f) break;
        trips *= 4;
    }
    if (e == cudaSuccess) {
        double want = seconds * 1e3 / (ms > 0.f ? ms : 1.f) * (double)trips;
        trips = want < 1.0 ? 1 : (long long)want;
        e = run<T>(nsm, trips, sink, st, &ms);
    }
    if (e == cudaSuccess) {
        const double fma = (double)nsm * kBlocksPerSm * kThreads * kChains * kUnroll * (double)trips;
        *flop_s = 2.0 * fma / (ms * 1e-3);
        if (secs_out) *secs_out = ms * 1e-3;
    }
    cudaStreamDestroy(st);
    cudaFree(sink);
    return e;
}

}  // namespace
}  // namespace rh

extern "C" int rh_fma_peak(int32_t device, int32_t precision, double seconds, double *flop_s_out,
                           double *seconds_out)
{
    if (!flop_s_out || (precision != 0 && precision != 1) || !(seconds > 0.0 && seconds <= 10.0)) return RH_EINVAL;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (cudaSetDevice(device) != cudaSuccess) return RH_ECUDA;
    cudaError_t e = precision == 1 ? rh::measure<float>(seconds, flop_s_out, seconds_out)
                                   : rh::measure<double>(seconds, flop_s_out, seconds_out);
    if (prev >= 0) cudaSetDevice(prev);
    return e == cudaSuccess ? RH_OK : RH_ECUDA;
}
