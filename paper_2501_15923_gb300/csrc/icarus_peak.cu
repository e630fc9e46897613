// icarus_peak.cu -- measured fused multiply-add rate of this GPU in double and single precision:
// the denominator of the arithmetic roofline that bounds the FP64 solver (its flux and update
// kernels are limited by the FP64 pipe, not by HBM).
//
// Every thread runs `chains` independent FMA recurrences x <- x * a + b for `iters` rounds (so the
// pipe always has independent work; chains = 1 gives the dependent, latency-bound rate). The
// grid is blocks_per_sm x the SM count of 256-thread blocks. The rate is
// 2 flop x threads x chains x iters / the kernel's CUDA-event duration (one warm-up launch first).
#include <cuda_runtime.h>

#include "../../include/icarus.h"
#include "icarus_ops.h"

namespace {

__device__ double g_sink_d;   // written only when a result takes an impossible value: keeps the chains
__device__ float g_sink_f;

__device__ __forceinline__ double fma_rn(double x, double a, double b) { return __fma_rn(x, a, b); }
__device__ __forceinline__ float fma_rn(float x, float a, float b) { return __fmaf_rn(x, a, b); }

template <typename T, int CH>
__global__ void __launch_bounds__(256) k_fma_rate(long long iters, T a, T b)
{
    T x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = T(threadIdx.x + 1 + 37 * c) * T(1e-3);
    for (long long it = 0; it < iters; it += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) x[c] = fma_rn(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    if (s == T(-1.25)) {
        if (sizeof(T) == 8) g_sink_d = (double)s;
        else g_sink_f = (float)s;
    }
}

template <typename T, int CH>
cudaError_t launch(int blocks, long long iters, cudaStream_t st)
{
    // x -> b / (1 - a) = 1: the recurrence stays finite and normal for any number of rounds
    k_fma_rate<T, CH><<<blocks, 256, 0, st>>>(iters, T(0.999), T(0.001));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_chains(int chains, int blocks, long long iters, cudaStream_t st)
{
    switch (chains) {
    case 1: return launch<T, 1>(blocks, iters, st);
    case 4: return launch<T, 4>(blocks, iters, st);
    case 8: return launch<T, 8>(blocks, iters, st);
    default: return launch<T, 16>(blocks, iters, st);
    }
}

}  // namespace

extern "C" int icarus_fma_rate(int precision, int chains, int blocks_per_sm, long long iters, double *tflops,
                               double *ms)
{
    if (!tflops || !ms) return icarus::report_error(ICARUS_EINVAL, "NULL argument");
    if (precision != ICARUS_FP64 && precision != ICARUS_FP32)
        return icarus::report_error(ICARUS_EINVAL, "precision must be ICARUS_FP64 or ICARUS_FP32");
    if (chains != 1 && chains != 4 && chains != 8 && chains != 16)
        return icarus::report_error(ICARUS_EINVAL, "chains must be 1, 4, 8 or 16");
    if (blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 4 || iters > (1LL << 40) || iters % 4)
        return icarus::report_error(ICARUS_EINVAL, "need blocks_per_sm in [1, 8] and iters a multiple of 4 in [4, 2^40]");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return icarus::report_error(ICARUS_ECUDA, "no CUDA device");
    const int blocks = sms * blocks_per_sm;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return icarus::report_error(ICARUS_ECUDA, "stream creation failed");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto run = [&](long long n) {
        return precision == ICARUS_FP64 ? launch_chains<double>(chains, blocks, n, st)
                                        : launch_chains<float>(chains, blocks, n, st);
    };
    cudaError_t e = run(iters);                       // warm-up (clocks up, code loaded)
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = run(iters);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) return icarus::report_error(ICARUS_ECUDA, cudaGetErrorString(e));
    *ms = t;
    *tflops = 2.0 * blocks * 256.0 * chains * (double)iters / (t * 1e-3) / 1e12;
    return ICARUS_OK;
}
