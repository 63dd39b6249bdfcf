// k_peak.cu -- measured FP32 FMA throughput of the device (the denominator
// of the FP32 nearest-codevector kernel's roofline).  No counterpart in the
// paper: it measures the machine, not the method.
//
// Every thread runs CHAINS independent FMA chains (a = a * x + y); 512-thread
// CTAs, two per SM, give 32 warps per SM (8 per sub-partition, 64 independent
// FMAs each), far more than the FMA latency needs.  The chains' results feed one store behind a condition
// that never holds, so the compiler keeps every FMA.
#include "lbgvq.h"
#include "lbg_internal.cuh"

namespace lbg {
namespace {

constexpr int PEAK_THREADS = 512;
constexpr int PEAK_CTAS_PER_SM = 2;
constexpr int CHAINS = 8;
constexpr int UNROLL = 16;

__global__ void __launch_bounds__(PEAK_THREADS) k_ffma_peak(float x, float y, int iters, float *sink)
{
    float a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) a[c] = fmaf(a[c], x, y);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += a[c];
    if (s == -1.2345e30f) sink[threadIdx.x] = s;   // never true for the arguments used
}

}  // namespace
}  // namespace lbg

using namespace lbg;

extern "C" lbg_status lbg_measure_fp32_peak(void *stream, double *tflops, int32_t *sms)
{
    const int n_sm = num_sms();
    if (sms) *sms = n_sm;
    if (!tflops) return LBG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lbg_status rc = LBG_OK;
    // |x| < 1 keeps the chains finite: a -> y / (1 - x)
    const float x = 0.999f, y = 1e-3f;
    const int grid = n_sm * PEAK_CTAS_PER_SM;
    // about 16 ms at ~80 TFLOP/s on 152 SMs; the warm-up launch is a tenth of it
    const int iters = 32768;
    if (cudaMalloc(&sink, sizeof(float) * PEAK_THREADS) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = LBG_ERR_CUDA;
    } else {
        LBG_COUNTED k_ffma_peak<<<grid, PEAK_THREADS, 0, s>>>(x, y, iters / 10, sink);
        cudaEventRecord(e0, s);
        LBG_COUNTED k_ffma_peak<<<grid, PEAK_THREADS, 0, s>>>(x, y, iters, sink);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            ms <= 0.f) {
            rc = LBG_ERR_CUDA;
        } else {
            const double fma = (double)grid * PEAK_THREADS * CHAINS * UNROLL * (double)iters;
            *tflops = 2.0 * fma / (ms * 1e-3) / 1e12;
        }
    }
    (void)cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    return rc;
}
