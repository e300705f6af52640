// Measured FP32 fused multiply-add throughput of the current GPU: the
// non-tensor arithmetic ceiling that bounds the 16-bit storage modes, whose
// collision is held by instruction issue rather than by DRAM.  The method
// (arXiv 2505.10171) has no counterpart; this is a measurement utility.
#include <cuda_runtime.h>

#include "lbm.h"

namespace {

constexpr int FMA_THREADS = 256;  // threads per CTA
constexpr int FMA_CTAS_PER_SM = 8;  // 2048 resident threads per SM
constexpr int FMA_CHAINS = 8;     // independent multiply-add chains per thread
constexpr int FMA_UNROLL = 16;    // chain steps per loop trip
constexpr int FMA_TRIPS = 2048;

// every thread advances FMA_CHAINS independent chains x <- x a + b; the sum
// of the chains is stored only under a condition the values never meet, which
// keeps every multiply-add live without a store per thread
__global__ void __launch_bounds__(FMA_THREADS) k_fma_peak(float *sink, int trips, float a, float b)
{
    float x[FMA_CHAINS];
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; c++) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int t = 0; t < trips; t++) {
#pragma unroll
        for (int u = 0; u < FMA_UNROLL; u++) {
#pragma unroll
            for (int c = 0; c < FMA_CHAINS; c++) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; c++) s += x[c];
    if (s == -1.0f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" lbm_status lbm_fp32_fma_peak(double *tflops)
{
    if (!tflops) return LBM_ERR_ARG;
    *tflops = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return LBM_ERR_CUDA;
    const int ctas = sms * FMA_CTAS_PER_SM;
    float *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lbm_status status = LBM_ERR_CUDA;
    if (cudaMalloc((void **)&sink, sizeof(float) * ctas) == cudaSuccess &&
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        // a = 1 - 2^-10, b = 2^-10: the chains converge to 1 and stay finite
        const float a = 0.9990234375f, b = 0.0009765625f;
        k_fma_peak<<<ctas, FMA_THREADS, 0, st>>>(sink, FMA_TRIPS / 8, a, b);  // warm-up
        float best = -1.0f;
        bool ok = cudaGetLastError() == cudaSuccess;
        for (int r = 0; r < 5 && ok; r++) {
            float ms = 0.0f;
            ok = cudaEventRecord(e0, st) == cudaSuccess;
            if (ok) k_fma_peak<<<ctas, FMA_THREADS, 0, st>>>(sink, FMA_TRIPS, a, b);
            ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, st) == cudaSuccess &&
                 cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            if (ok && (best < 0.0f || ms < best)) best = ms;
        }
        if (ok && best > 0.0f) {
            const double fma = (double)ctas * FMA_THREADS * FMA_CHAINS * FMA_UNROLL * (double)FMA_TRIPS;
            *tflops = 2.0 * fma / (best * 1e-3) / 1e12;
            status = LBM_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(sink);
    return status;
}
