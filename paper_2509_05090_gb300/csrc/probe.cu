// Measured FP64 peak of the device: the roofline denominator of the FP64
// contractions (GB300 has no FP64 tensor-core kind, so the DFMA pipe is the
// FP64 ceiling).  Each thread runs NCH independent chains of dependent fused
// multiply-adds, enough to cover the pipe's latency; the result is written out
// so the chains are not optimised away.
#include "ctm_ctx.h"

namespace {

constexpr int PROBE_NCH = 16;
constexpr int PROBE_ITERS = 4096;
constexpr int PROBE_THREADS = 256;

__device__ double g_probe_sink;   // the chains' sum lands here in the (never taken) branch below

__global__ void __launch_bounds__(PROBE_THREADS) dfma_probe_kernel(double a, double b)
{
    double x[PROBE_NCH];
#pragma unroll
    for (int i = 0; i < PROBE_NCH; ++i) x[i] = (double)(threadIdx.x + i) * 1e-3;
    for (int it = 0; it < PROBE_ITERS; ++it) {
#pragma unroll
        for (int i = 0; i < PROBE_NCH; ++i) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < PROBE_NCH; ++i) s += x[i];
    if (s == 12345.678) g_probe_sink = s;   // keeps the chains live
}

}  // namespace

extern "C" int ctm_probe_fp64_peak(void *stream, double *tflops_host)
{
    if (!tflops_host) return CTM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = 4 * device_sm_count();
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return CTM_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return CTM_ECUDA;
    }
    int rc = CTM_OK;
    float best = 1e30f;
    for (int rep = 0; rep < 4 && rc == CTM_OK; ++rep) {   // first launch warms up
        cudaEventRecord(e0, st);
        dfma_probe_kernel<<<blocks, PROBE_THREADS, 0, st>>>(0.999999, 1e-7);
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = CTM_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep && ms < best) best = ms;
    }
    CTM_COUNT_LAUNCH(4);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CTM_OK) return rc;
    const double flops = 2.0 * PROBE_NCH * (double)PROBE_ITERS * PROBE_THREADS * blocks;
    *tflops_host = flops / (best * 1e-3) / 1e12;
    return CTM_OK;
}
