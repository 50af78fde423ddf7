// mg_probe.cu -- measured FP64 arithmetic rate of the device (the denominator
// of the FP64 roofline of the outer-iteration kernels).
//
// The FP64 outer kernels (residual, norms, face set-up) issue a handful of
// FP64 operations per cell, and on this GPU the FP64 pipe is narrow, so their
// bound is min(HBM bandwidth, FP64 issue rate).  The copy bandwidth is
// measured elsewhere; this file measures the FP64 rate the same way: a kernel
// of independent fused multiply-add chains over every SM, timed with CUDA
// events, best of several launches.
#include "gbmg.h"
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;           // independent FMA chains per thread
constexpr int kProbeThreads = 256;

// Each thread runs kChains chains a <- a * m + c for `iters` steps; the chains
// stay in (0, 2) for m < 1, c small, so no value overflows or goes subnormal.
// The final sums are compared with an impossible value so the chains are live
// without a store per thread.
__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma(double *out, int iters, double m, double c)
{
    double a[kChains];
#pragma unroll
    for (int u = 0; u < kChains; u++) a[u] = 1.0 + 1e-3 * u + 1e-9 * threadIdx.x;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < kChains; u++) a[u] = fma(a[u], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < kChains; u++) s += a[u];
    if (s == -1.0) out[0] = s;
}

}  // namespace

extern "C" int mg_probe_fp64_rate(int iters, int repeats, double *fma_per_s, void *stream)
{
    if (!fma_per_s || iters < 1 || repeats < 1) return MG_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MG_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MG_ECUDA;
    const int blocks = sms * 8;
    cudaStream_t s = (cudaStream_t)stream;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MG_OK;
    double best = 0.0;
    if (cudaMalloc((void **)&out, sizeof(double)) != cudaSuccess) return MG_ENOMEM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = MG_ECUDA;
        goto done;
    }
    k_fp64_fma<<<blocks, kProbeThreads, 0, s>>>(out, iters / 8 + 1, 0.999999, 1e-7);  // warm-up
    for (int r = 0; r < repeats && rc == MG_OK; r++) {
        float ms = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = MG_ECUDA;
        k_fp64_fma<<<blocks, kProbeThreads, 0, s>>>(out, iters, 0.999999, 1e-7);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            rc = MG_ECUDA;
        else if (ms > 0.f) {
            const double ops = (double)blocks * kProbeThreads * kChains * (double)iters;
            const double rate = ops / (ms * 1e-3);
            if (rate > best) best = rate;
        }
    }
    *fma_per_s = best;
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}
