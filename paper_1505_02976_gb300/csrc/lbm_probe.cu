// lbm_probe.cu -- FP64 fused multiply-add throughput of the device: the
// denominator of the FP64 step's roofline (that step is bound by the FP64
// pipe, not by memory).  The paper has no counterpart; this is a
// measurement helper.
#include <cuda_runtime.h>

#include "lbm.h"

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread (hide the pipe latency)
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__device__ double g_probe_sink;

// Every thread runs kChains independent chains a <- a * b + c for `iters`
// rounds.  The sum of the chains is stored only if it equals -1, which it
// never does for the inputs below (0 < a, b < 1, c > 0), so the compiler must
// keep every FMA while the kernel writes nothing.
__global__ void __launch_bounds__(kThreads) k_fp64_fma(int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 0.25 + 1e-3 * (threadIdx.x & 31) + 1e-2 * j;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -1.0) g_probe_sink = s;
}

}  // namespace

extern "C" lbm_status lbm_fp64_peak(void* stream, double* flops_per_s) {
    if (!flops_per_s) return LBM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaStreamGetDevice(st, &dev) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LBM_ERR_CUDA;
    const int blocks = sms * kBlocksPerSm;
    const int iters = 20000;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LBM_ERR_CUDA;
    }
    k_fp64_fma<<<blocks, kThreads, 0, st>>>(iters / 10, 0.999999, 1e-7);  // warm-up
    cudaEventRecord(e0, st);
    k_fp64_fma<<<blocks, kThreads, 0, st>>>(iters, 0.999999, 1e-7);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0.f) return LBM_ERR_CUDA;
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
    *flops_per_s = flops / (ms * 1e-3);
    return LBM_OK;
}
