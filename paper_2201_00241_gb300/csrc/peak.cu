// peak.cu -- FP64 FMA throughput of the device (a measurement utility).
//
// The direction kernel of Algorithm 2 is bound by the FP64 pipe, so the roofline
// it is reported against is the chip's FP64 FMA rate.  This kernel measures that
// rate: every thread runs kChains independent FMA chains for `iters` steps, so the
// pipe, not the latency of one chain, is the limit once a few warps per SM issue.
#include <cuda_runtime.h>

#include "../../include/rh.h"

namespace {

constexpr int kChains = 8;

__global__ void k_fma_rate(double* out, int64_t iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = (double)(threadIdx.x + k);
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" rh_status rh_fp64_fma_rate(int32_t device, int32_t ctas_per_sm, int32_t threads_per_cta, int64_t iters,
                                      double* gflops, float* ms) {
    if (ctas_per_sm < 1 || threads_per_cta < 32 || threads_per_cta > 1024 || threads_per_cta % 32 || iters < 1 ||
        !gflops)
        return RH_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return RH_ECUDA;
    int n_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return RH_ECUDA;
    const int grid = n_sm * ctas_per_sm;
    double* out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rh_status st = RH_ECUDA;
    float t = 0.0f;
    if (cudaMalloc(&out, sizeof(double) * (size_t)grid * threads_per_cta) != cudaSuccess) return RH_ENOMEM;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
        // a = a b + c with b = 1 - 2^-20 and c = 2^-20 stays near 1: no overflow, no denormals
        const double b = 1.0 - 1.0 / 1048576.0, c = 1.0 / 1048576.0;
        k_fma_rate<<<grid, threads_per_cta, 0, s>>>(out, iters / 16 + 1, b, c);   // warm-up
        cudaEventRecord(e0, s);
        k_fma_rate<<<grid, threads_per_cta, 0, s>>>(out, iters, b, c);
        cudaEventRecord(e1, s);
        if (cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess &&
            cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && t > 0.0f) {
            *gflops = 2.0 * kChains * (double)iters * grid * threads_per_cta / (t * 1e-3) * 1e-9;
            if (ms) *ms = t;
            st = RH_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    return st;
}
