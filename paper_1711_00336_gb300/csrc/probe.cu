// probe.cu -- measured FP64 throughput of the GPU, the denominator of the
// roofline of the FP64-bound kernels (the DEM pair chain, the FP64
// collide-stream).  Not part of the method: a dense chain of independent
// fused multiply-adds on every SM, timed with CUDA events.  Also the check
// entry of the lubrication term's logarithm (tlog.cuh) on the host or the
// device, beside the library logarithm.
#include <cuda_runtime.h>

#include "dps.h"
#include "tlog.cuh"

namespace {

constexpr int CHAINS = 8;     // independent FMA chains per thread
constexpr int ITERS = 4096;   // FMAs per chain

__global__ void __launch_bounds__(256) k_fma64(double seed, double *out) {
    double a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
    const double m = 0.9999999, b = 1e-7;
    for (int k = 0; k < ITERS; ++k) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) a[c] = fma(a[c], m, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += a[c];
    if (s == 12345.678) out[0] = s;  // keeps the chains live; never true
}

__global__ void k_tlog_check(const double *x, double *y, double *y_lib, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        y[i] = dps::tlog(x[i]);
        y_lib[i] = log(x[i]);
    }
}

}  // namespace

extern "C" int dps_check_tlog(const double *x, double *y, double *y_lib, int64_t n, int device) {
    if (n < 0 || (n && (!x || !y || !y_lib))) return DPS_ERR_ARG;
    if (!device) {
        for (int64_t i = 0; i < n; ++i) {
            y[i] = dps::tlog(x[i]);
            y_lib[i] = std::log(x[i]);
        }
        return DPS_OK;
    }
    if (n == 0) return DPS_OK;
    double *d = nullptr;
    const size_t bytes = sizeof(double) * (size_t)n;
    if (cudaMalloc(&d, 3 * bytes) != cudaSuccess) {
        cudaGetLastError();
        return DPS_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_tlog_check<<<256, 256>>>(d, d + n, d + 2 * n, (long long)n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(y, d + n, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(y_lib, d + 2 * n, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DPS_ERR_CUDA;
    }
    return DPS_OK;
}

extern "C" int dps_probe_fp64_peak(double *gflops) {
    if (!gflops) return DPS_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return DPS_ERR_CUDA;
    }
    double *out = nullptr;
    cudaEvent_t e0, e1;
    if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return DPS_ERR_OOM;
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * 8, threads = 256;
    k_fma64<<<blocks, threads>>>(1.0, out);  // warm-up
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0);
        k_fma64<<<blocks, threads>>>(1.0 + r, out);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return DPS_ERR_CUDA;
    const double flops = 2.0 * (double)blocks * threads * CHAINS * ITERS;
    *gflops = flops / (best * 1e-3) / 1e9;
    return DPS_OK;
}
