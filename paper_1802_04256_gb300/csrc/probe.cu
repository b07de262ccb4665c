// FP64 throughput probes (DFMA pipe and FP64 tensor-core mma.sync).
#include <algorithm>

#include "../../include/rpim_probe.h"
#include "common.cuh"

namespace rpim {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) dfma_probe_kernel(double *out, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = 1e-3 * threadIdx.x + k;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) dmma_probe_kernel(double *out, int iters, double a)
{
    // four independent m8n8k4 accumulators per warp; A and B fragments are
    // one double per lane each, C/D two doubles per lane
    double fa = a + 1e-9 * (threadIdx.x & 31), fb = 1.0 - 1e-9 * (threadIdx.x & 31);
    double c[4][2];
#pragma unroll
    for (int k = 0; k < 4; k++) { c[k][0] = 0.0; c[k][1] = 0.0; }
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 4; k++)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                         : "+d"(c[k][0]), "+d"(c[k][1])
                         : "d"(fa), "d"(fb));
        fa *= 0.999999999;
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 4; k++) s += c[k][0] + c[k][1];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// even warps run the DFMA chains, odd warps the mma.sync loop: whether the
// two FP64 paths add up (separate units) or share one rate
__global__ void __launch_bounds__(256) mixed_probe_kernel(double *out, int iters_f, int iters_m, double a, double b)
{
    double s = 0.0;
    if (((threadIdx.x >> 5) & 1) == 0) {
        double x[kChains];
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = 1e-3 * threadIdx.x + k;
        for (int i = 0; i < iters_f; i++) {
#pragma unroll
            for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
        }
#pragma unroll
        for (int k = 0; k < kChains; k++) s += x[k];
    } else {
        double fa = a + 1e-9 * (threadIdx.x & 31), fb = 1.0 - 1e-9 * (threadIdx.x & 31);
        double c[4][2];
#pragma unroll
        for (int k = 0; k < 4; k++) { c[k][0] = 0.0; c[k][1] = 0.0; }
        for (int i = 0; i < iters_m; i++) {
#pragma unroll
            for (int k = 0; k < 4; k++)
                asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                             : "+d"(c[k][0]), "+d"(c[k][1])
                             : "d"(fa), "d"(fb));
            fa *= 0.999999999;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) s += c[k][0] + c[k][1];
    }
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class Launch>
static rpim_status time_best(int repeats, double flops, Launch launch, double *gflops)
{
    cudaEvent_t e0, e1;
    RPIM_CUDA(cudaEventCreate(&e0));
    RPIM_CUDA(cudaEventCreate(&e1));
    launch(); // warm-up
    RPIM_CUDA(cudaGetLastError());
    float best = 1e30f;
    for (int r = 0; r < std::max(1, repeats); r++) {
        RPIM_CUDA(cudaEventRecord(e0));
        launch();
        RPIM_CUDA(cudaEventRecord(e1));
        RPIM_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        RPIM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *gflops = flops / (best * 1e-3) / 1e9;
    return RPIM_OK;
}

} // namespace rpim

using namespace rpim;

extern "C" rpim_status rpim_probe_dfma(int32_t repeats, double *gflops)
{
    if (!gflops) return fail(RPIM_E_ARG, "null gflops");
    int dev = 0, sms = 0;
    RPIM_CUDA(cudaGetDevice(&dev));
    RPIM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256, iters = 4096;
    double *out = nullptr;
    note_device_alloc();
    RPIM_CUDA(cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)));
    const double flops = 2.0 * kChains * (double)iters * blocks * threads;
    rpim_status st = time_best(repeats, flops, [&] { dfma_probe_kernel<<<blocks, threads>>>(out, iters, 0.9999999, 1e-7); }, gflops);
    cudaFree(out);
    return st;
}

extern "C" rpim_status rpim_probe_dmma(int32_t repeats, double *gflops)
{
    if (!gflops) return fail(RPIM_E_ARG, "null gflops");
    int dev = 0, sms = 0;
    RPIM_CUDA(cudaGetDevice(&dev));
    RPIM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256, iters = 1024;
    double *out = nullptr;
    note_device_alloc();
    RPIM_CUDA(cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)));
    const double flops = 512.0 * 4 * (double)iters * blocks * (threads / 32);
    rpim_status st = time_best(repeats, flops, [&] { dmma_probe_kernel<<<blocks, threads>>>(out, iters, 1.0); }, gflops);
    cudaFree(out);
    return st;
}

extern "C" rpim_status rpim_probe_fp64_mixed(int32_t repeats, double *gflops)
{
    if (!gflops) return fail(RPIM_E_ARG, "null gflops");
    int dev = 0, sms = 0;
    RPIM_CUDA(cudaGetDevice(&dev));
    RPIM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // per warp: DFMA 2*8*32*iters_f flops, mma 512*4*iters_m flops; equal
    // work per half at iters_f = 4 iters_m
    const int blocks = sms * 8, threads = 256, iters_m = 1024, iters_f = 4 * iters_m;
    double *out = nullptr;
    note_device_alloc();
    RPIM_CUDA(cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)));
    const double warps = (double)blocks * (threads / 32) / 2;
    const double flops = warps * (2.0 * kChains * 32 * iters_f + 512.0 * 4 * iters_m);
    rpim_status st = time_best(repeats, flops,
                               [&] { mixed_probe_kernel<<<blocks, threads>>>(out, iters_f, iters_m, 0.9999999, 1e-7); },
                               gflops);
    cudaFree(out);
    return st;
}
