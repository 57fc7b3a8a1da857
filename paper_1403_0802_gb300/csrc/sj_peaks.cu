// sj_peaks.cu -- instruction-rate microbenchmarks for the roofline of the
// refinement kernels, which are bound by plain FP32 / FP64 arithmetic (no
// tensor-core path: nothing in the join is a dense contraction).
//
// Each kernel runs 8 independent dependency chains per thread so the pipes
// stay full; the rate is ops / (SM cycles x SMs), with cycles read by
// clock64() on every SM, and ops / second from CUDA events.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sj_peaks.h"

namespace {

constexpr int CHAINS = 8;

template <typename T>
__global__ void k_fma_rate(T *sink, int iters, T b, T c, unsigned long long *cycles) {
    T a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (T)(threadIdx.x + k);
    unsigned long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    unsigned long long t1 = clock64();
    T s = 0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == (T)12345.678) sink[0] = s;   // keeps the chains alive
    if (threadIdx.x == 0) atomicMax(cycles, t1 - t0);
}

template <typename T>
__global__ void k_add_rate(T *sink, int iters, T b, unsigned long long *cycles) {
    T a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (T)(threadIdx.x + k);
    unsigned long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = a[k] + b;
    }
    unsigned long long t1 = clock64();
    T s = 0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == (T)12345.678) sink[0] = s;
    if (threadIdx.x == 0) atomicMax(cycles, t1 - t0);
}

template <class Launch>
static int time_kernel(Launch launch, unsigned long long *dcyc, double *ms_out, double *cyc_out) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -4;
    launch();   // warm-up
    cudaMemset(dcyc, 0, sizeof(unsigned long long));
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -4;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long cyc = 0;
    cudaMemcpy(&cyc, dcyc, sizeof(cyc), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = ms;
    *cyc_out = (double)cyc;
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

}  // namespace

extern "C" int sj_peaks_measure(sj_peak_rates *out) {
    if (!out) return -1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -4;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double *sink = nullptr;
    unsigned long long *dcyc = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess || cudaMalloc(&dcyc, 8) != cudaSuccess) return -2;
    const int threads = 256, blocks = sms * 8;
    const double nthr = (double)threads * blocks;
    int rc = 0;
    double ms, cyc;
    const int it32 = 4096, it64 = 256;
    rc |= time_kernel([&] { k_fma_rate<float><<<blocks, threads>>>((float *)sink, it32, 0.999f, 0.001f, dcyc); },
                      dcyc, &ms, &cyc);
    double ops = nthr * CHAINS * it32;
    out->ffma_per_s = ops / (ms * 1e-3);
    out->ffma_per_clk_sm = ops / (cyc * sms);
    rc |= time_kernel([&] { k_add_rate<float><<<blocks, threads>>>((float *)sink, it32, 0.001f, dcyc); }, dcyc, &ms,
                      &cyc);
    out->fadd_per_s = ops / (ms * 1e-3);
    out->fadd_per_clk_sm = ops / (cyc * sms);
    rc |= time_kernel([&] { k_fma_rate<double><<<blocks, threads>>>(sink, it64, 0.999, 0.001, dcyc); }, dcyc, &ms,
                      &cyc);
    ops = nthr * CHAINS * it64;
    out->dfma_per_s = ops / (ms * 1e-3);
    out->dfma_per_clk_sm = ops / (cyc * sms);
    rc |= time_kernel([&] { k_add_rate<double><<<blocks, threads>>>(sink, it64, 0.001, dcyc); }, dcyc, &ms, &cyc);
    out->dadd_per_s = ops / (ms * 1e-3);
    out->dadd_per_clk_sm = ops / (cyc * sms);
    out->sms = sms;
    cudaFree(sink);
    cudaFree(dcyc);
    return rc ? -4 : 0;
}
