// Measurement probes used as roofline denominators (not part of the method):
// the shared-memory bandwidth of the shared-memory-resident relaxation
// kernels (every SM streams float4 reads from its own shared memory, the
// access width the kernels use for staged positions), and the FP64 issue
// rates of the FP64 kernel's operations (IEEE add/multiply, divide, square
// root: the correctly rounded intrinsics the kernel calls).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fe2_probe.h"

namespace {

__global__ void __launch_bounds__(1024) k_smem_read(float *out, int iters) {
    __shared__ float4 buf[4096];
    for (int i = threadIdx.x; i < 4096; i += blockDim.x)
        buf[i] = make_float4((float)i, (float)i + 1.f, (float)i + 2.f, (float)i + 3.f);
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const int stride = blockDim.x;
    int idx = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
        const float4 v = buf[idx & 4095];
        idx += stride;
        acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc.x + acc.y + acc.z + acc.w;
}

// FP64 throughput: every thread runs kChains independent dependency chains
// of one operation, enough to cover its latency at full occupancy.
constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fp64_fma(double *out, int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __fma_rn(a[k], b, c);
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) t += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void __launch_bounds__(256) k_fp64_div(double *out, int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.5 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __ddiv_rn(b, a[k]) + c;  // stays near 1.2
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) t += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void __launch_bounds__(256) k_fp64_sqrt(double *out, int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.5 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __dsqrt_rn(a[k] * b + c);  // stays near 1.6
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) t += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// Best-of-5 event time of one kernel, in ms.
template <class K>
float best_ms(K kernel, int blocks, int threads, double *out, int iters, double b, double c) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    kernel<<<blocks, threads>>>(out, iters / 10 + 1, b, c);  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0);
        kernel<<<blocks, threads>>>(out, iters, b, c);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

}  // namespace

extern "C" int fe2_probe_fp64_rates(double *fma_per_s, double *div_per_s, double *sqrt_per_s) {
    if (!fma_per_s || !div_per_s || !sqrt_per_s) return 1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 3;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = 8 * sms, threads = 256;
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return 2;
    const double ops = (double)blocks * threads * kChains;
    const int it_fma = 4000, it_div = 400, it_sqrt = 400;
    const float t_fma = best_ms(k_fp64_fma, blocks, threads, out, it_fma, 0.999999, 1e-6);
    const float t_div = best_ms(k_fp64_div, blocks, threads, out, it_div, 1.0, 0.4);
    const float t_sqrt = best_ms(k_fp64_sqrt, blocks, threads, out, it_sqrt, 0.5, 1.8);
    const cudaError_t err = cudaGetLastError();
    cudaFree(out);
    if (err != cudaSuccess) return 3;
    *fma_per_s = ops * it_fma / (t_fma * 1e-3);
    *div_per_s = ops * it_div / (t_div * 1e-3);
    *sqrt_per_s = ops * it_sqrt / (t_sqrt * 1e-3);
    return 0;
}

extern "C" int fe2_probe_smem_bandwidth(double *gbs, double *sm_clock_mhz) {
    if (!gbs) return 1;
    int dev = 0, sms = 0, clk = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 3;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    const int blocks = 2 * sms, threads = 1024, iters = 20000;
    float *out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return 2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_smem_read<<<blocks, threads>>>(out, 1000);  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0);
        k_smem_read<<<blocks, threads>>>(out, iters);
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
    if (err != cudaSuccess) return 3;
    *gbs = 16.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e9;
    if (sm_clock_mhz) *sm_clock_mhz = clk / 1000.0;
    return 0;
}
