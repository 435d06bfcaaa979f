// Shared-memory bandwidth probe used as the roofline denominator of the
// shared-memory-resident relaxation kernels: every SM streams float4 reads
// from its own shared memory (the access width the kernels use for staged
// positions). Not part of the method.
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

}  // namespace

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
