// peak_probe.cu -- measures the FP64 DFMA throughput of the current device
// (the roofline denominator of the FP64 kernels): 8 independent fma chains
// per thread, 8 CTAs of 256 threads per SM, timed with CUDA events after a
// warm-up launch.  Built as its own small library, separate from libghsvd.
#include <cuda_runtime.h>

__global__ void dfma_chains(double *out, int iters, double b, double c)
{
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" int hzpeak_fp64_tflops(int device, double *tflops)
{
    if (!tflops) return 1;
    *tflops = 0.0;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return 2;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * 8, threads = 256, iters = 4096;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) rc = 3;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = 4;
    float best = 1e30f;
    for (int rep = 0; !rc && rep < 3; ++rep) {
        cudaEventRecord(e0);
        dfma_chains<<<blocks, threads>>>(out, iters, 1.0000001, 1e-9);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = 5; break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    if (!rc) *tflops = 2.0 * 8 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    cudaSetDevice(prev);
    return rc;
}

// FP64 through the legacy tensor path (mma.sync m8n8k4, DMMA), for the
// record: on this GPU it is slower than plain DFMA.
__global__ void dmma_chains(double *out, int iters)
{
    const double a = 1.0 + threadIdx.x * 1e-6, b = 0.999999;
    double d[8][2];
#pragma unroll
    for (int k = 0; k < 8; ++k) { d[k][0] = k; d[k][1] = -k; }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(d[k][0]), "+d"(d[k][1]) : "d"(a), "d"(b));
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += d[k][0] + d[k][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void ffma_chains(float *out, int iters, float b, float c)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// which: 0 = FP64 DFMA, 1 = FP64 DMMA, 2 = FP32 FFMA.  Best of 2 timed runs.
extern "C" int hzpeak_tflops(int device, int which, double *tflops)
{
    if (!tflops || which < 0 || which > 2) return 1;
    if (which == 0) return hzpeak_fp64_tflops(device, tflops);
    *tflops = 0.0;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return 2;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * 8, threads = 256;
    const int iters = which == 1 ? 1024 : 65536;
    void *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) rc = 3;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = 4;
    float best = 1e30f;
    for (int rep = 0; !rc && rep < 3; ++rep) {
        cudaEventRecord(e0);
        if (which == 1) dmma_chains<<<blocks, threads>>>((double *)out, iters);
        else ffma_chains<<<blocks, threads>>>((float *)out, iters, 1.0000001f, 1e-9f);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = 5; break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    if (!rc) {
        const double flop = which == 1 ? 2.0 * 256 * 8 * iters * (double)blocks * (threads / 32)
                                       : 2.0 * 8 * iters * (double)blocks * threads;
        *tflops = flop / (best * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    cudaSetDevice(prev);
    return rc;
}
