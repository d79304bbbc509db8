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
