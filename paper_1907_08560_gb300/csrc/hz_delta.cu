// hz_delta.cu -- the block update of the FP64 sweeps (Section 6.4.3) for pairs
// whose transformation is close to the identity, in the delta form
//   [X_P X_Q] <- [X_P X_Q] + [X_P X_Q] E,   E = Z^ - I,
// with the product X E formed from FP32 roundings of X and E by FP32 FMAs and
// the sum taken in FP64.
//
// Accuracy: the FP32 product's error per entry is at most about
// (kk + 2) 2^-24 sum_l |x_il||e_lj| (rounding of X and E, FP32 accumulation of
// kk terms); with every entry of E at most DELTA_E = 2^-29 in real and
// imaginary part that is about 2^-47 sum_l |x_il| at kk = 64.  The FP64
// product's own bound, gamma_kk sum_l |x_il||z_lj|, is about 2^-47 |x_ij|, so
// for a row of comparable entries the FP32 product's bound is up to kk times
// larger; its typical (random-walk) error, about sqrt(kk) 2^-53 |x|, is the
// FP64 product's.  The sum is exact for an untouched column (E's column
// zero).  Late in an iteration most pairs
// rotate by far less than that (the big/small test of Section 6.1.7 already
// calls every rotation with sin < 2^-27 small), and the FP32 pipe of this GPU
// is 64 times faster than its FP64 pipe, so the update of those pairs becomes
// bound by HBM instead of by the FP64 pipe.  Pairs with larger entries keep
// the FP64 update (route64_kernel decides, per pair and step).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/ghsvd.h"
#include "hz_common.cuh"
#include "hz_delta.cuh"
#include "hz_launch.h"

namespace hz {

__global__ void route64_kernel(const double2 *__restrict__ zhat, const int *__restrict__ pair_flag, int kk,
                               int *__restrict__ delta_flag, int *__restrict__ df_flag,
                               int *__restrict__ full_flag, unsigned long long *__restrict__ count)
{
    const int pair = blockIdx.x;
    const bool active = pair_flag[pair] != 0;
    const int c = active ? route_class(zhat + (long long)pair * (KKMAX * KKMAX), kk) : 0;
    if (threadIdx.x == 0) {
        delta_flag[pair] = active && c == 0;
        df_flag[pair] = active && c == 1;
        full_flag[pair] = active && c == 2;
        if (active) atomicAdd(count + (c == 0 ? 0 : c == 1 ? 2 : 1), 1ull);
    }
}

// One CTA per (64-row tile, pair).
__global__ void __launch_bounds__(256)
update_delta64_kernel(double2 *__restrict__ W, StepArgs a, const double2 *__restrict__ zhat,
                      const int *__restrict__ delta_flag)
{
    const int pair = blockIdx.y;
    if (!delta_flag[pair]) return;
    extern __shared__ unsigned char smraw[];
    delta64_tile(W, a.ld, a.slotcol + pair * a.kk, a.kk, (long long)blockIdx.x * UPD_R,
                 zhat + (long long)pair * (KKMAX * KKMAX), smraw);
}

// One CTA per (32-row tile, pair), two CTAs per SM.
__global__ void __launch_bounds__(256, 2)
update_df64_kernel(double2 *__restrict__ W, StepArgs a, const double2 *__restrict__ zhat,
                   const int *__restrict__ df_flag)
{
    const int pair = blockIdx.y;
    if (!df_flag[pair]) return;
    extern __shared__ unsigned char smraw[];
    df64_tile(W, a.ld, a.slotcol + pair * a.kk, a.kk, (long long)blockIdx.x * DF_R,
              zhat + (long long)pair * (KKMAX * KKMAX), smraw);
}

cudaError_t delta64_setup()
{
    cudaError_t e = cudaFuncSetAttribute(update_delta64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)delta64_smem());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(update_df64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)df64_smem());
}

cudaError_t launch_route64(const double2 *zhat, const int *pair_flag, int kk, int npairs, int *delta_flag,
                           int *df_flag, int *full_flag, unsigned long long *count, cudaStream_t s)
{
    route64_kernel<<<npairs, 256, 0, s>>>(zhat, pair_flag, kk, delta_flag, df_flag, full_flag, count);
    return cudaGetLastError();
}

cudaError_t launch_update_df64(double2 *W, const StepArgs &a, const double2 *zhat, const int *df_flag,
                               cudaStream_t s)
{
    const long long Mt = (long long)a.m_pad + a.p_pad + a.n_pad;
    dim3 grid((unsigned)(Mt / DF_R), a.npairs);
    update_df64_kernel<<<grid, 256, df64_smem(), s>>>(W, a, zhat, df_flag);
    return cudaGetLastError();
}

cudaError_t launch_update_delta64(double2 *W, const StepArgs &a, const double2 *zhat, const int *delta_flag,
                                  cudaStream_t s)
{
    const long long Mt = (long long)a.m_pad + a.p_pad + a.n_pad;
    dim3 grid((unsigned)(Mt / UPD_R), a.npairs);
    update_delta64_kernel<<<grid, 256, delta64_smem(), s>>>(W, a, zhat, delta_flag);
    return cudaGetLastError();
}

namespace {

__global__ void block_update_setup(int *slotcol, int *flag)
{
    const int t = threadIdx.x;
    if (t < KKMAX) slotcol[t] = t;
    if (t == 0) flag[0] = 1;
}

}  // namespace
}  // namespace hz

extern "C" ghsvd_status ghsvd_fp64_block_update(int64_t rows, void *X, int64_t ldx, const void *Z, int route,
                                                void *stream)
{
    if (rows < 64 || rows % 64 != 0 || rows > (1 << 24) || ldx < rows || !X || !Z || route < 0 || route > 2)
        return GHSVD_ERR_INVALID_ARG;
    int dev = 0;
    cudaPointerAttributes ax{}, az{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&ax, X) != cudaSuccess ||
        cudaPointerGetAttributes(&az, Z) != cudaSuccess) {
        cudaGetLastError();
        return GHSVD_ERR_INVALID_ARG;
    }
    auto dev_ok = [dev](const cudaPointerAttributes &p) {
        return (p.type == cudaMemoryTypeDevice || p.type == cudaMemoryTypeManaged) && p.device == dev;
    };
    if (!dev_ok(ax) || !dev_ok(az)) return GHSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (hz::delta64_setup() != cudaSuccess || hz::setup_kernels() != cudaSuccess) return GHSVD_ERR_CUDA;
    int *slotcol = nullptr, *flag = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&slotcol, hz::KKMAX * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&flag, sizeof(int), st);
    if (e == cudaSuccess) {
        hz::block_update_setup<<<1, 64, 0, st>>>(slotcol, flag);
        e = cudaGetLastError();
    }
    hz::StepArgs sa{};
    sa.slotcol = slotcol;
    sa.npairs = 1;
    sa.kk = hz::KKMAX;
    sa.m_pad = (int)rows;
    sa.p_pad = 0;
    sa.n_pad = 0;
    sa.ld = ldx;
    const double2 *zp = (const double2 *)Z;
    if (e == cudaSuccess) {
        if (route == 0) e = hz::launch_update_delta64((double2 *)X, sa, zp, flag, st);
        else if (route == 1) e = hz::launch_update_df64((double2 *)X, sa, zp, flag, st);
        else e = hz::launch_update(X, false, sa, zp, flag, st);
    }
    cudaFreeAsync(slotcol, st);
    cudaFreeAsync(flag, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? GHSVD_OK : (e == cudaErrorMemoryAllocation ? GHSVD_ERR_NOMEM : GHSVD_ERR_CUDA);
}
