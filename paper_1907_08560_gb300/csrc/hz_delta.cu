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
// product's own bound, gamma_kk sum_l |x_il||z_lj|, is about 2^-47 |x_ij|:
// the two have the same size for the rows of comparable entries the stacked
// factors hold, and the typical (random-walk) error of the FP32 product is
// far below its bound.  The sum is exact for an untouched column (E's column
// zero).  Late in an iteration most pairs
// rotate by far less than that (the big/small test of Section 6.1.7 already
// calls every rotation with sin < 2^-27 small), and the FP32 pipe of this GPU
// is 64 times faster than its FP64 pipe, so the update of those pairs becomes
// bound by HBM instead of by the FP64 pipe.  Pairs with larger entries keep
// the FP64 update (route64_kernel decides, per pair and step).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hz_common.cuh"
#include "hz_launch.h"

namespace hz {

constexpr double DELTA_E = 1.0 / 536870912.0;    // 2^-29

// delta_flag[p] = 1 iff pair p applied a transformation and every entry of
// E = Z^ - I is at most DELTA_E in real and imaginary part; full_flag[p] = 1
// for the other pairs with a transformation; count[0] += pairs on the delta
// path, count[1] += pairs on the FP64 path.
__global__ void route64_kernel(const double2 *__restrict__ zhat, const int *__restrict__ pair_flag, int kk,
                               int *__restrict__ delta_flag, int *__restrict__ full_flag,
                               unsigned long long *__restrict__ count)
{
    __shared__ int large;
    const int pair = blockIdx.x;
    if (threadIdx.x == 0) large = 0;
    __syncthreads();
    const bool active = pair_flag[pair] != 0;
    if (active) {
        const double2 *zp = zhat + (long long)pair * (KKMAX * KKMAX);
        bool big = false;
        for (int e = threadIdx.x; e < kk * kk; e += blockDim.x) {
            const int l = e % kk, j = e / kk;
            const double2 z = zp[l + KKMAX * j];
            const double ex = z.x - (l == j ? 1.0 : 0.0);
            big |= !(fabs(ex) <= DELTA_E) || !(fabs(z.y) <= DELTA_E);   // NaN counts as large
        }
        if (big) large = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int d = active && !large;
        delta_flag[pair] = d;
        full_flag[pair] = active && large;
        if (d) atomicAdd(count, 1ull);
        else if (active) atomicAdd(count + 1, 1ull);
    }
}

// One CTA per (64-row tile, pair): the FP64 row tile and E in FP32 in shared
// memory, 16 x 16 threads with 4 x 4 outputs each (rows ty + 16 i, columns
// tx + 16 j), four FP32 FMA chains per complex product, the sum in FP64.
__global__ void __launch_bounds__(256)
update_delta64_kernel(double2 *__restrict__ W, StepArgs a, const double2 *__restrict__ zhat,
                      const int *__restrict__ delta_flag)
{
    const int pair = blockIdx.y;
    if (!delta_flag[pair]) return;
    extern __shared__ unsigned char smraw[];
    double2 *xs = reinterpret_cast<double2 *>(smraw);              // [UPD_R][UPD_LD] FP64 rows
    float2 *es = reinterpret_cast<float2 *>(xs + UPD_R * UPD_LD);   // [KKMAX][UPD_LD] E, row l, column j
    __shared__ int cols[KKMAX];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int kk = a.kk;
    const int *slot = a.slotcol + pair * kk;
    const long long row0 = (long long)blockIdx.x * UPD_R;
    if (tid < KKMAX) cols[tid] = tid < kk ? slot[tid] : -1;
    const double2 *zp = zhat + (long long)pair * (KKMAX * KKMAX);
    for (int idx = tid; idx < KKMAX * KKMAX; idx += 256) {
        const int l = idx % KKMAX, j = idx / KKMAX;
        float2 e = make_float2(0.0f, 0.0f);
        if (l < kk && j < kk) {
            const double2 z = zp[l + KKMAX * j];
            e = make_float2((float)(z.x - (l == j ? 1.0 : 0.0)), (float)z.y);
        }
        es[l * UPD_LD + j] = e;
    }
    __syncthreads();                               // cols
    for (int idx = tid; idx < UPD_R * KKMAX; idx += 256) {
        const int r = idx % UPD_R, s = idx / UPD_R;
        const int col = cols[s];
        if (col >= 0) cp_async<16>(&xs[r * UPD_LD + s], &W[(long long)col * a.ld + row0 + r]);
        else xs[r * UPD_LD + s] = make_double2(0.0, 0.0);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    float pr[4][4], pi[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { pr[i][j] = 0.0f; pi[i][j] = 0.0f; }
    for (int l = 0; l < kk; ++l) {
        float2 x[4], e[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double2 v = xs[(ty + 16 * i) * UPD_LD + l];
            x[i] = make_float2((float)v.x, (float)v.y);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) e[j] = es[l * UPD_LD + tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                pr[i][j] = fmaf(x[i].x, e[j].x, pr[i][j]);
                pr[i][j] = fmaf(-x[i].y, e[j].y, pr[i][j]);
                pi[i][j] = fmaf(x[i].x, e[j].y, pi[i][j]);
                pi[i][j] = fmaf(x[i].y, e[j].x, pi[i][j]);
            }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = ty + 16 * i, c = tx + 16 * j;
            const int col = cols[c];
            if (col < 0) continue;
            const double2 v = xs[r * UPD_LD + c];
            W[(long long)col * a.ld + row0 + r] = make_double2(v.x + (double)pr[i][j], v.y + (double)pi[i][j]);
        }
}

size_t delta64_smem() { return sizeof(double2) * UPD_R * UPD_LD + sizeof(float2) * KKMAX * UPD_LD; }

cudaError_t delta64_setup()
{
    return cudaFuncSetAttribute(update_delta64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)delta64_smem());
}

cudaError_t launch_route64(const double2 *zhat, const int *pair_flag, int kk, int npairs, int *delta_flag,
                           int *full_flag, unsigned long long *count, cudaStream_t s)
{
    route64_kernel<<<npairs, 256, 0, s>>>(zhat, pair_flag, kk, delta_flag, full_flag, count);
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

}  // namespace hz
