// hz_delta.cuh -- the delta-form updates of the FP64 sweeps (Section 6.4.3) for
// pairs whose transformation is close to the identity,
//   [X_P X_Q] <- [X_P X_Q] + [X_P X_Q] E,   E = Z^ - I,
// the product X E in FP32 (every entry of E at most 2^-29) or in double-float
// arithmetic (at most 2^-11), the sum in FP64; device bodies shared by the
// single-pencil kernels (hz_delta.cu) and the batched update (hz_batch.cu).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hz_common.cuh"
#include "hz_launch.h"

namespace hz {

constexpr double DELTA_E = 1.0 / 536870912.0;    // 2^-29
constexpr double DF_E = 1.0 / 2048.0;             // 2^-11
constexpr int DF_R = 32;                          // rows per double-float update tile

// The route class of a pair's transformation, by the largest entry e of
// E = Z^ - I (real and imaginary parts): 0 for e <= DELTA_E (FP32 delta
// product), 1 for DELTA_E < e <= DF_E (double-float delta product), 2 for the
// others (FP64 product; a NaN counts as large).  Called by every thread of a
// CTA; every thread returns the class.
__device__ __forceinline__ int route_class(const double2 *__restrict__ zp, int kk)
{
    __shared__ int cls;
    if (threadIdx.x == 0) cls = 0;
    __syncthreads();
    int c = 0;
    for (int e = threadIdx.x; e < kk * kk; e += blockDim.x) {
        const int l = e % kk, j = e / kk;
        const double2 z = zp[l + KKMAX * j];
        const double ex = fmax(fabs(z.x - (l == j ? 1.0 : 0.0)), fabs(z.y));
        if (!(ex <= DF_E)) c = 2;
        else if (!(ex <= DELTA_E) && c < 1) c = 1;
    }
    if (c) atomicMax(&cls, c);
    __syncthreads();
    const int r = cls;
    __syncthreads();                               // cls may be reused by a later call
    return r;
}

inline size_t delta64_smem() { return sizeof(double2) * UPD_R * UPD_LD + sizeof(float2) * KKMAX * UPD_LD; }
inline size_t df64_smem() { return sizeof(float2) * 2 * (DF_R + KKMAX) * UPD_LD; }

// The FP32 delta-form update of one 64-row tile (rows row0..) of a pair's
// kk slot columns `slot` of W (ld), E = zp - I (zp: the pair's Z^, ld
// KKMAX), by 256 threads: the FP64 row tile and E in FP32 in shared memory
// (smraw: delta64_smem() bytes), 16 x 16 threads with 4 x 4 outputs each
// (rows ty + 16 i, columns tx + 16 j), four FP32 FMA chains per complex
// product, the sum in FP64.
__device__ __forceinline__ void delta64_tile(double2 *__restrict__ W, long long ld, const int *__restrict__ slot,
                                             int kk, long long row0, const double2 *__restrict__ zp,
                                             unsigned char *smraw)
{
    double2 *xs = reinterpret_cast<double2 *>(smraw);              // [UPD_R][UPD_LD] FP64 rows
    float2 *es = reinterpret_cast<float2 *>(xs + UPD_R * UPD_LD);   // [KKMAX][UPD_LD] E, row l, column j
    __shared__ int cols[KKMAX];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < KKMAX) cols[tid] = tid < kk ? slot[tid] : -1;
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
        if (col >= 0) cp_async<16>(&xs[r * UPD_LD + s], &W[(long long)col * ld + row0 + r]);
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
            W[(long long)col * ld + row0 + r] = make_double2(v.x + (double)pr[i][j], v.y + (double)pi[i][j]);
        }
}

// Double-float arithmetic (a value v carried as hi + lo, hi = fl32(v),
// lo = fl32(v - hi): 48 significant bits; Dekker 1971).
__device__ __forceinline__ void df_split(double2 v, float2 &hi, float2 &lo)
{
    hi = make_float2((float)v.x, (float)v.y);
    lo = make_float2((float)(v.x - (double)hi.x), (float)(v.y - (double)hi.y));
}

// (sh, sl) += a b for double-float a = (ah, al), b = (bh, bl): the leading
// product ah bh split exactly by an FMA, the cross terms ah bl + al bh in
// FP32 (al bl, below 2^-48 |a b|, is dropped), the leading parts added by
// Knuth's error-free two-sum, the low parts added to its error, and the pair
// renormalized by a fast two-sum (the "sloppy" double-float addition):
// 15 FP32 operations.  The _rn intrinsics keep the compiler from fusing the
// sums into FMAs, which would break the error-free transformations.
__device__ __forceinline__ void df_mac(float &sh, float &sl, float ah, float al, float bh, float bl)
{
    const float p = __fmul_rn(ah, bh);
    float q = fmaf(ah, bh, -p);
    q = fmaf(ah, bl, q);
    q = fmaf(al, bh, q);
    const float t = __fadd_rn(sh, p);
    const float z = __fsub_rn(t, sh);
    float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
    e = __fadd_rn(e, __fadd_rn(sl, q));
    sh = __fadd_rn(t, e);
    sl = __fsub_rn(e, __fsub_rn(sh, t));
}

// The delta form X + X E with the product in double-float arithmetic, for
// pairs whose entries of E are at most DF_E = 2^-11.  Per entry the product
// carries at most about 2^-46 |x_l||e_lj| per term (two splittings of 2^-48,
// the dropped term, the FP32 roundings of the small parts) and the
// renormalized sums about 2^-47 of the partial sum per step: at most about
// 2^-41 sum_l |x_l||e_lj| <= 2^-52 sum_l |x_l| in all, about twice the FP64
// product's own bound gamma_kk sum_l |x_l||z_lj| ~ 2^-47 |x_j| for a row of
// comparable entries, where its typical (random-walk) error is also far below
// the FP64 product's.  (In a row whose other entries are far larger than
// x_j the terms x_l e_lj dominate, and the product's 48-bit rounding of them
// exceeds the FP64 product's.)  The FP32 pipe of this GPU is 64 times its FP64 pipe: with
// 60 FP32 operations per complex multiply-add instead of 3 FP64 FMAs (the 3M
// form), a pair costs about a third of its FP64 update.
//
// One 32-row tile (rows row0..) by 256 threads: X and E split into hi and lo
// parts in shared memory (smraw: df64_smem() bytes), 16 x 16 threads with
// 2 x 4 outputs each (rows ty + 16 i, columns tx + 16 j); the sum X + D is
// formed in FP64 from X as read from W.
__device__ __forceinline__ void df64_tile(double2 *__restrict__ W, long long ld, const int *__restrict__ slot,
                                          int kk, long long row0, const double2 *__restrict__ zp,
                                          unsigned char *smraw)
{
    float2 *xh = reinterpret_cast<float2 *>(smraw);   // [DF_R][UPD_LD]
    float2 *xl = xh + DF_R * UPD_LD;
    float2 *eh = xl + DF_R * UPD_LD;                  // [KKMAX][UPD_LD]: row l, column j
    float2 *el = eh + KKMAX * UPD_LD;
    __shared__ int cols[KKMAX];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < KKMAX) cols[tid] = tid < kk ? slot[tid] : -1;
    for (int idx = tid; idx < KKMAX * KKMAX; idx += 256) {
        const int l = idx % KKMAX, j = idx / KKMAX;
        double2 e = make_double2(0.0, 0.0);
        if (l < kk && j < kk) {
            const double2 z = zp[l + KKMAX * j];
            e = make_double2(z.x - (l == j ? 1.0 : 0.0), z.y);
        }
        float2 h, lo;
        df_split(e, h, lo);
        eh[l * UPD_LD + j] = h;
        el[l * UPD_LD + j] = lo;
    }
    __syncthreads();                               // cols
    // the row tile: 8 loads in flight per thread, consecutive threads on
    // consecutive rows of a column
    constexpr int PER = DF_R * KKMAX / 256;
    double2 v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int idx = tid + 256 * k;
        const int r = idx % DF_R, c = idx / DF_R;
        const int col = cols[c];
        v[k] = col >= 0 ? W[(long long)col * ld + row0 + r] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int idx = tid + 256 * k;
        const int r = idx % DF_R, c = idx / DF_R;
        float2 h, lo;
        df_split(v[k], h, lo);
        xh[r * UPD_LD + c] = h;
        xl[r * UPD_LD + c] = lo;
    }
    __syncthreads();
    float rh[2][4], rl[2][4], ih[2][4], il[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { rh[i][j] = 0.0f; rl[i][j] = 0.0f; ih[i][j] = 0.0f; il[i][j] = 0.0f; }
    for (int l = 0; l < kk; ++l) {
        float2 ah[2], al[2], bh[4], bl[4];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            ah[i] = xh[(ty + 16 * i) * UPD_LD + l];
            al[i] = xl[(ty + 16 * i) * UPD_LD + l];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            bh[j] = eh[l * UPD_LD + tx + 16 * j];
            bl[j] = el[l * UPD_LD + tx + 16 * j];
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                // Re += xr er - xi ei,  Im += xr ei + xi er
                df_mac(rh[i][j], rl[i][j], ah[i].x, al[i].x, bh[j].x, bl[j].x);
                df_mac(rh[i][j], rl[i][j], -ah[i].y, -al[i].y, bh[j].y, bl[j].y);
                df_mac(ih[i][j], il[i][j], ah[i].x, al[i].x, bh[j].y, bl[j].y);
                df_mac(ih[i][j], il[i][j], ah[i].y, al[i].y, bh[j].x, bl[j].x);
            }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = ty + 16 * i, c = tx + 16 * j;
            const int col = cols[c];
            if (col < 0) continue;
            double2 *dst = &W[(long long)col * ld + row0 + r];
            const double2 x = *dst;
            // hi + lo is exact in FP64
            *dst = make_double2(x.x + ((double)rh[i][j] + (double)rl[i][j]),
                                x.y + ((double)ih[i][j] + (double)il[i][j]));
        }
}

}  // namespace hz
