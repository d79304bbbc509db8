// hz_update.cuh -- the block update of one outer step (Section 6.4.3).
#pragma once
#include "hz_common.cuh"

namespace hz {

// ---------------------------------------------------------------------------
// (a5) Block update (Section 6.4.3): [X_P X_Q] <- [X_P X_Q] Z^ for the stacked
// rows of F, G and Z' (the paper's three ZGEMMs).  One CTA per (64-row tile,
// pair); pairs whose inner level applied nothing are skipped.
// ---------------------------------------------------------------------------
// The complex128 body: the three-multiplication form of the complex product,
//   x z = (xr zr - xi zi) + i ((xr + xi)(zr + zi) - xr zr - xi zi),
// three real FMA chains per output instead of four (the FP64 pipe bounds this
// kernel).  Its error is bounded entrywise by a small multiple of |x||z|, as
// the usual product's is, but the imaginary part of an output is not exact
// when its column of Z^ is e_j; such columns (untouched by the inner level)
// are copied instead, so that they stay exactly as they were.
__device__ __forceinline__ void update_body_3m(double2 *__restrict__ W, long long ld,
                                               const int *__restrict__ slot, int kk, long long row0,
                                               const double2 *__restrict__ zp, unsigned char *smraw)
{
    double2 *zs = reinterpret_cast<double2 *>(smraw);  // [KKMAX][UPD_LD] row l, col j
    double2 *xs = zs + KKMAX * UPD_LD;                   // [UPD_R][UPD_LD]
    double *zsum = reinterpret_cast<double *>(xs + UPD_R * UPD_LD);  // zr + zi
    double *xsum = zsum + KKMAX * UPD_LD;                // xr + xi
    __shared__ int cols[KKMAX];
    __shared__ int ident[KKMAX];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < KKMAX) cols[tid] = tid < kk ? slot[tid] : -1;
    // Z^ (column-major in zp) and the row tile by asynchronous copies, all in
    // flight at once; then the real sums from shared memory
    for (int idx = tid; idx < KKMAX * KKMAX; idx += 256) {
        const int l = idx % KKMAX, j = idx / KKMAX;
        if (l < kk && j < kk) cp_async<16>(&zs[l * UPD_LD + j], &zp[l + KKMAX * j]);
        else zs[l * UPD_LD + j] = make_double2(0.0, 0.0);
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
    for (int idx = tid; idx < KKMAX * KKMAX; idx += 256) {
        const int l = idx % KKMAX, j = idx / KKMAX;
        const double2 v = zs[l * UPD_LD + j];
        zsum[l * UPD_LD + j] = v.x + v.y;
    }
    for (int idx = tid; idx < UPD_R * KKMAX; idx += 256) {
        const int r = idx % UPD_R, s = idx / UPD_R;
        const double2 v = xs[r * UPD_LD + s];
        xsum[r * UPD_LD + s] = v.x + v.y;
    }
    if (tid < KKMAX) {
        int id = 1;
        for (int l = 0; l < KKMAX; ++l) {
            const double2 v = zs[l * UPD_LD + tid];
            id &= (v.x == (l == tid ? 1.0 : 0.0)) & (v.y == 0.0);
        }
        ident[tid] = id;
    }
    __syncthreads();
    double t1[4][4], t2[4][4], t3[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { t1[i][j] = 0; t2[i][j] = 0; t3[i][j] = 0; }
    for (int l = 0; l < kk; ++l) {
        double2 x[4], z[4];
        double xp[4], zq[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            x[i] = xs[(ty + 16 * i) * UPD_LD + l];
            xp[i] = xsum[(ty + 16 * i) * UPD_LD + l];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            z[j] = zs[l * UPD_LD + tx + 16 * j];
            zq[j] = zsum[l * UPD_LD + tx + 16 * j];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                t1[i][j] = fma(x[i].x, z[j].x, t1[i][j]);
                t2[i][j] = fma(x[i].y, z[j].y, t2[i][j]);
                t3[i][j] = fma(xp[i], zq[j], t3[i][j]);
            }
    }
    double2 v[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = tx + 16 * j;
            v[i][j] = ident[c] ? xs[(ty + 16 * i) * UPD_LD + c]
                               : make_double2(t1[i][j] - t2[i][j], (t3[i][j] - t1[i][j]) - t2[i][j]);
        }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) xs[(ty + 16 * i) * UPD_LD + tx + 16 * j] = v[i][j];
    __syncthreads();
    for (int idx = tid; idx < UPD_R * KKMAX; idx += 256) {
        const int r = idx % UPD_R, s = idx / UPD_R;
        const int col = cols[s];
        if (col >= 0) W[(long long)col * ld + row0 + r] = xs[r * UPD_LD + s];
    }
}

// The complex64 body (four real FMA chains per output; the FP32 pipe does
// not bound it), in the delta form X + X (Z^ - I): the rounding error of the
// product is then relative to |X||Z^ - I| instead of |X||Z^|, so that the
// small rotations of a converging sweep add little rounding noise, and a
// column whose Z^ column is e_j stays exactly as it was.
template <typename T, typename TZ>
__device__ __forceinline__ void update_body_4m(typename cplx<T>::t *__restrict__ W, long long ld,
                                               const int *__restrict__ slot, int kk, long long row0,
                                               const typename cplx<TZ>::t *__restrict__ zp,
                                               unsigned char *smraw)
{
    using T2 = typename cplx<T>::t;
    // rows padded to UPD_LD: the transposed stores of Z^ and of the row tile
    // (consecutive threads on consecutive rows) then hit distinct banks
    T2 *zs = reinterpret_cast<T2 *>(smraw);          // [KKMAX][UPD_LD] row l, col j
    T2 *xs = zs + KKMAX * UPD_LD;                     // [UPD_R][UPD_LD]
    static_assert(std::is_same<T, TZ>::value, "Z^ in the sweep's precision");
    __shared__ int cols[KKMAX];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < KKMAX) cols[tid] = tid < kk ? slot[tid] : -1;
    // Z^ (column-major in zp) and the row tile by asynchronous copies, all in
    // flight at once
    T2 zero;
    zero.x = 0;
    zero.y = 0;
    for (int idx = tid; idx < KKMAX * KKMAX; idx += 256) {
        const int l = idx % KKMAX, j = idx / KKMAX;
        if (l < kk && j < kk) cp_async<sizeof(T2)>(&zs[l * UPD_LD + j], &zp[l + KKMAX * j]);
        else zs[l * UPD_LD + j] = zero;
    }
    __syncthreads();                               // cols
    for (int idx = tid; idx < UPD_R * KKMAX; idx += 256) {
        const int r = idx % UPD_R, s = idx / UPD_R;
        const int col = cols[s];
        if (col >= 0) cp_async<sizeof(T2)>(&xs[r * UPD_LD + s], &W[(long long)col * ld + row0 + r]);
        else xs[r * UPD_LD + s] = zero;
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    if (tid < kk) zs[tid * UPD_LD + tid].x -= (T)1;   // E = Z^ - I (exact near 1)
    __syncthreads();
    T accr[4][4], acci[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { accr[i][j] = 0; acci[i][j] = 0; }
    for (int l = 0; l < kk; ++l) {
        T2 x[4], z[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = xs[(ty + 16 * i) * UPD_LD + l];
#pragma unroll
        for (int j = 0; j < 4; ++j) z[j] = zs[l * UPD_LD + tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                accr[i][j] = fma(x[i].x, z[j].x, accr[i][j]);
                accr[i][j] = fma(-x[i].y, z[j].y, accr[i][j]);
                acci[i][j] = fma(x[i].x, z[j].y, acci[i][j]);
                acci[i][j] = fma(x[i].y, z[j].x, acci[i][j]);
            }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            T2 &o = xs[(ty + 16 * i) * UPD_LD + tx + 16 * j];   // read, then written, by this thread only
            T2 v;
            v.x = o.x + accr[i][j];
            v.y = o.y + acci[i][j];
            o = v;
        }
    __syncthreads();
    for (int idx = tid; idx < UPD_R * KKMAX; idx += 256) {
        const int r = idx % UPD_R, s = idx / UPD_R;
        const int col = cols[s];
        if (col >= 0) W[(long long)col * ld + row0 + r] = xs[r * UPD_LD + s];
    }
}

// The body, for one (pair, 64-row tile): rows [row0, row0 + 64) of W (ld)
// in the pair's kk slot columns `slot`, times its Z^ `zp` (ld KKMAX).
template <typename T, typename TZ>
__device__ __forceinline__ void update_body(typename cplx<T>::t *__restrict__ W, long long ld,
                                            const int *__restrict__ slot, int kk, long long row0,
                                            const typename cplx<TZ>::t *__restrict__ zp,
                                            unsigned char *smraw)
{
    if constexpr (std::is_same<T, double>::value && std::is_same<TZ, double>::value)
        update_body_3m(W, ld, slot, kk, row0, zp, smraw);
    else
        update_body_4m<T, TZ>(W, ld, slot, kk, row0, zp, smraw);
}

// One outer step of one pencil: CTA = (64-row tile, pair); pairs whose inner
// level applied nothing are skipped.
template <typename T, typename TZ>
__global__ void __launch_bounds__(256)
update_kernel(typename cplx<T>::t *__restrict__ W, StepArgs a,
              const typename cplx<TZ>::t *__restrict__ zhat, const int *__restrict__ pair_flag)
{
    extern __shared__ unsigned char smraw[];
    const int pair = blockIdx.y;
    if (!pair_flag[pair]) return;
    update_body<T, TZ>(W, a.ld, a.slotcol + pair * a.kk, a.kk, (long long)blockIdx.x * UPD_R,
                       zhat + (long long)pair * KKMAX * KKMAX, smraw);
}

}  // namespace hz
