// hz_inner.cuh -- the inner level on the block pivots of one outer step (Section 6.4.2).
#pragma once
#include "hz_common.cuh"

namespace hz {

// ---------------------------------------------------------------------------
// (a3, a4) The inner level on one block pivot (Section 6.4.2): sum the Gram
// partials, then run `inner_sweeps` sweeps of the pointwise method on the
// pair (H^, S^) two-sidedly (the block pivots are transformed by
// congruence, H^ <- Z'^* H^ Z', S^ <- Z'^* S^ Z'), accumulating Z^ <- Z^ Z'.
// All kk/2 pivots of an inner step are disjoint and are transformed at once:
// with Z_all the block-diagonal product of the step's 2x2 transformations,
// each 2x2 block (I, J) of H^ becomes Z_I^* H^_IJ Z_J; only I <= J is
// computed, the mirror block is its conjugate transpose.
// One CTA (1024 threads) per block pivot; H^, S^, Z^ live in shared memory.
// ---------------------------------------------------------------------------
template <typename TP>   // type of the Gram partials (double or float)
__global__ void __launch_bounds__(1024)
inner_kernel(const typename cplx<TP>::t *__restrict__ partial, const int *__restrict__ slotcol,
             InnerArgs a, double2 *__restrict__ zhat, int *__restrict__ pair_flag,
             unsigned long long *__restrict__ counters, int *__restrict__ err)
{
    extern __shared__ double2 smem[];
    double2 *H = smem;                       // [KKMAX * KKMAX], column-major
    double2 *S = H + KKMAX * KKMAX;
    double2 *Z = S + KKMAX * KKMAX;
    __shared__ double zp[KKMAX / 2][8];      // the step's 2x2 transformations
    __shared__ int tr[KKMAX / 2];            // pivot transformed?
    __shared__ int pslot[KKMAX];             // slots of pivot l: 2l, 2l+1
    __shared__ int valid[KKMAX];
    __shared__ int s_all, s_big, s_err;
    const int pair = blockIdx.x;
    const int tid = threadIdx.x;
    const int kk = a.kk, np = kk / 2;
    if (tid < KKMAX) valid[tid] = tid < kk ? (slotcol[pair * kk + tid] >= 0) : 0;
    if (tid == 0) { s_all = 0; s_big = 0; s_err = 0; }
    __syncthreads();

    // sum the partial Grams in chunk order (deterministic)
    const typename cplx<TP>::t *pp = partial + (long long)pair * a.cpp * (KKMAX * KKMAX);
    for (int idx = tid; idx < kk * kk; idx += blockDim.x) {
        const int i = idx % kk, j = idx / kk;
        const int e = i + KKMAX * j;
        double hr = 0, hi = 0, sr = 0, si = 0;
        for (int c = 0; c < a.chunks_h; ++c) {
            hr += (double)pp[(long long)c * KKMAX * KKMAX + e].x;
            hi += (double)pp[(long long)c * KKMAX * KKMAX + e].y;
        }
        for (int c = a.chunks_h; c < a.cpp; ++c) {
            sr += (double)pp[(long long)c * KKMAX * KKMAX + e].x;
            si += (double)pp[(long long)c * KKMAX * KKMAX + e].y;
        }
        if (i == j) {          // Hermitian: real diagonal; bordered slot: S = 1
            hi = 0; si = 0;
            if (!valid[i]) { sr = 1.0; hr = 0.0; }
        }
        H[i + kk * j] = make_double2(hr, hi);
        S[i + kk * j] = make_double2(sr, si);
        Z[i + kk * j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();

    int my_all = 0, my_big = 0;
    __shared__ int s_sweep;
    for (int isw = 0; isw < a.inner_sweeps; ++isw) {
        if (tid == 0) s_sweep = 0;
        __syncthreads();
        for (int r = 0; r < kk - 1; ++r) {
            // pivots of the step, spread over four warps (one per SM sub-partition)
            const int warp = tid >> 5, lane = tid & 31;
            if (warp < 4) {
                int step_all = 0;
                for (int l = lane * 4 + warp; l < np; l += 128) {
                    int pa, pb;
                    rr_pair(kk, r, l, &pa, &pb);
                    pslot[2 * l] = pa;
                    pslot[2 * l + 1] = pb;
                    int rc = PIV_NONE, big = 0;
                    if (valid[pa] && valid[pb]) {
                        const double2 hab = H[pa + kk * pb], sab = S[pa + kk * pb];
                        rc = pivot2x2(H[pa + kk * pa].x, H[pb + kk * pb].x, hab.x, hab.y,
                                      S[pa + kk * pa].x, S[pb + kk * pb].x, sab.x, sab.y,
                                      a.tol, a.crit_mode, zp[l], &big);
                    }
                    if (rc < 0) {
                        atomicOr(&s_err, rc == PIV_ERR_RANK ? DEVERR_RANK : DEVERR_NONFINITE);
                        rc = PIV_NONE;
                    }
                    tr[l] = rc == PIV_TRANSFORM;
                    if (rc == PIV_TRANSFORM) { my_all += 1; my_big += big; step_all += 1; }
                }
                if (step_all) atomicAdd(&s_sweep, step_all);
            }
            __syncthreads();
            // two-sided update of H^ and S^ by 2x2 blocks (I <= J), and Z^ <- Z^ Z'
            const int nblk = np * (np + 1) / 2;
            const int nitems = 2 * nblk + kk * np;
            for (int it = tid; it < nitems; it += blockDim.x) {
                if (it < 2 * nblk) {
                    const int mat = it >= nblk;
                    int b = it - mat * nblk;
                    // decode b -> (I, J), I <= J, row-major upper triangle
                    int I = 0;
                    while (b >= np - I) { b -= np - I; ++I; }
                    const int Jb = I + b;
                    if (!tr[I] && !tr[Jb]) continue;
                    double2 *A = mat ? S : H;
                    const int aI = pslot[2 * I], bI = pslot[2 * I + 1];
                    const int aJ = pslot[2 * Jb], bJ = pslot[2 * Jb + 1];
                    double2 x00 = A[aI + kk * aJ], x01 = A[aI + kk * bJ];
                    double2 x10 = A[bI + kk * aJ], x11 = A[bI + kk * bJ];
                    if (tr[Jb]) {            // right: [x] <- [x] Z_J
                        const double *z = zp[Jb];
                        double2 y00, y01, y10, y11;
                        y00.x = x00.x * z[0] - x00.y * z[1] + x01.x * z[4] - x01.y * z[5];
                        y00.y = x00.x * z[1] + x00.y * z[0] + x01.x * z[5] + x01.y * z[4];
                        y01.x = x00.x * z[2] - x00.y * z[3] + x01.x * z[6] - x01.y * z[7];
                        y01.y = x00.x * z[3] + x00.y * z[2] + x01.x * z[7] + x01.y * z[6];
                        y10.x = x10.x * z[0] - x10.y * z[1] + x11.x * z[4] - x11.y * z[5];
                        y10.y = x10.x * z[1] + x10.y * z[0] + x11.x * z[5] + x11.y * z[4];
                        y11.x = x10.x * z[2] - x10.y * z[3] + x11.x * z[6] - x11.y * z[7];
                        y11.y = x10.x * z[3] + x10.y * z[2] + x11.x * z[7] + x11.y * z[6];
                        x00 = y00; x01 = y01; x10 = y10; x11 = y11;
                    }
                    if (tr[I]) {             // left: [x] <- Z_I^* [x]
                        const double *z = zp[I];
                        // Z^* = [conj z11, conj z21; conj z12, conj z22]
                        double2 y00, y01, y10, y11;
                        y00.x = z[0] * x00.x + z[1] * x00.y + z[4] * x10.x + z[5] * x10.y;
                        y00.y = z[0] * x00.y - z[1] * x00.x + z[4] * x10.y - z[5] * x10.x;
                        y01.x = z[0] * x01.x + z[1] * x01.y + z[4] * x11.x + z[5] * x11.y;
                        y01.y = z[0] * x01.y - z[1] * x01.x + z[4] * x11.y - z[5] * x11.x;
                        y10.x = z[2] * x00.x + z[3] * x00.y + z[6] * x10.x + z[7] * x10.y;
                        y10.y = z[2] * x00.y - z[3] * x00.x + z[6] * x10.y - z[7] * x10.x;
                        y11.x = z[2] * x01.x + z[3] * x01.y + z[6] * x11.x + z[7] * x11.y;
                        y11.y = z[2] * x01.y - z[3] * x01.x + z[6] * x11.y - z[7] * x11.x;
                        x00 = y00; x01 = y01; x10 = y10; x11 = y11;
                    }
                    if (I == Jb) { x00.y = 0.0; x11.y = 0.0; x10 = make_double2(x01.x, -x01.y); }
                    A[aI + kk * aJ] = x00; A[aI + kk * bJ] = x01;
                    A[bI + kk * aJ] = x10; A[bI + kk * bJ] = x11;
                    if (I != Jb) {
                        A[aJ + kk * aI] = make_double2(x00.x, -x00.y);
                        A[bJ + kk * aI] = make_double2(x01.x, -x01.y);
                        A[aJ + kk * bI] = make_double2(x10.x, -x10.y);
                        A[bJ + kk * bI] = make_double2(x11.x, -x11.y);
                    }
                } else {
                    const int q = it - 2 * nblk;
                    const int row = q % kk, l = q / kk;
                    if (!tr[l]) continue;
                    const double *z = zp[l];
                    const int pa = pslot[2 * l], pb = pslot[2 * l + 1];
                    const double2 u = Z[row + kk * pa], w = Z[row + kk * pb];
                    double2 ya, yb;
                    ya.x = u.x * z[0] - u.y * z[1] + w.x * z[4] - w.y * z[5];
                    ya.y = u.x * z[1] + u.y * z[0] + w.x * z[5] + w.y * z[4];
                    yb.x = u.x * z[2] - u.y * z[3] + w.x * z[6] - w.y * z[7];
                    yb.y = u.x * z[3] + u.y * z[2] + w.x * z[7] + w.y * z[6];
                    Z[row + kk * pa] = ya;
                    Z[row + kk * pb] = yb;
                }
            }
            __syncthreads();
        }
        // FB: stop after an inner sweep without any transformation
        // (Section 6.1.7: the inner levels count all transformations)
        const int swept = s_sweep;
        __syncthreads();
        if (swept == 0) break;
    }
    if (my_all) atomicAdd(&s_all, my_all);
    if (my_big) atomicAdd(&s_big, my_big);
    __syncthreads();
    // Zhat[pair] (kk x kk, column-major, ld KKMAX)
    double2 *zo = zhat + (long long)pair * KKMAX * KKMAX;
    for (int idx = tid; idx < kk * kk; idx += blockDim.x) {
        const int i = idx % kk, j = idx / kk;
        zo[i + KKMAX * j] = Z[i + kk * j];
    }
    if (tid == 0) {
        pair_flag[pair] = s_all > 0;
        if (s_all) atomicAdd(&counters[0], (unsigned long long)s_all);
        if (s_big) atomicAdd(&counters[1], (unsigned long long)s_big);
        if (s_err) atomicOr(err, s_err);
    }
}

}  // namespace hz
