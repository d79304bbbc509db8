// hz_inner.cuh -- the inner level on the block pivots of one outer step (Section 6.4.2).
#pragma once
#include <cooperative_groups.h>

#include "hz_common.cuh"

namespace hz {

// Synchronization and replicated stores of the inner level.  With CL = 1 the
// block pivot lives in one CTA; with CL > 1 a thread-block cluster of CL CTAs
// (on CL SMs) keeps one copy of (H^, S^, Z^) in each CTA's shared memory, every
// CTA transforms 1/CL of the entries and stores each result into all CL copies
// through distributed shared memory.
template <int CL>
struct InnerSync {
    __device__ __forceinline__ static int rank()
    {
        if constexpr (CL == 1) return 0;
        else return (int)cooperative_groups::this_cluster().block_rank();
    }
    __device__ __forceinline__ static void sync()
    {
        if constexpr (CL == 1) __syncthreads();
        else cooperative_groups::this_cluster().sync();
    }
    template <typename T>
    __device__ __forceinline__ static T *remote(T *local, int r)
    {
        if constexpr (CL == 1) return local;
        else return cooperative_groups::this_cluster().map_shared_rank(local, (unsigned)r);
    }
};

// Complex helpers for the shared-memory block pivots (T = double or float).
template <typename T2, typename T>
__device__ __forceinline__ T2 c_make(T x, T y)
{
    T2 r;
    r.x = x;
    r.y = y;
    return r;
}

// [x0 x1] <- [x0 x1] Z, Z = {z11, z12; z21, z22} given as z[0..7] (re, im).
// z11 and z22 are real (z[1] = z[7] = 0): eq. 6.9 with the phases moved off
// the diagonal (Section 6.1.5), scaled by the real D0 of Section 6.1.1; the
// terms with z[1] and z[7] are left out (12 real products instead of 16).
template <typename T2, typename T>
__device__ __forceinline__ void c_right(T2 &x0, T2 &x1, const T *z)
{
    const T2 a = x0, b = x1;
    x0.x = a.x * z[0] + b.x * z[4] - b.y * z[5];
    x0.y = a.y * z[0] + b.x * z[5] + b.y * z[4];
    x1.x = a.x * z[2] - a.y * z[3] + b.x * z[6];
    x1.y = a.x * z[3] + a.y * z[2] + b.y * z[6];
}

// [x0; x1] <- Z^* [x0; x1] (Z^* = {conj z11, conj z21; conj z12, conj z22}),
// z11 and z22 real as above.
template <typename T2, typename T>
__device__ __forceinline__ void c_left(T2 &x0, T2 &x1, const T *z)
{
    const T2 a = x0, b = x1;
    x0.x = z[0] * a.x + z[4] * b.x + z[5] * b.y;
    x0.y = z[0] * a.y + z[4] * b.y - z[5] * b.x;
    x1.x = z[2] * a.x + z[3] * a.y + z[6] * b.x;
    x1.y = z[2] * a.y - z[3] * a.x + z[6] * b.y;
}

// ---------------------------------------------------------------------------
// (a3, a4) The inner level on one block pivot (Section 6.4.2): sum the Gram
// partials, then run `inner_sweeps` sweeps of the pointwise method on the
// pair (H^, S^) two-sidedly (the block pivots are transformed by
// congruence, H^ <- Z'^* H^ Z', S^ <- Z'^* S^ Z'), accumulating Z^ <- Z^ Z'.
// All kk/2 pivots of an inner step are disjoint and are transformed at once:
// with Z_all the block-diagonal product of the step's 2x2 transformations,
// each 2x2 block (I, J) of H^ becomes Z_I^* H^_IJ Z_J; only I <= J is
// computed, the mirror block is its conjugate transpose.
//
// TP is the type of the Gram partials, TU the type in which the block
// pivots are kept and transformed (double for the FP64 sweeps, float for the
// complex64 preconditioning sweeps).  The 2x2 parameters (eq. 6.5-6.12) are
// computed in FP64 from the pivot entries: correctly rounded step by step in
// the FP64 sweeps (pivot2x2), with shared reciprocals in the complex64 sweeps
// (pivot2x2_fast_x2, two lanes per pivot); with a.param32 the complex64 sweeps compute them in FP32
// instead.  The complex64 sweeps count "big" by the FP64 test (sin(phi) or
// sin(psi) >= 2^-27), which keeps the stagnation test of the mixed
// schedule's refinement rounds as with exact FP64 parameters.
//
// The Gram kernel writes the entries on and above the diagonal; an entry
// below it is the conjugate of its mirror (the block pivots are Hermitian).
// One CTA (1024 threads) per block pivot; H^, S^, Z^ live in shared memory.
// ---------------------------------------------------------------------------
// The body, for one block pivot: pp = its cpp Gram partials, slot = its kk
// slot columns, zo = its Z^ (in the sweep's precision TU, ld KKMAX), flag =
// its "transformed" flag.
template <typename TP, typename TU, int CL = 1>
__device__ __forceinline__ void inner_body(const typename cplx<TP>::t *__restrict__ pp,
                                           const int *__restrict__ slot, InnerArgs a,
                                           typename cplx<TU>::t *__restrict__ zo,
                                           int *__restrict__ flag,
                                           unsigned long long *__restrict__ counters,
                                           int *__restrict__ err, unsigned char *smraw_inner)
{
    using U2 = typename cplx<TU>::t;
    using X = InnerSync<CL>;
    // column-major with columns of INNER_LD = KKMAX + 1 entries, so that the
    // entries of a row (stride one column) fall in different banks
    U2 *H = reinterpret_cast<U2 *>(smraw_inner);
    U2 *S = H + KKMAX * INNER_LD;
    U2 *Z = S + KKMAX * INNER_LD;
    const int crank = X::rank();
    // the CL copies of the block pivot (H^, S^, Z^ are consecutive)
    U2 *copies[CL];
#pragma unroll
    for (int r = 0; r < CL; ++r) copies[r] = X::remote(H, r);
    // A[off] = v in every copy; off is an offset from H
    auto put = [&](int off, U2 v) {
#pragma unroll
        for (int r = 0; r < CL; ++r) copies[r][off] = v;
    };
    const int HS = KKMAX * INNER_LD;            // offset of S from H (Z: 2 HS)
    __shared__ TU zu[KKMAX / 2][8];          // the step's 2x2 transformations
    __shared__ int tr[KKMAX / 2];            // pivot transformed?
    __shared__ int pslot[KKMAX];             // slots of pivot l: 2l, 2l+1
    __shared__ int valid[KKMAX];
    __shared__ int s_all, s_big, s_err, s_sweep;
    const int tid = threadIdx.x;
    const int kk = a.kk, np = kk / 2;
    if (tid < KKMAX) valid[tid] = tid < kk ? (slot[tid] >= 0) : 0;
    if (tid == 0) { s_all = 0; s_big = 0; s_err = 0; }
    // every CTA of the cluster has started before any shared-memory copy is
    // written from another CTA
    X::sync();

    // sum the partial Grams in chunk order (deterministic, in FP64); each
    // CTA of a cluster sums 1/CL of the entries and stores them in all copies
    for (int idx = tid * CL + crank; idx < kk * kk; idx += CL * blockDim.x) {
        const int i = idx % kk, j = idx / kk;
        const bool mirror = i > j;                  // below the diagonal: conj of (j, i)
        const int e = mirror ? j + KKMAX * i : i + KKMAX * j;
        double hr = 0, hi = 0, sr = 0, si = 0;
        for (int c = 0; c < a.chunks_h; ++c) {
            hr += (double)pp[(long long)c * KKMAX * KKMAX + e].x;
            hi += (double)pp[(long long)c * KKMAX * KKMAX + e].y;
        }
        for (int c = a.chunks_h; c < a.cpp; ++c) {
            sr += (double)pp[(long long)c * KKMAX * KKMAX + e].x;
            si += (double)pp[(long long)c * KKMAX * KKMAX + e].y;
        }
        if (mirror) { hi = -hi; si = -si; }
        if (i == j) {          // Hermitian: real diagonal; bordered slot: S = 1
            hi = 0; si = 0;
            if (!valid[i]) { sr = 1.0; hr = 0.0; }
        }
        put(i + INNER_LD * j, c_make<U2, TU>((TU)hr, (TU)hi));
        put(HS + i + INNER_LD * j, c_make<U2, TU>((TU)sr, (TU)si));
        put(2 * HS + i + INNER_LD * j, c_make<U2, TU>((TU)(i == j ? 1 : 0), (TU)0));
    }
    X::sync();

    int my_all = 0, my_big = 0;
    for (int isw = 0; isw < a.inner_sweeps; ++isw) {
        if (tid == 0) s_sweep = 0;
        __syncthreads();
        for (int r = 0; r < kk - 1; ++r) {
            // pivots of the step, spread over four warps (one per SM sub-partition);
            // FP64 parameters take two lanes per pivot (pivot2x2_x2 in the FP64
            // sweeps, pivot2x2_fast_x2 in the complex64 ones), FP32 ones one
            const int warp = tid >> 5, lane = tid & 31;
            const bool paired = !(sizeof(TU) == sizeof(float) && a.param32);
            const int pk = paired ? (lane & 1) : 0;
            const unsigned pmask = 3u << (lane & 30);
            if (warp < 4) {
                int step_all = 0;
                for (int l = (paired ? lane >> 1 : lane) * 4 + warp; l < np; l += paired ? 64 : 128) {
                    int pa, pb;
                    rr_pair(kk, r, l, &pa, &pb);
                    if (pk == 0) {
                        pslot[2 * l] = pa;
                        pslot[2 * l + 1] = pb;
                    }
                    int rc = PIV_NONE, big = 0;
                    TU zl[8];
                    double zrow[4];                     // paired: this lane's row of Z'
                    if (valid[pa] && valid[pb]) {
                        const U2 hab = H[pa + INNER_LD * pb], sab = S[pa + INNER_LD * pb];
                        if (paired) {
                            if (sizeof(TU) == sizeof(double))
                                rc = pivot2x2_x2<TU>(pk, pmask, H[pa + INNER_LD * pa].x, H[pb + INNER_LD * pb].x,
                                                     hab.x, hab.y, S[pa + INNER_LD * pa].x,
                                                     S[pb + INNER_LD * pb].x, sab.x, sab.y, a.tol, a.crit_mode,
                                                     zrow, &big);
                            else
                                rc = pivot2x2_fast_x2<TU>(pk, pmask, H[pa + INNER_LD * pa].x,
                                                          H[pb + INNER_LD * pb].x, hab.x, hab.y,
                                                          S[pa + INNER_LD * pa].x, S[pb + INNER_LD * pb].x,
                                                          sab.x, sab.y, a.tol, a.crit_mode, zrow, &big);
                        } else {                        // complex64 sweeps, FP32 parameters
                            rc = pivot2x2<TU>(H[pa + INNER_LD * pa].x, H[pb + INNER_LD * pb].x, hab.x,
                                              hab.y, S[pa + INNER_LD * pa].x, S[pb + INNER_LD * pb].x,
                                              sab.x, sab.y, (TU)a.tol, a.crit_mode, zl, &big);
                        }
                    }
                    // complex64 preconditioning sweeps leave a pivot that looks
                    // dependent at their rounding level alone; the FP64 sweeps
                    // that follow decide about rank deficiency
                    if (rc == PIV_ERR_RANK && sizeof(TU) == sizeof(float)) rc = PIV_NONE;
                    if (paired && rc == PIV_TRANSFORM) {   // each lane stores its row of Z'
#pragma unroll
                        for (int q = 0; q < 4; ++q) zu[l][4 * pk + q] = (TU)zrow[q];
                    }
                    if (pk != 0) continue;                  // the pair's second lane
                    if (rc < 0) {
                        atomicOr(&s_err, rc == PIV_ERR_RANK ? DEVERR_RANK : DEVERR_NONFINITE);
                        rc = PIV_NONE;
                    }
                    tr[l] = rc == PIV_TRANSFORM;
                    if (rc == PIV_TRANSFORM) {
                        if (!paired) {
#pragma unroll
                            for (int q = 0; q < 8; ++q) zu[l][q] = zl[q];
                        }
                        my_all += 1;
                        my_big += big;
                        step_all += 1;
                    }
                }
                if (step_all) atomicAdd(&s_sweep, step_all);
            }
            // every copy must be read by phase A before any CTA overwrites it
            X::sync();
            // two-sided update of H^ and S^ by 2x2 blocks (I <= J), and Z^ <- Z^ Z';
            // each item owns the entries it writes, so items of different CTAs
            // never touch the same entry; items are dealt round-robin to the
            // CTAs of a cluster
            const int nblk = np * (np + 1) / 2;
            const int nitems = 2 * nblk + kk * np;
            for (int it = tid * CL + crank; it < nitems; it += CL * blockDim.x) {
                if (it < 2 * nblk) {
                    const int mat = it >= nblk;
                    int b = it - mat * nblk;
                    // decode b -> (I, J), I <= J, row-major upper triangle
                    int I = 0;
                    while (b >= np - I) { b -= np - I; ++I; }
                    const int Jb = I + b;
                    if (!tr[I] && !tr[Jb]) continue;
                    U2 *A = mat ? S : H;
                    const int ab = mat ? HS : 0;
                    const int aI = pslot[2 * I], bI = pslot[2 * I + 1];
                    const int aJ = pslot[2 * Jb], bJ = pslot[2 * Jb + 1];
                    U2 x00 = A[aI + INNER_LD * aJ], x01 = A[aI + INNER_LD * bJ];
                    U2 x10 = A[bI + INNER_LD * aJ], x11 = A[bI + INNER_LD * bJ];
                    if (tr[Jb]) {            // right: rows of the block times Z_J
                        c_right<U2, TU>(x00, x01, zu[Jb]);
                        c_right<U2, TU>(x10, x11, zu[Jb]);
                    }
                    if (tr[I]) {             // left: Z_I^* times columns of the block
                        c_left<U2, TU>(x00, x10, zu[I]);
                        c_left<U2, TU>(x01, x11, zu[I]);
                    }
                    if (I == Jb) {
                        x00.y = 0;
                        x11.y = 0;
                        x10 = c_make<U2, TU>(x01.x, -x01.y);
                    }
                    put(ab + aI + INNER_LD * aJ, x00); put(ab + aI + INNER_LD * bJ, x01);
                    put(ab + bI + INNER_LD * aJ, x10); put(ab + bI + INNER_LD * bJ, x11);
                    if (I != Jb) {
                        put(ab + aJ + INNER_LD * aI, c_make<U2, TU>(x00.x, -x00.y));
                        put(ab + bJ + INNER_LD * aI, c_make<U2, TU>(x01.x, -x01.y));
                        put(ab + aJ + INNER_LD * bI, c_make<U2, TU>(x10.x, -x10.y));
                        put(ab + bJ + INNER_LD * bI, c_make<U2, TU>(x11.x, -x11.y));
                    }
                } else {
                    const int q = it - 2 * nblk;
                    const int row = q % kk, l = q / kk;
                    if (!tr[l]) continue;
                    const int pa = pslot[2 * l], pb = pslot[2 * l + 1];
                    U2 u = Z[row + INNER_LD * pa], w = Z[row + INNER_LD * pb];
                    c_right<U2, TU>(u, w, zu[l]);
                    put(2 * HS + row + INNER_LD * pa, u);
                    put(2 * HS + row + INNER_LD * pb, w);
                }
            }
            X::sync();
        }
        // FB: stop after an inner sweep without any transformation
        // (Section 6.1.7, the inner levels count all transformations)
        const int swept = s_sweep;
        __syncthreads();
        if (swept == 0) break;
    }
    if (my_all) atomicAdd(&s_all, my_all);
    if (my_big) atomicAdd(&s_big, my_big);
    __syncthreads();
    // Z^ (kk x kk, column-major, ld KKMAX), FP64; the copies are identical,
    // each CTA of a cluster writes 1/CL of the entries
    for (int idx = tid * CL + crank; idx < kk * kk; idx += CL * blockDim.x) {
        const int i = idx % kk, j = idx / kk;
        const U2 v = Z[i + INNER_LD * j];
        zo[i + KKMAX * j] = v;
    }
    if (tid == 0 && crank == 0) {
        *flag = s_all > 0;
        if (s_all) atomicAdd(&counters[0], (unsigned long long)s_all);
        if (s_big) atomicAdd(&counters[1], (unsigned long long)s_big);
        if (s_err) atomicOr(err, s_err);
    }
}

// One outer step of one pencil: CTA = block pivot.
template <typename TP, typename TU>
__global__ void __launch_bounds__(1024)
inner_kernel(const typename cplx<TP>::t *__restrict__ partial, const int *__restrict__ slotcol,
             InnerArgs a, typename cplx<TU>::t *__restrict__ zhat, int *__restrict__ pair_flag,
             unsigned long long *__restrict__ counters, int *__restrict__ err)
{
    extern __shared__ unsigned char smraw_inner[];
    const int pair = blockIdx.x;
    inner_body<TP, TU>(partial + (long long)pair * a.cpp * (KKMAX * KKMAX), slotcol + pair * a.kk, a,
                       zhat + (long long)pair * KKMAX * KKMAX, pair_flag + pair, counters, err,
                       smraw_inner);
}

// The same with a cluster of CL CTAs per block pivot (grid = npairs * CL).
template <typename TP, typename TU, int CL>
__global__ void __launch_bounds__(1024)
inner_cluster_kernel(const typename cplx<TP>::t *__restrict__ partial, const int *__restrict__ slotcol,
                     InnerArgs a, typename cplx<TU>::t *__restrict__ zhat, int *__restrict__ pair_flag,
                     unsigned long long *__restrict__ counters, int *__restrict__ err)
{
    extern __shared__ unsigned char smraw_inner[];
    const int pair = blockIdx.x / CL;
    inner_body<TP, TU, CL>(partial + (long long)pair * a.cpp * (KKMAX * KKMAX), slotcol + pair * a.kk,
                           a, zhat + (long long)pair * KKMAX * KKMAX, pair_flag + pair, counters, err,
                           smraw_inner);
}

}  // namespace hz
