// hz_gram.cuh -- the block-pivot Gram kernel of one outer step (Section 6.4.2).
#pragma once
#include "hz_common.cuh"

namespace hz {

// ---------------------------------------------------------------------------
// (a2) Block pivots, eq. 6.1 on block column pairs (Section 6.4.2):
//   H^ = F_PQ^* J F_PQ (rows [0, m_pad)), S^ = G_PQ^* G_PQ (rows of G).
// One CTA per (pair, row chunk); the CTA writes the partial Gram of its rows;
// the inner kernel sums the partials in a fixed order.
//
// The block pivots are Hermitian, so only the entries on and above the
// diagonal are computed.  The complex64 body takes the 16 x 16 tiles on and
// above the diagonal (10 of 16 for kk = 64, 3 of 4 for kk = 32), 16 threads
// per tile, each a 4 x 4 set of complex outputs (rows 16 ti + ly + 4i,
// columns 16 tj + lx + 4j), skipping in the diagonal tiles the 4 x 4 blocks
// below the diagonal; the complex128 body deals the same entries out in equal
// FP64 shares per warp (below).  J enters as a sign flip of the conjugated
// factor (an integer xor on the sign bits).
// ---------------------------------------------------------------------------
// The tile of one thread: the nt diagonal tiles first (so that warps hold two
// diagonal tiles or two off-diagonal ones), then the tiles above the diagonal
// in row-major order.  Returns false for the threads without a tile.
__device__ __forceinline__ bool gram_tile(int kk, int tile, int &ti, int &tj)
{
    const int nt = (kk + 15) >> 4;
    const int ntiles = nt * (nt + 1) / 2;
    ti = 0;
    tj = 0;
    if (tile >= ntiles) return false;
    if (tile < nt) {
        ti = tj = tile;
    } else {
        int rem = tile - nt;
        while (rem >= nt - 1 - ti) { rem -= nt - 1 - ti; ++ti; }
        tj = ti + 1 + rem;
    }
    return true;
}

// The complex128 body: the three-multiplication form of conj(x) y,
//   Re = xr yr + xi yi,  Im = (xr - xi)(yr + yi) - xr yr + xi yi,
// three real FMA chains per entry instead of four (the FP64 pipe bounds this
// kernel); xr - xi and xr + xi are formed once per staged element.  The error
// of an entry stays bounded by a small multiple of sum |x||y|, as with the
// usual product.
//
// The FP64 pipe of a sub-partition spends the same time on a warp instruction
// whatever its active lanes, so the work is dealt in equal shares per warp:
// gram_threads_c128(kk) threads, one warp per two of the off-diagonal 16 x 16
// tiles (4 x 4 strided entries per thread, as in the complex64 body), and one
// warp for the entries strictly above the diagonal of the nt diagonal tiles:
// 8 lanes per tile, lane rho holding row rho (columns rho+1..15) and row
// 14 - rho (columns 15-rho..15), 16 entries (row 7 alone: 8).  The real
// diagonal sum J |x|^2 is split over every thread: thread t adds the squares
// of the real (t even) or imaginary (t odd) parts of column t / 2.
__device__ __forceinline__ void gram_body_3m(const double2 *__restrict__ W, long long ld,
                                             const int8_t *__restrict__ Jrow,
                                             const int *__restrict__ slot, int kk, int r0, int r1,
                                             bool isH, double2 *__restrict__ out)
{
    __shared__ double2 xs[GRAM_KT][KKMAX + 1];   // padded: the staging stores walk down rows
    __shared__ double xd[GRAM_KT][KKMAX + 1];    // xr - xi
    __shared__ double xp[GRAM_KT][KKMAX + 1];    // xr + xi
    __shared__ unsigned long long sgn[GRAM_KT];
    __shared__ int cols[KKMAX];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int nt = (kk + 15) >> 4;
    const bool dwarp = warp == (nthr >> 5) - 1;  // the diagonal tiles' warp
    // off-diagonal tile: rows qr + ly + 4i, columns qc + lx + 4j
    const int ly = (tid >> 2) & 3, lx = tid & 3;
    int qr = 0, qc = 0;
    bool active;
    // diagonal tile: base db, lane rho, its two rows ra, rb; slots s < split
    // take row ra and column db + rho + 1 + s, the others row rb, column db + s
    const int rho = lane & 7, db = 16 * (lane >> 3);
    const int ra = db + rho, rb = db + 14 - rho, split = 15 - rho;
    if (!dwarp) {
        int u = tid >> 4, ti = 0;
        active = u < nt * (nt - 1) / 2;
        if (active) {
            while (u >= nt - 1 - ti) { u -= nt - 1 - ti; ++ti; }
            qr = 16 * ti;
            qc = 16 * (ti + 1 + u);
        }
    } else {
        active = (lane >> 3) < nt;
    }
    const int dc = tid >> 1, dpart = tid & 1;   // diagonal sum share
    const bool dact = dc < 16 * nt;
    for (int s = tid; s < KKMAX; s += nthr) cols[s] = s < kk ? slot[s] : -1;
    const unsigned long long signbit = 1ull << 63;

    double t1[16], t2[16], t3[16], dsum = 0.0;
#pragma unroll
    for (int e = 0; e < 16; ++e) { t1[e] = 0; t2[e] = 0; t3[e] = 0; }

    for (int k0 = r0; k0 < r1; k0 += GRAM_KT) {
        __syncthreads();
        for (int e = tid; e < GRAM_KT * KKMAX; e += nthr) {
            const int r = e % GRAM_KT, s = e / GRAM_KT;
            const int col = cols[s];
            double2 v = make_double2(0.0, 0.0);
            if (col >= 0) v = W[(long long)col * ld + k0 + r];
            xs[r][s] = v;
            xd[r][s] = v.x - v.y;
            xp[r][s] = v.x + v.y;
        }
        if (tid < GRAM_KT) sgn[tid] = (isH && Jrow[k0 + tid] < 0) ? signbit : 0ull;
        __syncthreads();
        if (dact) {
#pragma unroll 4
            for (int k = 0; k < GRAM_KT; ++k) {
                const double2 v = xs[k][dc];
                const double c = dpart ? v.y : v.x;
                dsum = fma(__longlong_as_double(__double_as_longlong(c) ^ sgn[k]), c, dsum);
            }
        }
        if (!active) continue;
        if (!dwarp) {
#pragma unroll 1
            for (int k = 0; k < GRAM_KT; ++k) {
                const unsigned long long sb = sgn[k];
                double2 x[4], y[4];
                double d[4], p[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    x[i] = xs[k][qr + ly + 4 * i];
                    d[i] = xd[k][qr + ly + 4 * i];
                    x[i].x = __longlong_as_double(__double_as_longlong(x[i].x) ^ sb);
                    x[i].y = __longlong_as_double(__double_as_longlong(x[i].y) ^ sb);
                    d[i] = __longlong_as_double(__double_as_longlong(d[i]) ^ sb);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    y[j] = xs[k][qc + lx + 4 * j];
                    p[j] = xp[k][qc + lx + 4 * j];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        t1[4 * i + j] = fma(x[i].x, y[j].x, t1[4 * i + j]);
                        t2[4 * i + j] = fma(x[i].y, y[j].y, t2[4 * i + j]);
                        t3[4 * i + j] = fma(d[i], p[j], t3[4 * i + j]);
                    }
            }
        } else {
#pragma unroll 1
            for (int k = 0; k < GRAM_KT; ++k) {
                const unsigned long long sb = sgn[k];
                double2 xa = xs[k][ra], xb = xs[k][rb];
                double da = xd[k][ra], dbv = xd[k][rb];
                xa.x = __longlong_as_double(__double_as_longlong(xa.x) ^ sb);
                xa.y = __longlong_as_double(__double_as_longlong(xa.y) ^ sb);
                xb.x = __longlong_as_double(__double_as_longlong(xb.x) ^ sb);
                xb.y = __longlong_as_double(__double_as_longlong(xb.y) ^ sb);
                da = __longlong_as_double(__double_as_longlong(da) ^ sb);
                dbv = __longlong_as_double(__double_as_longlong(dbv) ^ sb);
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const bool a = e < split;
                    const int c = db + (a ? rho + 1 + e : e);
                    const double2 y = xs[k][c];
                    const double p = xp[k][c];
                    t1[e] = fma(a ? xa.x : xb.x, y.x, t1[e]);
                    t2[e] = fma(a ? xa.y : xb.y, y.y, t2[e]);
                    t3[e] = fma(a ? da : dbv, p, t3[e]);
                }
            }
        }
    }
    // the diagonal: both halves of column dc meet in lanes 2c, 2c + 1
    dsum += __shfl_xor_sync(0xffffffffu, dsum, 1);
    if (dact && dpart == 0) out[dc + KKMAX * dc] = make_double2(dsum, 0.0);
    if (!active) return;
    if (!dwarp) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int e = 4 * i + j;
                out[(qr + ly + 4 * i) + KKMAX * (qc + lx + 4 * j)] =
                    make_double2(t1[e] + t2[e], (t3[e] - t1[e]) + t2[e]);
            }
    } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            if (rho == 7 && e >= 8) continue;      // row 7 has 8 entries
            const bool a = e < split;
            const int r = a ? ra : rb, c = db + (a ? rho + 1 + e : e);
            out[r + KKMAX * c] = make_double2(t1[e] + t2[e], (t3[e] - t1[e]) + t2[e]);
        }
    }
}

// The body, for one (pair, row chunk): rows [r0, r1) of W (ld), the pair's
// kk slot columns `slot`, J signs applied iff isH; writes the partial to out.
// The complex64 form uses four real FMA chains per entry, and stages the row
// blocks in two shared buffers: the cp.async copies of block b + 1 are in
// flight while block b is multiplied (the FP32 pipe does not hide a load
// round trip per block by itself).
template <typename T>
__device__ __forceinline__ void gram_body_4m(const typename cplx<T>::t *__restrict__ W, long long ld,
                                          const int8_t *__restrict__ Jrow,
                                          const int *__restrict__ slot, int kk, int r0, int r1,
                                          bool isH, typename cplx<T>::t *__restrict__ out)
{
    using T2 = typename cplx<T>::t;
    using U = typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned int>::type;
    __shared__ T2 xs[2][GRAM_KT][KKMAX + 1];   // padded: the staging stores walk down rows
    __shared__ U sgn[2][GRAM_KT];
    __shared__ int cols[KKMAX];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lx = tid & 3, ly = (tid >> 2) & 3;
    int ti, tj;
    const bool active = gram_tile(kk, tid >> 4, ti, tj);
    const bool diag = ti == tj;
    const int qr = 16 * ti, qc = 16 * tj;
    for (int s = tid; s < KKMAX; s += nthr) cols[s] = s < kk ? slot[s] : -1;
    const U signbit = (U)1 << (sizeof(T) * 8 - 1);

    T accr[4][4], acci[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { accr[i][j] = 0; acci[i][j] = 0; }

    // stage GRAM_KT rows x KKMAX slots of block k0 into buffer b;
    // consecutive threads copy consecutive rows
    auto stage = [&](int b, int k0) {
        for (int e = tid; e < GRAM_KT * KKMAX; e += nthr) {
            const int r = e % GRAM_KT, s = e / GRAM_KT;
            const int col = cols[s];
            if (col >= 0) {
                cp_async<sizeof(T2)>(&xs[b][r][s], W + (long long)col * ld + k0 + r);
            } else {
                T2 z;
                z.x = 0;
                z.y = 0;
                xs[b][r][s] = z;
            }
        }
        cp_async_commit();
    };
    __syncthreads();                               // cols
    stage(0, r0);
    if (tid < GRAM_KT) sgn[0][tid] = (isH && Jrow[r0 + tid] < 0) ? signbit : (U)0;
    int b = 0;
    for (int k0 = r0; k0 < r1; k0 += GRAM_KT, b ^= 1) {
        const bool more = k0 + GRAM_KT < r1;
        int8_t jnext = 1;                          // sign of row tid of the next block
        if (more) {
            stage(b ^ 1, k0 + GRAM_KT);
            if (isH && tid < GRAM_KT) jnext = Jrow[k0 + GRAM_KT + tid];
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (active) {
#pragma unroll 4
            for (int k = 0; k < GRAM_KT; ++k) {
                const U sb = sgn[b][k];
                T2 x[4], y[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    x[i] = xs[b][k][qr + ly + 4 * i];
                    if (sizeof(T) == 8) {
                        x[i].x = __longlong_as_double(__double_as_longlong(x[i].x) ^ sb);
                        x[i].y = __longlong_as_double(__double_as_longlong(x[i].y) ^ sb);
                    } else {
                        x[i].x = __int_as_float(__float_as_int(x[i].x) ^ (unsigned)sb);
                        x[i].y = __int_as_float(__float_as_int(x[i].y) ^ (unsigned)sb);
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) y[j] = xs[b][k][qc + lx + 4 * j];
                // acc_ij += conj(J x_i) y_j; in a diagonal tile the entries below
                // the diagonal (i > j) are not needed (the block pivot is Hermitian)
                if (diag) {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = i; j < 4; ++j) {
                            accr[i][j] = fma(x[i].x, y[j].x, accr[i][j]);
                            accr[i][j] = fma(x[i].y, y[j].y, accr[i][j]);
                            acci[i][j] = fma(x[i].x, y[j].y, acci[i][j]);
                            acci[i][j] = fma(-x[i].y, y[j].x, acci[i][j]);
                        }
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            accr[i][j] = fma(x[i].x, y[j].x, accr[i][j]);
                            accr[i][j] = fma(x[i].y, y[j].y, accr[i][j]);
                            acci[i][j] = fma(x[i].x, y[j].y, acci[i][j]);
                            acci[i][j] = fma(-x[i].y, y[j].x, acci[i][j]);
                        }
                }
            }
        }
        if (more && tid < GRAM_KT) sgn[b ^ 1][tid] = jnext < 0 ? signbit : (U)0;
        __syncthreads();                           // buffer b is free for block k0 + 2 GRAM_KT
    }
    // out[i + KKMAX j] (column-major), entries on and above the diagonal only
    if (!active) return;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ii = qr + ly + 4 * i, jj = qc + lx + 4 * j;
            if (ii > jj) continue;
            T2 v;
            v.x = accr[i][j];
            v.y = acci[i][j];
            out[ii + KKMAX * jj] = v;
        }
}

template <typename T>
__device__ __forceinline__ void gram_body(const typename cplx<T>::t *__restrict__ W, long long ld,
                                          const int8_t *__restrict__ Jrow,
                                          const int *__restrict__ slot, int kk, int r0, int r1,
                                          bool isH, typename cplx<T>::t *__restrict__ out)
{
    if constexpr (std::is_same<T, double>::value)
        gram_body_3m(W, ld, Jrow, slot, kk, r0, r1, isH, out);
    else
        gram_body_4m<T>(W, ld, Jrow, slot, kk, r0, r1, isH, out);
}

// One outer step of one pencil: CTA = (pair, row chunk).
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 128 : 160, 3)
gram_kernel(const typename cplx<T>::t *__restrict__ W, const int8_t *__restrict__ Jrow,
            StepArgs a, typename cplx<T>::t *__restrict__ partial)
{
    const int cpp = a.chunks_h + a.chunks_s;
    const int pair = blockIdx.x / cpp;
    const int c = blockIdx.x % cpp;
    const bool isH = c < a.chunks_h;
    const int r0 = isH ? c * a.kc : a.m_pad + (c - a.chunks_h) * a.kc;
    const int r1 = isH ? min(r0 + a.kc, a.m_pad) : min(r0 + a.kc, a.m_pad + a.p_pad);
    gram_body<T>(W, a.ld, Jrow, a.slotcol + pair * a.kk, a.kk, r0, r1, isH,
                 partial + ((long long)pair * cpp + c) * (KKMAX * KKMAX));
}

}  // namespace hz
