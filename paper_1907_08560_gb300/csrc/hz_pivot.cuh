// hz_pivot.cuh -- the 2x2 Hari-Zimmermann transformation on the GPU.
//
// arXiv 1907.08560, Section 6.1: given the pivot submatrices of eq. 6.1,
//   H^ = [hpp hpq; conj(hpq) hqq],  S^ = [spp spq; conj(spq) sqq],
// decide by eq. 6.12 whether to transform and build Z' = D0^ Z^ from
// eq. 6.5, 6.7, 6.10 and 6.11, with the exceptional cases of Section 6.1.6.
// The FP64 sweeps compute the parameters in FP64; the complex64 sweeps of
// the mixed schedule in FP32, with the big/small classification of FP64.
//
// Readings where the paper is silent or garbled:
//   - eq. 6.12 is applied to the prescaled pivot with square roots of the
//     diagonal magnitudes (crit_mode 0), or as printed (crit_mode 1);
//   - sigma = sgn(h) with sgn(0) = +1;
//   - sin(2 theta), cos(2 theta) come from the tan(2 theta) fraction by
//     hypot, cos(2 theta) >= 0;
//   - no transformation applies nothing (not even D0^);
//   - x = |s_pq| >= 1 after prescaling, or a nonpositive s_pp, is a
//     numerically dependent G pivot (error).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace hz {

// Correctly rounded operations that the compiler may not contract into FMAs,
// for both precisions of the parameters.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// sqrt(a^2 + b^2) that never falls below max(|a|, |b|): when the smaller
// argument is negligible it returns the larger one exactly, so that the
// cosines formed as ratios below never exceed 1 by a rounding error (a cosine
// above 1 would misclassify a negligible transformation as "big").
template <typename T>
__device__ __forceinline__ T hyp(T a, T b)
{
    a = fabs(a);
    b = fabs(b);
    const T M = fmax(a, b), mn = fmin(a, b);
    if (M == T(0) || mn == T(0)) return M;
    const T q = mn / M;
    return mul_rn(M, sqrt(fma_rn(q, q, T(1))));
}

// Result codes of pivot2x2.
constexpr int PIV_NONE = 0;
constexpr int PIV_TRANSFORM = 1;
constexpr int PIV_ERR_RANK = -2;
constexpr int PIV_ERR_NONFINITE = -3;

// z[0..7] = re/im of z11, z12, z21, z22 (row-major 2x2) on PIV_TRANSFORM.
// T = double for the FP64 sweeps; T = float for the complex64 sweeps (their
// data are complex64), where "big" is decided by the FP64 criterion on
// sin(phi) and sin(psi) rather than by cos = 1 in FP32.
template <typename T>
__device__ __forceinline__ int pivot2x2(T hpp, T hqq, T hpq_re, T hpq_im, T spp, T sqq, T spq_re,
                                        T spq_im, T tol, int crit_mode, T z[8], int *big)
{
    const T one = T(1), zero = T(0), half = T(0.5);
    *big = 0;
    if (!(spp > zero) || !(sqq > zero)) return PIV_ERR_RANK;
    if (!isfinite(hpp) || !isfinite(hqq) || !isfinite(hpq_re) || !isfinite(hpq_im) ||
        !isfinite(spp) || !isfinite(sqq) || !isfinite(spq_re) || !isfinite(spq_im))
        return PIV_ERR_NONFINITE;

    // Section 6.1.1: prescale the pivot so that diag(D0 S^ D0) = I.
    const T dp = one / sqrt(spp);
    const T dq = one / sqrt(sqq);
    const T dpq = dp * dq;
    const T h11 = mul_rn(mul_rn(hpp, dp), dp);
    const T h22 = mul_rn(mul_rn(hqq, dq), dq);
    const T h12r = hpq_re * dpq, h12i = hpq_im * dpq;
    const T s12r = spq_re * dpq, s12i = spq_im * dpq;

    // eq. 6.12 on the prescaled pivot.
    const T a1 = fabs(h11), a2 = fabs(h22);
    const T hmax = fmax(a1, a2), hmin = fmin(a1, a2);
    const T ah12 = hyp(h12r, h12i);
    const T x = hyp(s12r, s12i);
    const bool crit_h = crit_mode == 0 ? ah12 >= (sqrt(hmax) * tol) * sqrt(hmin)
                                       : ah12 >= (hmax * tol) * hmin;
    if (!crit_h && !(x >= tol)) return PIV_NONE;
    // Section 6.1.6: both pivots already diagonal.
    if (h12r == zero && h12i == zero && s12r == zero && s12i == zero) return PIV_NONE;
    if (!(x < one)) return PIV_ERR_RANK;

    // Section 6.1.2: e^{i alpha_1} = s_pq / |s_pq| (alpha_1 = 0 when x = 0).
    T e1r = one, e1i = zero;
    if (x != zero) { e1r = s12r / x; e1i = s12i / x; }
    const T t = sqrt((one - x) * (one + x));
    // eq. 6.5: u + iv = e^{-i alpha_1} h_pq.
    const T u = e1r * h12r + e1i * h12i;
    const T v = e1r * h12i - e1i * h12r;
    const T h = h22 - h11;

    T z11r, z11i, z12r, z12i, z21r, z21i, z22r, z22i;
    if (h == zero && v == zero) {
        // Section 6.1.6: Z^ = R1^ D2^, R1^ of eq. 6.2 at phi_1 = -pi/4,
        // D2^ = diag((1+x)^{-1/2}, (1-x)^{-1/2}) (Section 6.1.3).
        const T c = T(0.70710678118654752440);   // cos(pi/4)
        const T d1 = one / sqrt(one + x), d2 = one / sqrt(one - x);
        z11r = c * d1;        z11i = zero;
        z12r = -e1r * c * d2; z12i = -e1i * c * d2;
        z21r = e1r * c * d1;  z21i = -e1i * c * d1;
        z22r = c * d2;        z22i = zero;
        *big = 1;
    } else {
        const T sigma = h >= zero ? one : -one;                 // eq. 6.6
        const T hv = hyp(h, T(2) * v);
        const T num = sigma * (T(2) * u - (h11 + h22) * x);     // eq. 6.7
        const T den = mul_rn(t, hv);
        const T r = hyp(num, den);
        const T s2t = num / r, c2t = den / r;
        const T cg = fabs(h) / hv;                              // eq. 6.11
        const T sg = sigma * T(2) * v / hv;
        // eq. 6.10, evaluated in this order without contraction: whether
        // cos(phi) and cos(psi) round to exactly 1 decides "big" (6.1.7)
        const T xs = mul_rn(x, s2t);
        const T tcc = mul_rn(mul_rn(t, cg), c2t);
        const T cphi = sqrt(mul_rn(add_rn(add_rn(one, xs), tcc), half));
        const T cpsi = sqrt(mul_rn(add_rn(sub_rn(one, xs), tcc), half));
        const T tsc = t * sg * c2t;
        // e^{i alpha} sin(phi) = e^{i alpha_1} ((s2t - x) + i tsc) / (2 cos psi)
        const T ar = (s2t - x) / (T(2) * cpsi), ai = tsc / (T(2) * cpsi);
        // e^{-i beta} sin(psi) = e^{-i alpha_1} ((s2t + x) - i tsc) / (2 cos phi)
        const T br = (s2t + x) / (T(2) * cphi), bi = -tsc / (T(2) * cphi);
        const T it = one / t;
        // eq. 6.9 with the phases removed by Phi_4 (Section 6.1.5).
        z11r = cphi * it;                     z11i = zero;
        z12r = (e1r * ar - e1i * ai) * it;    z12i = (e1r * ai + e1i * ar) * it;
        z21r = -(e1r * br + e1i * bi) * it;   z21i = -(e1r * bi - e1i * br) * it;
        z22r = cpsi * it;                     z22i = zero;
        if (sizeof(T) == sizeof(double)) {
            *big = !(cphi == one && cpsi == one);   // Section 6.1.7
        } else {
            // FP32 parameters (complex64 sweeps): classify as the FP64 test
            // would; cos^2(phi) = 1 - sin^2(phi) rounds to 1 in FP64 iff
            // sin(phi) < 2^-27 (about); sin(phi) and sin(psi) are
            // |ar + i ai| and |br + i bi|, accurate in FP32
            const T thr = T(7.450580596923828e-09);
            *big = hyp(ar, ai) >= thr || hyp(br, bi) >= thr;
        }
    }
    // Z' = D0^ Z^.
    z[0] = dp * z11r; z[1] = dp * z11i; z[2] = dp * z12r; z[3] = dp * z12i;
    z[4] = dq * z21r; z[5] = dq * z21i; z[6] = dq * z22r; z[7] = dq * z22i;
    return PIV_TRANSFORM;
}

// The partner lane's value (lanes 2i, 2i+1 of the mask m).
__device__ __forceinline__ double pswap(double v, unsigned m) { return __shfl_xor_sync(m, v, 1); }

// The input tests of pivot2x2 on a lane pair: each lane tests the four
// inputs it owns (s_pp or s_qq first: PIV_ERR_RANK before
// PIV_ERR_NONFINITE), in the inputs' own precision; 0 if both pass.
template <typename TI>
__device__ __forceinline__ int pair_checks(unsigned m, TI s_own, TI h_own, TI hpq_own, TI spq_own)
{
    const int rank = !(s_own > TI(0));
    const int fin = isfinite(s_own) && isfinite(h_own) && isfinite(hpq_own) && isfinite(spq_own);
    const int bits = rank | (fin ? 0 : 2);
    const int both = bits | __shfl_xor_sync(m, bits, 1);
    return (both & 1) ? PIV_ERR_RANK : (both & 2) ? PIV_ERR_NONFINITE : 0;
}

// pivot2x2<double> on two lanes (k = 0, 1 of a lane pair; m = the pair's
// mask), for the FP64 sweeps: every value is formed by the same operations
// as in pivot2x2, in the lane that owns it (lane 0: the p side, real parts,
// phi; lane 1: the q side, imaginary parts, psi), and the two lanes swap by
// shuffles.  The chain holds 10 divisions and 7 square roots instead of 17
// and 11 (an FP64 warp instruction occupies the FP64 pipe for the same time
// whatever its active lanes).  Each lane reads and tests the four inputs it
// owns (in their own precision TI) and returns its own row of Z',
// zrow[0..3] = (re, im) of z_k1, z_k2 (lane 0: z11, z12; lane 1: z21, z22);
// both lanes return the same code and *big.
template <typename TI>
__device__ __forceinline__ int pivot2x2_x2(int k, unsigned m, TI hpp, TI hqq, TI hpq_re, TI hpq_im, TI spp,
                                           TI sqq, TI spq_re, TI spq_im, double tol, int crit_mode,
                                           double zrow[4], int *big)
{
    const double one = 1.0, zero = 0.0, half = 0.5;
    *big = 0;
    const TI s_own = k ? sqq : spp, h_own = k ? hqq : hpp;
    const TI hpq_own = k ? hpq_im : hpq_re, spq_own = k ? spq_im : spq_re;
    if (const int bad = pair_checks<TI>(m, s_own, h_own, hpq_own, spq_own)) return bad;
    // Section 6.1.1
    const double d = one / sqrt((double)s_own), d_o = pswap(d, m);
    const double dp = k ? d_o : d, dq = k ? d : d_o;
    const double dpq = dp * dq;
    const double hh = mul_rn(mul_rn((double)h_own, d), d), hh_o = pswap(hh, m);
    const double h11 = k ? hh_o : hh, h22 = k ? hh : hh_o;
    const double ho = (double)hpq_own * dpq, so = (double)spq_own * dpq;
    const double ho_o = pswap(ho, m), so_o = pswap(so, m);
    const double h12r = k ? ho_o : ho, h12i = k ? ho : ho_o;
    const double s12r = k ? so_o : so, s12i = k ? so : so_o;
    // eq. 6.12 (lane 0: |h_pq|, sqrt(hmax); lane 1: x, sqrt(hmin))
    const double a1 = fabs(h11), a2 = fabs(h22);
    const double hmax = fmax(a1, a2), hmin = fmin(a1, a2);
    const double hx = k ? hyp(s12r, s12i) : hyp(h12r, h12i), hx_o = pswap(hx, m);
    const double ah12 = k ? hx_o : hx, x = k ? hx : hx_o;
    bool crit_h;
    if (crit_mode == 0) {
        const double sr = sqrt(k ? hmin : hmax), sr_o = pswap(sr, m);
        crit_h = ah12 >= ((k ? sr_o : sr) * tol) * (k ? sr : sr_o);
    } else {
        crit_h = ah12 >= (hmax * tol) * hmin;
    }
    if (!crit_h && !(x >= tol)) return PIV_NONE;
    if (h12r == zero && h12i == zero && s12r == zero && s12i == zero) return PIV_NONE;
    if (!(x < one)) return PIV_ERR_RANK;
    // Section 6.1.2
    double e1r = one, e1i = zero;
    if (x != zero) {
        const double e = (k ? s12i : s12r) / x, e_o = pswap(e, m);
        e1r = k ? e_o : e;
        e1i = k ? e : e_o;
    }
    const double pmx = k ? one + x : one - x;
    const double t = sqrt(k ? pswap(pmx, m) * pmx : pmx * pswap(pmx, m));   // (1 - x)(1 + x)
    // eq. 6.5 (lane 0: u, lane 1: v)
    const double uv = k ? e1r * h12i - e1i * h12r : e1r * h12r + e1i * h12i, uv_o = pswap(uv, m);
    const double u = k ? uv_o : uv, v = k ? uv : uv_o;
    const double h = h22 - h11;
    double zr0, zi0, zr1, zi1;      // lane 0: z11, z12; lane 1: z21, z22
    if (h == zero && v == zero) {                           // Section 6.1.6
        const double c = 0.70710678118654752440;
        const double dd = one / sqrt(k ? one - x : one + x), dd_o = pswap(dd, m);
        const double d1 = k ? dd_o : dd, d2 = k ? dd : dd_o;
        if (k == 0) { zr0 = c * d1; zi0 = zero; zr1 = -e1r * c * d2; zi1 = -e1i * c * d2; }
        else { zr0 = e1r * c * d1; zi0 = -e1i * c * d1; zr1 = c * d2; zi1 = zero; }
        *big = 1;
    } else {
        const double sigma = h >= zero ? one : -one;        // eq. 6.6
        const double hv = hyp(h, 2.0 * v);
        // eq. 6.7 (lane 0: num, lane 1: den)
        const double nd = k ? mul_rn(t, hv) : sigma * (2.0 * u - (h11 + h22) * x), nd_o = pswap(nd, m);
        const double num = k ? nd_o : nd, den = k ? nd : nd_o;
        const double r = hyp(num, den);
        const double sc = nd / r, sc_o = pswap(sc, m);      // sin 2theta | cos 2theta
        const double s2t = k ? sc_o : sc, c2t = k ? sc : sc_o;
        // eq. 6.11 (lane 0: cos gamma, lane 1: sin gamma)
        const double gg = k ? sigma * 2.0 * v / hv : fabs(h) / hv, gg_o = pswap(gg, m);
        const double cg = k ? gg_o : gg, sg = k ? gg : gg_o;
        // eq. 6.10 in the order of pivot2x2, without contraction
        const double xt = k ? mul_rn(mul_rn(t, cg), c2t) : mul_rn(x, s2t), xt_o = pswap(xt, m);
        const double xs = k ? xt_o : xt, tcc = k ? xt : xt_o;
        const double cc = k ? sqrt(mul_rn(add_rn(sub_rn(one, xs), tcc), half))
                            : sqrt(mul_rn(add_rn(add_rn(one, xs), tcc), half));   // cos phi | cos psi
        const double cc_o = pswap(cc, m);
        const double cphi = k ? cc_o : cc, cpsi = k ? cc : cc_o;
        const double tsc = t * sg * c2t;
        // lane 0: e^{i alpha} sin(phi) = ((s2t - x) + i tsc) / (2 cos psi)
        // lane 1: e^{-i beta} sin(psi) = ((s2t + x) - i tsc) / (2 cos phi)
        const double den2 = 2.0 * (k ? cphi : cpsi);
        const double abr = (k ? s2t + x : s2t - x) / den2, abi = (k ? -tsc : tsc) / den2;
        const double abr_o = pswap(abr, m), abi_o = pswap(abi, m);
        const double ar = k ? abr_o : abr, ai = k ? abi_o : abi;
        const double br = k ? abr : abr_o, bi = k ? abi : abi_o;
        const double it = one / t;
        if (k == 0) {
            zr0 = cphi * it;                  zi0 = zero;
            zr1 = (e1r * ar - e1i * ai) * it; zi1 = (e1r * ai + e1i * ar) * it;
        } else {
            zr0 = -(e1r * br + e1i * bi) * it; zi0 = -(e1r * bi - e1i * br) * it;
            zr1 = cpsi * it;                   zi1 = zero;
        }
        *big = !(cphi == one && cpsi == one);               // Section 6.1.7
    }
    // Z' = D0^ Z^: lane 0 scales the first row by dp, lane 1 the second by dq
    zrow[0] = d * zr0; zrow[1] = d * zi0; zrow[2] = d * zr1; zrow[3] = d * zi1;
    return PIV_TRANSFORM;
}

// The same 2x2 transformation with FP64 parameters for the complex64 sweeps
// of the mixed schedule: the formulas of pivot2x2 with every square root and
// division taken from one reciprocal square root (sqrt(q) = q rsqrt(q),
// 1/sqrt(q) = rsqrt(q)), eq. 6.12 compared in squares (errors of a few FP64
// ulps, far below the complex64 data the parameters are applied to), and
// "big" decided by sin(phi), sin(psi) >= 2^-27, the FP64 test on a cosine
// rounding to 1.
//
// It runs on two lanes (k = 0, 1 of a lane pair; m = the pair's mask).  An
// FP64 warp instruction occupies a sub-partition's FP64 pipe for the same
// time whatever its active lanes, and nearly every quantity of eq. 6.5-6.11
// comes in a pair (the p and q sides, real and imaginary parts, phi and psi):
// lane 0 computes one member, lane 1 the other, and the two swap by a
// shuffle (measured on the one-lane form of the same formulas: eight
// reciprocal square roots and about twice the products on the critical
// path).  Inputs and outputs as pivot2x2_x2: each lane tests and converts
// its own four inputs and returns its own row of Z' in zrow[0..3]; both lanes
// return the same code and *big.
template <typename TI>
__device__ __forceinline__ int pivot2x2_fast_x2(int k, unsigned m, TI hpp, TI hqq, TI hpq_re, TI hpq_im,
                                                TI spp, TI sqq, TI spq_re, TI spq_im, double tol,
                                                int crit_mode, double zrow[4], int *big)
{
    *big = 0;
    const TI s_own = k ? sqq : spp, h_own = k ? hqq : hpp;
    const TI hpq_own = k ? hpq_im : hpq_re, spq_own = k ? spq_im : spq_re;
    if (const int bad = pair_checks<TI>(m, s_own, h_own, hpq_own, spq_own)) return bad;
    // Section 6.1.1 (lane 0: p, lane 1: q)
    const double d = rsqrt((double)s_own), d_o = pswap(d, m);
    const double dp = k ? d_o : d, dq = k ? d : d_o;
    const double dpq = dp * dq;
    const double hh = (double)h_own * d * d, hh_o = pswap(hh, m);
    const double h11 = k ? hh_o : hh, h22 = k ? hh : hh_o;
    const double ho = (double)hpq_own * dpq, so = (double)spq_own * dpq;
    const double ho_o = pswap(ho, m), so_o = pswap(so, m);
    const double h12r = k ? ho_o : ho, h12i = k ? ho : ho_o;
    const double s12r = k ? so_o : so, s12i = k ? so : so_o;
    const double a1 = fabs(h11), a2 = fabs(h22);
    const double hmax = fmax(a1, a2), hmin = fmin(a1, a2);
    // |h_pq|^2 (lane 0) and x^2 (lane 1)
    const double sq = k ? s12r * s12r + s12i * s12i : h12r * h12r + h12i * h12i, sq_o = pswap(sq, m);
    const double ah2 = k ? sq_o : sq, x2 = k ? sq : sq_o;
    const double ch = crit_mode == 0 ? (hmax * tol) * (hmin * tol) : (hmax * tol) * hmin;
    const bool crit_h = crit_mode == 0 ? ah2 >= ch : ah2 >= ch * ch;
    if (!crit_h && !(x2 >= tol * tol)) return PIV_NONE;    // eq. 6.12
    if (h12r == 0.0 && h12i == 0.0 && s12r == 0.0 && s12i == 0.0) return PIV_NONE;
    if (!(x2 < 1.0)) return PIV_ERR_RANK;
    double x = 0.0, e1r = 1.0, e1i = 0.0;                  // Section 6.1.2
    if (x2 != 0.0) {
        const double ix = rsqrt(x2);
        x = x2 * ix;
        const double e = (k ? s12i : s12r) * ix, e_o = pswap(e, m);
        e1r = k ? e_o : e;
        e1i = k ? e : e_o;
    }
    const double pmx = k ? 1.0 + x : 1.0 - x;
    const double t2 = pmx * pswap(pmx, m);                 // (1 - x)(1 + x)
    const double it = rsqrt(t2), t = t2 * it;
    // eq. 6.5: u (lane 0), v (lane 1)
    const double uv = k ? e1r * h12i - e1i * h12r : e1r * h12r + e1i * h12i, uv_o = pswap(uv, m);
    const double u = k ? uv_o : uv, v = k ? uv : uv_o;
    const double h = h22 - h11;
    double zr0, zi0, zr1, zi1;      // lane 0: z11, z12; lane 1: z21, z22
    if (h == 0.0 && v == 0.0) {                             // Section 6.1.6
        const double c = 0.70710678118654752440;
        const double d1 = rsqrt(1.0 + x), d2 = rsqrt(1.0 - x);
        if (k == 0) { zr0 = c * d1; zi0 = 0.0; zr1 = -e1r * c * d2; zi1 = -e1i * c * d2; }
        else { zr0 = e1r * c * d1; zi0 = -e1i * c * d1; zr1 = c * d2; zi1 = 0.0; }
        *big = 1;
    } else {
        const double sigma = h >= 0.0 ? 1.0 : -1.0;        // eq. 6.6
        const double hv2 = h * h + 4.0 * v * v;
        const double ihv = rsqrt(hv2), hv = hv2 * ihv;
        // eq. 6.7: num (lane 0), den (lane 1)
        const double nd = k ? t * hv : sigma * (2.0 * u - (h11 + h22) * x), nd_o = pswap(nd, m);
        const double num = k ? nd_o : nd, den = k ? nd : nd_o;
        const double ir = rsqrt(num * num + den * den);
        const double sc = nd * ir, sc_o = pswap(sc, m);    // sin 2theta | cos 2theta
        const double s2t = k ? sc_o : sc, c2t = k ? sc : sc_o;
        // eq. 6.11: cos gamma (lane 0), sin gamma (lane 1)
        const double gg = k ? sigma * 2.0 * v * ihv : fabs(h) * ihv, gg_o = pswap(gg, m);
        const double cg = k ? gg_o : gg, sg = k ? gg : gg_o;
        // eq. 6.10: x sin 2theta (lane 0), t cos gamma cos 2theta (lane 1)
        const double xt = k ? t * cg * c2t : x * s2t, xt_o = pswap(xt, m);
        const double xs = k ? xt_o : xt, tcc = k ? xt : xt_o;
        const double q = k ? (1.0 - xs + tcc) * 0.5 : (1.0 + xs + tcc) * 0.5;   // phi | psi
        const double r = rsqrt(q), c = q * r;             // 1/cos, cos
        const double r_o = pswap(r, m);
        const double ipq = 0.5 * r_o;                       // 1/(2 cos psi) | 1/(2 cos phi)
        const double tsc = t * sg * c2t;
        const double abr = (k ? s2t + x : s2t - x) * ipq;  // ar | br
        const double abi = (k ? -tsc : tsc) * ipq;         // ai | bi
        const double abr_o = pswap(abr, m), abi_o = pswap(abi, m);
        const double ar = k ? abr_o : abr, ai = k ? abi_o : abi;
        const double br = k ? abr : abr_o, bi = k ? abi : abi_o;
        if (k == 0) {
            zr0 = c * it;                    zi0 = 0.0;
            zr1 = (e1r * ar - e1i * ai) * it; zi1 = (e1r * ai + e1i * ar) * it;
        } else {
            zr0 = -(e1r * br + e1i * bi) * it; zi0 = -(e1r * bi - e1i * br) * it;
            zr1 = c * it;                      zi1 = 0.0;
        }
        const double thr2 = 5.551115123125783e-17;         // (2^-27)^2
        const int own = abr * abr + abi * abi >= thr2;
        *big = own | __shfl_xor_sync(m, own, 1);
    }
    // Z' = D0^ Z^: lane 0 scales the first row by dp, lane 1 the second by dq
    zrow[0] = zr0 * d; zrow[1] = zi0 * d; zrow[2] = zr1 * d; zrow[3] = zi1 * d;
    return PIV_TRANSFORM;
}

// Round-robin (circle) ordering of N (even) slots, step r, pair k: slot N-1
// meets slot r; slot (r+k) mod (N-1) meets slot (r-k) mod (N-1); the smaller
// slot first.  Every pair appears exactly once in N-1 steps (Section 6.3).
__host__ __device__ __forceinline__ void rr_pair(int N, int r, int k, int *a, int *b)
{
    int p, q;
    if (k == 0) { p = N - 1; q = r; }
    else { p = (r + k) % (N - 1); q = (r - k + (N - 1)) % (N - 1); }
    *a = p < q ? p : q;
    *b = p < q ? q : p;
}

}  // namespace hz
