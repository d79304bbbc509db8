// hz_pivot.cuh -- the 2x2 Hari-Zimmermann transformation on the GPU, FP64.
//
// arXiv 1907.08560, Section 6.1: given the pivot submatrices of eq. 6.1,
//   H^ = [hpp hpq; conj(hpq) hqq],  S^ = [spp spq; conj(spq) sqq],
// decide by eq. 6.12 whether to transform and build Z' = D0^ Z^ from
// eq. 6.5, 6.7, 6.10 and 6.11, with the exceptional cases of Section 6.1.6.
// The rotation parameters are always computed in FP64, whatever the
// precision of the data they are applied to.
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

// sqrt(a^2 + b^2) that never falls below max(|a|, |b|): when the smaller
// argument is negligible it returns the larger one exactly, so that the
// cosines formed as ratios below never exceed 1 by a rounding error (a cosine
// above 1 would misclassify a negligible transformation as "big").
__device__ __forceinline__ double hyp(double a, double b)
{
    a = fabs(a);
    b = fabs(b);
    const double M = fmax(a, b), mn = fmin(a, b);
    if (M == 0.0 || mn == 0.0) return M;
    const double q = mn / M;
    return __dmul_rn(M, sqrt(__fma_rn(q, q, 1.0)));
}

// Result codes of pivot2x2.
constexpr int PIV_NONE = 0;
constexpr int PIV_TRANSFORM = 1;
constexpr int PIV_ERR_RANK = -2;
constexpr int PIV_ERR_NONFINITE = -3;

// z[0..7] = re/im of z11, z12, z21, z22 (row-major 2x2) on PIV_TRANSFORM.
__device__ __forceinline__ int pivot2x2(double hpp, double hqq, double hpq_re, double hpq_im,
                                        double spp, double sqq, double spq_re, double spq_im,
                                        double tol, int crit_mode, double z[8], int *big)
{
    *big = 0;
    if (!(spp > 0.0) || !(sqq > 0.0)) return PIV_ERR_RANK;
    if (!isfinite(hpp) || !isfinite(hqq) || !isfinite(hpq_re) || !isfinite(hpq_im) ||
        !isfinite(spp) || !isfinite(sqq) || !isfinite(spq_re) || !isfinite(spq_im))
        return PIV_ERR_NONFINITE;

    // Section 6.1.1: prescale the pivot so that diag(D0 S^ D0) = I.
    const double dp = 1.0 / sqrt(spp);
    const double dq = 1.0 / sqrt(sqq);
    const double dpq = dp * dq;
    const double h11 = __dmul_rn(__dmul_rn(hpp, dp), dp);
    const double h22 = __dmul_rn(__dmul_rn(hqq, dq), dq);
    const double h12r = hpq_re * dpq, h12i = hpq_im * dpq;
    const double s12r = spq_re * dpq, s12i = spq_im * dpq;

    // eq. 6.12 on the prescaled pivot.
    const double a1 = fabs(h11), a2 = fabs(h22);
    const double hmax = fmax(a1, a2), hmin = fmin(a1, a2);
    const double ah12 = hyp(h12r, h12i);
    const double x = hyp(s12r, s12i);
    const bool crit_h = crit_mode == 0 ? ah12 >= (sqrt(hmax) * tol) * sqrt(hmin)
                                       : ah12 >= (hmax * tol) * hmin;
    if (!crit_h && !(x >= tol)) return PIV_NONE;
    // Section 6.1.6: both pivots already diagonal.
    if (h12r == 0.0 && h12i == 0.0 && s12r == 0.0 && s12i == 0.0) return PIV_NONE;
    if (!(x < 1.0)) return PIV_ERR_RANK;

    // Section 6.1.2: e^{i alpha_1} = s_pq / |s_pq| (alpha_1 = 0 when x = 0).
    double e1r = 1.0, e1i = 0.0;
    if (x != 0.0) { e1r = s12r / x; e1i = s12i / x; }
    const double t = sqrt((1.0 - x) * (1.0 + x));
    // eq. 6.5: u + iv = e^{-i alpha_1} h_pq.
    const double u = e1r * h12r + e1i * h12i;
    const double v = e1r * h12i - e1i * h12r;
    const double h = h22 - h11;

    double z11r, z11i, z12r, z12i, z21r, z21i, z22r, z22i;
    if (h == 0.0 && v == 0.0) {
        // Section 6.1.6: Z^ = R1^ D2^, R1^ of eq. 6.2 at phi_1 = -pi/4,
        // D2^ = diag((1+x)^{-1/2}, (1-x)^{-1/2}) (Section 6.1.3).
        const double c = 0.70710678118654752440;   // cos(pi/4)
        const double d1 = 1.0 / sqrt(1.0 + x), d2 = 1.0 / sqrt(1.0 - x);
        z11r = c * d1;        z11i = 0.0;
        z12r = -e1r * c * d2; z12i = -e1i * c * d2;
        z21r = e1r * c * d1;  z21i = -e1i * c * d1;
        z22r = c * d2;        z22i = 0.0;
        *big = 1;
    } else {
        const double sigma = h >= 0.0 ? 1.0 : -1.0;              // eq. 6.6
        const double hv = hyp(h, 2.0 * v);
        const double num = sigma * (2.0 * u - (h11 + h22) * x);   // eq. 6.7
        const double den = __dmul_rn(t, hv);
        const double r = hyp(num, den);
        const double s2t = num / r, c2t = den / r;
        const double cg = fabs(h) / hv;                           // eq. 6.11
        const double sg = sigma * 2.0 * v / hv;
        // eq. 6.10, evaluated in this order without contraction: whether
        // cos(phi) and cos(psi) round to exactly 1 decides "big" (6.1.7)
        const double xs = __dmul_rn(x, s2t);
        const double tcc = __dmul_rn(__dmul_rn(t, cg), c2t);
        const double cphi = sqrt(__dmul_rn(__dadd_rn(__dadd_rn(1.0, xs), tcc), 0.5));
        const double cpsi = sqrt(__dmul_rn(__dadd_rn(__dsub_rn(1.0, xs), tcc), 0.5));
        const double tsc = t * sg * c2t;
        // e^{i alpha} sin(phi) = e^{i alpha_1} ((s2t - x) + i tsc) / (2 cos psi)
        const double ar = (s2t - x) / (2.0 * cpsi), ai = tsc / (2.0 * cpsi);
        // e^{-i beta} sin(psi) = e^{-i alpha_1} ((s2t + x) - i tsc) / (2 cos phi)
        const double br = (s2t + x) / (2.0 * cphi), bi = -tsc / (2.0 * cphi);
        const double it = 1.0 / t;
        // eq. 6.9 with the phases removed by Phi_4 (Section 6.1.5).
        z11r = cphi * it;                     z11i = 0.0;
        z12r = (e1r * ar - e1i * ai) * it;    z12i = (e1r * ai + e1i * ar) * it;
        z21r = -(e1r * br + e1i * bi) * it;   z21i = -(e1r * bi - e1i * br) * it;
        z22r = cpsi * it;                     z22i = 0.0;
        *big = !(cphi == 1.0 && cpsi == 1.0);   // Section 6.1.7
    }
    // Z' = D0^ Z^.
    z[0] = dp * z11r; z[1] = dp * z11i; z[2] = dp * z12r; z[3] = dp * z12i;
    z[4] = dq * z21r; z[5] = dq * z21i; z[6] = dq * z22r; z[7] = dq * z22i;
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
