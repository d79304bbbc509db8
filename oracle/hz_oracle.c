/*
 * hz_oracle.c -- plain, slow, FP64 CPU oracle for the implicit one-sided
 * Hari-Zimmermann (HZ) generalized hyperbolic SVD (Singer, Di Napoli,
 * Novakovic, Caklovic, arXiv 1907.08560, Section 6).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the
 * CUDA path.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or helper
 * with the GPU library, and the GPU library never calls it.
 *
 * Everything is written out in the paper's order and notation, with no
 * blocking, fusion or reordering beyond what the paper states:
 *   - hzo_pivot:     the 2x2 transformation Z' of Section 6.1 (eq. 6.1-6.11,
 *                    the exceptional cases of Section 6.1.6, the criterion
 *                    eq. 6.12 and the big/small classification of 6.1.7);
 *   - hzo_pointwise: Algorithm 1 of Section 6.1.8 (the pointwise implicit HZ
 *                    G(H)SVD), with a parallel cyclic (round-robin) strategy
 *                    (Section 6.3) and bordering for odd n (Section 6.3.2);
 *   - hzo_blocked:   the Level-2 block algorithm of Section 6.4 (block-column
 *                    partition 6.4.1, block pivots 6.4.2, BO/FB inner level,
 *                    block update 6.4.3, sweep completion);
 *   - hzo_finalize:  the outputs of Section 6.1.7 and eq. 3.2.
 *
 * Readings of the paper where it is silent or garbled (each is repeated in
 * the design notes):
 *   R1 eq. 6.12 compares |h_pq| with a product of two diagonal entries, which
 *      is not scale-consistent; the default (crit_mode 0) takes the square
 *      roots, |h_pq| >= (sqrt(max)*(eps*sqrt(n)))*sqrt(min), on the
 *      prescaled pivot; crit_mode 1 is the printed form.  eps = 2^-53.
 *   R2 stopping: a sweep with no "big" transformation ends the iteration
 *      (Section 6.1.7), at most max_sweeps (C_max = 30) sweeps.
 *   R3 sigma = sgn(h) with sgn(0) = +1.
 *   R4 sin(2 theta), cos(2 theta) come from the tan(2 theta) fraction of
 *      eq. 6.7 by hypot, with cos(2 theta) >= 0, i.e. theta in (-pi/4, pi/4].
 *   R5 no transformation (criterion not met, or h_pq = s_pq = 0) applies
 *      nothing, not even D0.
 *   R6 strategy: the round-robin (circle) ordering at both levels.
 *   R7 odd orders are bordered by a slot that never pairs with a column
 *      (its pivot pairs are exactly the h_pq = s_pq = 0 case).
 *   R8 the inner level of the block algorithm transforms the block pivots
 *      (H^, S^) two-sidedly, accumulating Z^, instead of factoring them into
 *      square factors first; both give the same Z^ in exact arithmetic.
 *   R9 x = |s_pq| >= 1 after prescaling means the pivot columns of G are
 *      numerically dependent: the oracle stops with an error (Section 6.4.2
 *      stops on a rank-deficient block pivot).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zc;

/* Return codes. */
#define HZO_OK 0
#define HZO_ERR_RANK -2     /* x >= 1 or s_pp <= 0: G columns dependent */
#define HZO_ERR_NONFINITE -3
#define HZO_ERR_ARG -1

/* ---------------------------------------------------------------------- */
/* Section 6.1: one 2x2 pivot.                                             */
/* ---------------------------------------------------------------------- */

/*
 * Given the pivot submatrices of eq. 6.1,
 *   H^ = [hpp hpq; conj(hpq) hqq],  S^ = [spp spq; conj(spq) sqq],
 * decide by eq. 6.12 whether to transform, and if so return
 * Z' = D0^ * Z^ (Section 6.1.5) in Zp = {z11, z12, z21, z22} (complex,
 * row-major 2x2), and *big = 1 unless cos(phi) = cos(psi) = 1.
 * tol = eps*sqrt(n).  Returns 1 (transform), 0 (none) or an error code.
 */
int hzo_pivot(double hpp, double hqq, zc hpq, double spp, double sqq, zc spq,
              double tol, int crit_mode, zc *Zp, int *big)
{
    *big = 0;
    if (!(spp > 0.0) || !(sqq > 0.0)) return HZO_ERR_RANK;
    if (!isfinite(hpp) || !isfinite(hqq) || !isfinite(creal(hpq)) ||
        !isfinite(cimag(hpq)) || !isfinite(spp) || !isfinite(sqq) ||
        !isfinite(creal(spq)) || !isfinite(cimag(spq)))
        return HZO_ERR_NONFINITE;

    /* 6.1.1: per-pivot prescaling, D0^ = diag(spp^{-1/2}, sqq^{-1/2}), so
     * that the diagonal of D0^ S^ D0^ is the identity. */
    double dp = 1.0 / sqrt(spp), dq = 1.0 / sqrt(sqq);
    double h11 = (hpp * dp) * dp;
    double h22 = (hqq * dq) * dq;
    zc h12 = hpq * (dp * dq);
    zc s12 = spq * (dp * dq);

    /* eq. 6.12 (reading R1), on the prescaled pivot. */
    double a1 = fabs(h11), a2 = fabs(h22);
    double hmax = a1 > a2 ? a1 : a2, hmin = a1 > a2 ? a2 : a1;
    int crit_h = crit_mode == 0 ? cabs(h12) >= (sqrt(hmax) * tol) * sqrt(hmin)
                                : cabs(h12) >= (hmax * tol) * hmin;
    int crit_s = cabs(s12) >= tol;
    if (!crit_h && !crit_s) return 0;

    /* 6.1.6, first exceptional case: both pivots already diagonal. */
    if (h12 == 0.0 && s12 == 0.0) return 0;

    /* 6.1.2: x = |s_pq|, alpha_1 = arg(s_pq) (0 if x = 0, second
     * exceptional case). */
    double x = cabs(s12);
    if (!(x < 1.0)) return HZO_ERR_RANK;
    zc e1 = x == 0.0 ? 1.0 : s12 / x;          /* e^{i alpha_1} */
    double t = sqrt((1.0 - x) * (1.0 + x));    /* t = sqrt(1 - x^2), eq. 6.7 */

    /* eq. 6.5: u + iv = e^{-i alpha_1} h_pq. */
    zc uv = conj(e1) * h12;
    double u = creal(uv), v = cimag(uv);
    double h = h22 - h11;                       /* h = h_qq - h_pp */

    zc z11, z12, z21, z22;
    if (h == 0.0 && v == 0.0) {
        /* 6.1.6, third exceptional case: Z^ = R1^ D2^, with R1^ the rotation
         * of eq. 6.2 at phi_1 = -pi/4, alpha_1, and
         * D2^ = diag((1+x)^{-1/2}, (1-x)^{-1/2}) (Section 6.1.3). */
        double c1 = cos(-M_PI / 4.0), s1 = sin(-M_PI / 4.0);
        double d21 = 1.0 / sqrt(1.0 + x), d22 = 1.0 / sqrt(1.0 - x);
        zc r11 = c1, r12 = e1 * s1, r21 = -conj(e1) * s1, r22 = c1;
        z11 = r11 * d21; z12 = r12 * d22;
        z21 = r21 * d21; z22 = r22 * d22;
        *big = 1;
    } else {
        /* eq. 6.6: sigma = sgn(h) (reading R3). */
        double sigma = h >= 0.0 ? 1.0 : -1.0;
        /* eq. 6.7: tan(2 theta) = sigma (2u - (h_pp + h_qq) x) /
         *                          (t sqrt(h^2 + 4 v^2)). */
        double hv = hypot(h, 2.0 * v);
        double num = sigma * (2.0 * u - (h11 + h22) * x);
        double den = t * hv;
        double r = hypot(num, den);
        double sin2t = num / r, cos2t = den / r;   /* reading R4 */
        /* eq. 6.11: tan(gamma) = 2v / h, gamma in (-pi/2, pi/2]. */
        double cosg = fabs(h) / hv;
        double sing = sigma * 2.0 * v / hv;
        /* eq. 6.10 */
        double cphi = sqrt((1.0 + x * sin2t + t * cosg * cos2t) / 2.0);
        double cpsi = sqrt((1.0 - x * sin2t + t * cosg * cos2t) / 2.0);
        zc ea_sphi = e1 * ((sin2t - x) + I * (t * sing * cos2t)) / (2.0 * cpsi);
        zc eb_spsi = conj(e1) * ((sin2t + x) - I * (t * sing * cos2t)) / (2.0 * cphi);
        /* eq. 6.9 with the phase factor removed by Phi_4 (Section 6.1.5). */
        z11 = cphi / t;
        z12 = ea_sphi / t;
        z21 = -eb_spsi / t;
        z22 = cpsi / t;
        /* Section 6.1.7: "small" iff cos(phi) = cos(psi) = 1. */
        *big = !(cphi == 1.0 && cpsi == 1.0);
    }
    /* Z' = D0^ Z^ */
    Zp[0] = dp * z11; Zp[1] = dp * z12;
    Zp[2] = dq * z21; Zp[3] = dq * z22;
    return 1;
}

/* ---------------------------------------------------------------------- */
/* Section 6.3: parallel cyclic strategy (reading R6).                    */
/* ---------------------------------------------------------------------- */

/*
 * Round-robin (circle method) ordering of N (even) slots: N-1 steps of N/2
 * disjoint pairs covering every pair exactly once.  In step r, slot N-1
 * meets slot r, and slot (r+k) mod (N-1) meets slot (r-k) mod (N-1) for
 * k = 1 .. N/2-1.  Each pair is returned with its smaller slot first.
 */
static void rr_pair(long N, long r, long k, long *a, long *b)
{
    long p, q;
    if (k == 0) { p = N - 1; q = r; }
    else { p = (r + k) % (N - 1); q = (r - k + (N - 1)) % (N - 1); }
    *a = p < q ? p : q;
    *b = p < q ? q : p;
}

/* ---------------------------------------------------------------------- */
/* Column kernels: J-dot products (eq. 6.1) and the 2-column update.      */
/* ---------------------------------------------------------------------- */

/* a^* J b over len rows; J == NULL means J = I. */
static zc jdot(long len, const zc *a, const zc *b, const signed char *J)
{
    zc s = 0.0;
    for (long i = 0; i < len; ++i) {
        zc t = conj(a[i]) * b[i];
        s += (J && J[i] < 0) ? -t : t;
    }
    return s;
}

/* [x_p, x_q] = [x_p, x_q] * Z' (the ZVROTM update of Section 6.2.1). */
static void rot2(long len, zc *xp, zc *xq, const zc *Zp)
{
    for (long i = 0; i < len; ++i) {
        zc a = xp[i], b = xq[i];
        xp[i] = a * Zp[0] + b * Zp[2];
        xq[i] = a * Zp[1] + b * Zp[3];
    }
}

static double eps_sqrt_n(long n) { return ldexp(1.0, -53) * sqrt((double)n); }

/* ---------------------------------------------------------------------- */
/* Algorithm 1 (Section 6.1.8): the pointwise implicit HZ G(H)SVD.         */
/* ---------------------------------------------------------------------- */

/*
 * F (m x n, ld ldf), G (p x n, ld ldg), Z (n x n, ld ldz) are complex,
 * column-major, overwritten in place; Z must hold the initial Z' (usually
 * I).  J has m entries +-1 (NULL: J = I).  Runs at most max_sweeps sweeps.
 * counts (may be NULL) receives 2 longs per sweep: all and big
 * transformations.  *sweeps receives the number of sweeps run.
 * Returns 0 when converged (a sweep without big transformations),
 * 1 when max_sweeps was reached, or a negative error code.
 */
int hzo_pointwise(long m, long p, long n, zc *F, long ldf, const signed char *J,
                  zc *G, long ldg, zc *Z, long ldz, int max_sweeps,
                  int crit_mode, int nthreads, long *sweeps, long *counts)
{
    if (m < 1 || p < 1 || n < 1 || ldf < m || ldg < p || ldz < n) return HZO_ERR_ARG;
    *sweeps = 0;
    if (n == 1) return 0;
    long N = n + (n & 1);            /* Section 6.3.2 bordering (R7) */
    double tol = eps_sqrt_n(n);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int status = 1;
    for (int it = 1; it <= max_sweeps; ++it) {
        long n_all = 0, n_big = 0;
        int err = 0;
        for (long r = 0; r < N - 1; ++r) {                   /* steps S_j */
#pragma omp parallel for schedule(static) reduction(+ : n_all, n_big) reduction(min : err)
            for (long k = 0; k < N / 2; ++k) {               /* disjoint pairs */
                long a, b;
                rr_pair(N, r, k, &a, &b);
                if (b >= n) continue;                        /* bordered slot */
                zc *fp = F + a * ldf, *fq = F + b * ldf;
                zc *gp = G + a * ldg, *gq = G + b * ldg;
                /* eq. 6.1 */
                double hpp = creal(jdot(m, fp, fp, J));
                double hqq = creal(jdot(m, fq, fq, J));
                zc hpq = jdot(m, fp, fq, J);
                double spp = creal(jdot(p, gp, gp, NULL));
                double sqq = creal(jdot(p, gq, gq, NULL));
                zc spq = jdot(p, gp, gq, NULL);
                zc Zp[4];
                int big;
                int rc = hzo_pivot(hpp, hqq, hpq, spp, sqq, spq, tol, crit_mode, Zp, &big);
                if (rc < 0) { if (rc < err) err = rc; continue; }
                if (rc == 0) continue;
                rot2(m, fp, fq, Zp);
                rot2(p, gp, gq, Zp);
                rot2(n, Z + a * ldz, Z + b * ldz, Zp);
                n_all += 1;
                n_big += big;
            }
            if (err < 0) { *sweeps = it; return err; }
        }
        *sweeps = it;
        if (counts) { counts[2 * (it - 1)] = n_all; counts[2 * (it - 1) + 1] = n_big; }
        if (n_big == 0) { status = 0; break; }
    }
    return status;
}

/* ---------------------------------------------------------------------- */
/* Section 6.4: the Level-2 block algorithm.                               */
/* ---------------------------------------------------------------------- */

/*
 * Section 6.4.1: split n columns into nb (even) block columns of width wb
 * or wb-1, widths non-increasing, from a prescribed maximal width w.
 * Writes the block offsets to off[0..nb] and returns nb (or -1).
 */
long hzo_partition(long n, long w, long *off, long max_nb)
{
    if (n < 2 || w < 1) return -1;
    long nb = (n + w - 1) / w;
    if (nb & 1) nb += 1;
    if (nb < 2) nb = 2;
    if (nb > n) nb = n & ~1L;
    if (nb > max_nb) return -1;
    long wb = (n + nb - 1) / nb;
    long wide = n - nb * (wb - 1);          /* blocks of width wb */
    off[0] = 0;
    for (long b = 0; b < nb; ++b) off[b + 1] = off[b] + (b < wide ? wb : wb - 1);
    return nb;
}

/* A <- Z'^* A Z' on rows and columns (a, b) of a k x k matrix (ld k). */
static void congruence2(long k, zc *A, long a, long b, const zc *Zp)
{
    rot2(k, A + a * k, A + b * k, Zp);              /* columns: A Z' */
    for (long j = 0; j < k; ++j) {                  /* rows: Z'^* (A Z') */
        zc x = A[a + j * k], y = A[b + j * k];
        A[a + j * k] = conj(Zp[0]) * x + conj(Zp[2]) * y;
        A[b + j * k] = conj(Zp[1]) * x + conj(Zp[3]) * y;
    }
}

/*
 * One block pivot (Section 6.4.2): given the kk = 2*wb slot layout of a block
 * column pair (slot s maps to column col[s], or -1 for an empty slot), form
 * H^ = F^* J F and S^ = G^* G on those columns, run inner_sweeps inner
 * sweeps of the pointwise method on the pivot pair (two-sidedly, reading
 * R8), and return the accumulated Z^ (kk x kk, column-major) in Zh.
 * Returns the number of transformations applied (*nbig: big ones), or a
 * negative error code.  For FB (inner_sweeps > 1) the inner iteration
 * stops early after an inner sweep with no transformation at all
 * (Section 6.1.7, inner levels count all transformations).
 */
static long block_pivot(long m, long p, const zc *F, long ldf, const signed char *J,
                        const zc *G, long ldg, long kk, const long *col,
                        double tol, int crit_mode, int inner_sweeps,
                        zc *Hh, zc *Sh, zc *Zh, long *nbig, int *err)
{
    *nbig = 0;
    *err = 0;
    /* H^ = F_jl^* J F_jl, S^ = G_jl^* G_jl (the ZGEMM / ZHERK of 6.4.2);
     * an empty slot borders the pivot with a zero row/column in H^ and a
     * unit diagonal entry in S^ (Section 6.3.2). */
    for (long j = 0; j < kk; ++j)
        for (long i = 0; i < kk; ++i) {
            zc h = 0.0, s = 0.0;
            if (col[i] >= 0 && col[j] >= 0) {
                h = jdot(m, F + col[i] * ldf, F + col[j] * ldf, J);
                s = jdot(p, G + col[i] * ldg, G + col[j] * ldg, NULL);
            } else if (i == j) {
                s = 1.0;
            }
            Hh[i + j * kk] = h;
            Sh[i + j * kk] = s;
            Zh[i + j * kk] = i == j ? 1.0 : 0.0;
        }
    long n_all = 0;
    for (int isw = 0; isw < inner_sweeps; ++isw) {
        long sweep_all = 0;
        for (long r = 0; r < kk - 1; ++r)
            for (long k = 0; k < kk / 2; ++k) {
                long a, b;
                rr_pair(kk, r, k, &a, &b);
                if (col[a] < 0 || col[b] < 0) continue;   /* bordered slot */
                zc Zp[4];
                int big;
                int rc = hzo_pivot(creal(Hh[a + a * kk]), creal(Hh[b + b * kk]), Hh[a + b * kk],
                                   creal(Sh[a + a * kk]), creal(Sh[b + b * kk]), Sh[a + b * kk],
                                   tol, crit_mode, Zp, &big);
                if (rc < 0) { *err = rc; return n_all; }
                if (rc == 0) continue;
                congruence2(kk, Hh, a, b, Zp);
                congruence2(kk, Sh, a, b, Zp);
                rot2(kk, Zh + a * kk, Zh + b * kk, Zp);  /* Z^ <- Z^ Z' */
                sweep_all += 1;
                *nbig += big;
            }
        n_all += sweep_all;
        if (sweep_all == 0) break;
    }
    return n_all;
}

/* X(:, col) <- X(:, col) * Zh over len rows (the block update of 6.4.3). */
static void block_update(long len, zc *X, long ldx, long kk, const long *col,
                         const zc *Zh, zc *tmp)
{
    for (long i = 0; i < len; ++i) {
        for (long j = 0; j < kk; ++j) {
            zc s = 0.0;
            for (long l = 0; l < kk; ++l)
                if (col[l] >= 0) s += X[i + col[l] * ldx] * Zh[l + j * kk];
            tmp[j] = s;
        }
        for (long j = 0; j < kk; ++j)
            if (col[j] >= 0) X[i + col[j] * ldx] = tmp[j];
    }
}

/*
 * One outer step r of the block algorithm: every block column pair (P, Q) of
 * the step (disjoint, so processed in parallel): block pivots, inner level,
 * block update.  Block column pair (P, Q) occupies slots [0, |P|) and
 * [wb, wb + |Q|) of a 2*wb slot layout, wb = the widest block.  Adds the
 * transformation counts to *n_all, *n_big; returns 0 or an error code.
 */
static int outer_step(long m, long p, long n, zc *F, long ldf, const signed char *J, zc *G,
                      long ldg, zc *Z, long ldz, const long *off, long nb, int inner_sweeps,
                      long r, double tol, int crit_mode, long *n_all_out, long *n_big_out)
{
    long wb = off[1] - off[0], kk = 2 * wb;
    long n_all = 0, n_big = 0;
    int err = 0;
#pragma omp parallel reduction(+ : n_all, n_big) reduction(min : err)
    {
        zc *Hh = malloc(sizeof(zc) * kk * kk);
        zc *Sh = malloc(sizeof(zc) * kk * kk);
        zc *Zh = malloc(sizeof(zc) * kk * kk);
        zc *tmp = malloc(sizeof(zc) * kk);
        long *col = malloc(sizeof(long) * kk);
#pragma omp for schedule(static)
        for (long k = 0; k < nb / 2; ++k) {
            long P, Q;
            rr_pair(nb, r, k, &P, &Q);
            for (long s = 0; s < kk; ++s) col[s] = -1;
            for (long c = off[P]; c < off[P + 1]; ++c) col[c - off[P]] = c;
            for (long c = off[Q]; c < off[Q + 1]; ++c) col[wb + c - off[Q]] = c;
            long nbig;
            int e;
            long na = block_pivot(m, p, F, ldf, J, G, ldg, kk, col, tol, crit_mode,
                                  inner_sweeps, Hh, Sh, Zh, &nbig, &e);
            if (e < 0) { if (e < err) err = e; continue; }
            n_all += na;
            n_big += nbig;
            if (na == 0) continue;             /* Z^ = I: copy only (6.4.3) */
            block_update(m, F, ldf, kk, col, Zh, tmp);
            block_update(p, G, ldg, kk, col, Zh, tmp);
            block_update(n, Z, ldz, kk, col, Zh, tmp);
        }
        free(Hh); free(Sh); free(Zh); free(tmp); free(col);
    }
    *n_all_out += n_all;
    *n_big_out += n_big;
    return err;
}

/*
 * The Level-2 block HZ (Section 6.4).  Arguments as for hzo_pointwise, plus
 * the prescribed maximal block width w and the number of inner sweeps per
 * block pivot (1 = BO, up to 30 = FB).  Returns as hzo_pointwise.
 */
int hzo_blocked(long m, long p, long n, zc *F, long ldf, const signed char *J,
                zc *G, long ldg, zc *Z, long ldz, long w, int inner_sweeps,
                int max_sweeps, int crit_mode, int nthreads, long *sweeps, long *counts)
{
    if (m < 1 || p < 1 || n < 1 || ldf < m || ldg < p || ldz < n || w < 1 || inner_sweeps < 1)
        return HZO_ERR_ARG;
    *sweeps = 0;
    if (n == 1) return 0;
    long *off = malloc(sizeof(long) * (n + 2));
    long nb = hzo_partition(n, w, off, n + 1);
    if (nb < 2) { free(off); return HZO_ERR_ARG; }
    double tol = eps_sqrt_n(n);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int status = 1;
    int err = 0;
    for (int it = 1; it <= max_sweeps && err == 0; ++it) {
        long n_all = 0, n_big = 0;
        for (long r = 0; r < nb - 1 && err == 0; ++r)
            err = outer_step(m, p, n, F, ldf, J, G, ldg, Z, ldz, off, nb, inner_sweeps, r, tol,
                             crit_mode, &n_all, &n_big);
        *sweeps = it;
        if (counts) { counts[2 * (it - 1)] = n_all; counts[2 * (it - 1) + 1] = n_big; }
        if (err < 0) break;
        if (n_big == 0) { status = 0; break; }
    }
    free(off);
    return err < 0 ? err : status;
}

/*
 * One outer step r (0 <= r < nb - 1) of hzo_blocked on its own, for
 * step-level checks and for timing.  Returns the number of transformations
 * applied (big ones in *nbig) or a negative error code.
 */
long hzo_blocked_step(long m, long p, long n, zc *F, long ldf, const signed char *J,
                      zc *G, long ldg, zc *Z, long ldz, long w, int inner_sweeps,
                      long r, int crit_mode, int nthreads, long *nbig_out)
{
    long *off = malloc(sizeof(long) * (n + 2));
    long nb = hzo_partition(n, w, off, n + 1);
    if (nb < 2 || r < 0 || r >= nb - 1) { free(off); return HZO_ERR_ARG; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    long n_all = 0, n_big = 0;
    int err = outer_step(m, p, n, F, ldf, J, G, ldg, Z, ldz, off, nb, inner_sweeps, r,
                         eps_sqrt_n(n), crit_mode, &n_all, &n_big);
    free(off);
    if (nbig_out) *nbig_out = n_big;
    return err < 0 ? err : n_all;
}

/*
 * The H^, S^ block pivots and the inner-level Z^ of block pair k of outer
 * step r, without updating F, G (for kernel-level parity checks).
 * Hh, Sh, Zh: kk x kk column-major, kk = 2 * widest block.  Returns kk, or
 * a negative error code; *n_all and *nbig receive the transformation counts.
 */
long hzo_block_pivot(long m, long p, long n, const zc *F, long ldf, const signed char *J,
                     const zc *G, long ldg, long w, int inner_sweeps, long r, long k,
                     int crit_mode, zc *Hh, zc *Sh, zc *Zh, zc *H0, zc *S0,
                     long *n_all, long *nbig)
{
    long *off = malloc(sizeof(long) * (n + 2));
    long nb = hzo_partition(n, w, off, n + 1);
    if (nb < 2 || r < 0 || r >= nb - 1 || k < 0 || k >= nb / 2) { free(off); return HZO_ERR_ARG; }
    long wb = off[1] - off[0], kk = 2 * wb;
    long *col = malloc(sizeof(long) * kk);
    long P, Q;
    rr_pair(nb, r, k, &P, &Q);
    for (long s = 0; s < kk; ++s) col[s] = -1;
    for (long c = off[P]; c < off[P + 1]; ++c) col[c - off[P]] = c;
    for (long c = off[Q]; c < off[Q + 1]; ++c) col[wb + c - off[Q]] = c;
    int e;
    if (H0 && S0) {   /* the block pivots as formed, before the inner level */
        long dummy;
        block_pivot(m, p, F, ldf, J, G, ldg, kk, col, eps_sqrt_n(n), crit_mode, 0,
                    H0, S0, Zh, &dummy, &e);
    }
    *n_all = block_pivot(m, p, F, ldf, J, G, ldg, kk, col, eps_sqrt_n(n), crit_mode,
                         inner_sweeps, Hh, Sh, Zh, nbig, &e);
    free(col); free(off);
    return e < 0 ? e : kk;
}

/* ---------------------------------------------------------------------- */
/* Section 6.1.7 outputs and eq. 3.2.                                       */
/* ---------------------------------------------------------------------- */

/*
 * lambda_j = (f_j^* J f_j) / (g_j^* g_j)  (= diag(Lambda_G^{-1} Lambda_F),
 * eq. 3.2, signs from J through f_j^* J f_j), and, when V != NULL,
 * V = Z' diag(1 / ||g_j||), the S-orthonormal generalized eigenvectors
 * (V^* S V = I, V^* H V = diag(lambda)).  Also returns, when sf/sg are not
 * NULL, Sigma_F' = |f_j^* J f_j|^{1/2} and Sigma_G' = ||g_j||.
 */
int hzo_finalize(long m, long p, long n, const zc *F, long ldf, const signed char *J,
                 const zc *G, long ldg, const zc *Z, long ldz, double *lambda,
                 zc *V, long ldv, double *sf, double *sg)
{
    for (long j = 0; j < n; ++j) {
        double hf = creal(jdot(m, F + j * ldf, F + j * ldf, J));
        double gg = creal(jdot(p, G + j * ldg, G + j * ldg, NULL));
        if (!(gg > 0.0)) return HZO_ERR_RANK;
        lambda[j] = hf / gg;
        if (sf) sf[j] = sqrt(fabs(hf));
        if (sg) sg[j] = sqrt(gg);
        if (V) {
            double sc = 1.0 / sqrt(gg);
            for (long i = 0; i < n; ++i) V[i + j * ldv] = Z[i + j * ldz] * sc;
        }
    }
    return 0;
}

/* The round-robin table itself, for checking the strategy definition. */
void hzo_rr_table(long N, long *pairs /* (N-1) x (N/2) x 2 */)
{
    for (long r = 0; r < N - 1; ++r)
        for (long k = 0; k < N / 2; ++k)
            rr_pair(N, r, k, &pairs[2 * (r * (N / 2) + k)], &pairs[2 * (r * (N / 2) + k) + 1]);
}

int hzo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* hzo_pivot with the pivot entries packed as
 * in = {hpp, hqq, re hpq, im hpq, spp, sqq, re spq, im spq}. */
int hzo_pivot2(const double *in, double tol, int crit_mode, zc *Zp, int *big)
{
    return hzo_pivot(in[0], in[1], in[2] + I * in[3], in[4], in[5], in[6] + I * in[7],
                     tol, crit_mode, Zp, big);
}

/*
 * Numerical rank check of G after the iteration (reading of Section 6.4.2,
 * which stops on a rank-deficient block pivot; with the pivots transformed
 * two-sidedly a dependent G need not show up in any 2x2 pivot, so it is
 * detected at the end): G V has orthonormal columns, hence
 * kappa_est = ||G||_F max_j ||v_j|| estimates cond(G) within a factor sqrt(n).
 * Returns HZO_ERR_RANK if kappa_est > 1 / (8 eps sqrt(n)), eps = 2^-53.
 */
int hzo_rank_check(long p, long n, const zc *G0, long ldg, const zc *V, long ldv, double *kappa)
{
    double g2 = 0.0, vmax = 0.0;
    for (long j = 0; j < n; ++j) {
        g2 += creal(jdot(p, G0 + j * ldg, G0 + j * ldg, NULL));
        double v2 = creal(jdot(n, V + j * ldv, V + j * ldv, NULL));
        if (v2 > vmax) vmax = v2;
    }
    double k = sqrt(g2) * sqrt(vmax);
    if (kappa) *kappa = k;
    return (!(k <= 0.125 / (ldexp(1.0, -53) * sqrt((double)n)))) ? HZO_ERR_RANK : 0;
}
