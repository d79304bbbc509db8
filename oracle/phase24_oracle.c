/*
 * phase24_oracle.c -- plain FP64 CPU oracle for the phases around the
 * Hari-Zimmermann iteration in arXiv 1907.08560: Phase 2 (Section 5, the
 * optional (J, I) URV shortening of the tall factors) and Phase 4 (Section 7,
 * X = Z^{-1} for the full GHSVD).
 *
 * TEST INFRASTRUCTURE ONLY.  Like hz_oracle.c this file is the independent
 * checker of the CUDA path: only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it, and it shares nothing with
 * the GPU library.
 *
 *   - p24_jqr:    the hyperbolic QR of F~ with the diagonal pivoting and the
 *                 Bunch-Kaufman partial pivoting of Section 5.2 (alpha =
 *                 (1 + sqrt 17) / 8), row pivoting by the sign of the pivot's
 *                 J-norm, hyperbolic Householder reflectors H(s) = I + tau s
 *                 s^* J_k of Theorem 5.1 / Section 5.3, and 2x2 pivots through
 *                 a Jacobi rotation R_k, two reflectors and R_k^* (Section 5.3).
 *   - p24_qr:     the Householder QR of G~ P2 (the tall-and-skinny QR of
 *                 Section 5, without row pivoting).
 *   - p24_lu_complete / p24_inverse: Z = P^T L U Q^T by Gaussian elimination
 *                 with complete pivoting and X = Z^{-1} by solving Z X = I
 *                 (Section 7).
 *
 * Readings (repeated in the design notes):
 *   R10 the J_k-norm that fixes a reflector is the one of the column as it
 *       stands (after the Jacobi rotation, for a 2x2 pivot), computed
 *       directly; in exact arithmetic it is the d_k of Section 5.3.
 *   R11 ties in every pivot search go to the smallest index (the paper says
 *       "the smallest index" for the column searches; the same is used for
 *       the row search by |f_l1| and, column-major, for complete pivoting).
 *   R12 a single pivot whose J_k-norm is zero is a breakdown unless its
 *       column is zero (then nothing is done); so is a row search that finds
 *       no sign equal to the sign of the pivot's J_k-norm.
 *   R13 the entry (k, k+1) left by the first reflector of a 2x2 pivot (zero
 *       in exact arithmetic) is kept as computed, then the 2x2 block is
 *       multiplied by R_k^*.
 *   R14 complete pivoting does not perturb small pivots (LAPACK's ZGETC2
 *       does); an exactly zero pivot is reported as singular.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex zc;

#define P24_OK 0
#define P24_ERR_ARG -1
#define P24_ERR_BREAKDOWN -4
#define P24_ERR_SINGULAR -5

/* sum_{i=k}^{m-1} conj(a_i) J_i b_i  (the J_k-dot product of Section 5.1) */
static zc jdot_k(long k, long m, const zc *a, const zc *b, const signed char *J)
{
    zc s = 0.0;
    for (long i = k; i < m; ++i) s += (double)J[i] * (conj(a[i]) * b[i]);
    return s;
}

static double jnorm2_k(long k, long m, const zc *a, const signed char *J)
{
    double s = 0.0;
    for (long i = k; i < m; ++i) s += (double)J[i] * (creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]));
    return s;
}

static void swap_cols(long m, zc *F, long ldf, long a, long b)
{
    if (a == b) return;
    for (long i = 0; i < m; ++i) {
        zc t = F[i + ldf * a];
        F[i + ldf * a] = F[i + ldf * b];
        F[i + ldf * b] = t;
    }
}

static void swap_rows(long n, zc *F, long ldf, long a, long b)
{
    if (a == b) return;
    for (long j = 0; j < n; ++j) {
        zc t = F[a + ldf * j];
        F[a + ldf * j] = F[b + ldf * j];
        F[b + ldf * j] = t;
    }
}

/*
 * One hyperbolic Householder step on column k (rows k..m-1) of F: bring a row
 * whose sign in J equals sgn(f^* J_k f) to position k if needed, then map the
 * column to -c1 e_k with c1 = |f^* J_k f|^{1/2} f_kk / |f_kk| (Section 5.3)
 * and apply the same reflector to the columns first..n-1 (first > k).
 */
static int reflect(long m, long n, zc *F, long ldf, signed char *J, long k, long first,
                   zc *s /* m */)
{
    zc *f = F + ldf * k;
    const double h = jnorm2_k(k, m, f, J);
    if (h == 0.0) {
        for (long i = k; i < m; ++i)
            if (f[i] != 0.0) return P24_ERR_BREAKDOWN;
        return P24_OK;                                    /* zero column: nothing to do */
    }
    const int sg = h > 0.0 ? 1 : -1;
    if (J[k] != sg) {                                     /* row pivoting */
        long l = -1;
        double best = -1.0;
        for (long i = k + 1; i < m; ++i)
            if (J[i] == sg && cabs(f[i]) > best) { best = cabs(f[i]); l = i; }
        if (l < 0) return P24_ERR_BREAKDOWN;
        swap_rows(n, F, ldf, k, l);
        signed char t = J[k]; J[k] = J[l]; J[l] = t;
    }
    const double r1 = cabs(f[k]);
    const zc eid = r1 > 0.0 ? f[k] / r1 : 1.0;
    const double rh = sqrt(fabs(h));
    const zc c1 = rh * eid;
    const double tau = -1.0 / (h + rh * r1 * (double)J[k]);
    for (long i = k; i < m; ++i) s[i] = f[i];
    s[k] += c1;
    for (long j = first; j < n; ++j) {
        zc *g = F + ldf * j;
        const zc t = tau * jdot_k(k, m, s, g, J);
        for (long i = k; i < m; ++i) g[i] += t * s[i];
    }
    f[k] = -c1;
    for (long i = k + 1; i < m; ++i) f[i] = 0.0;
    return P24_OK;
}

/*
 * The hyperbolic QR (JQR) of Section 5, in place.  On return rows 0..n-1 of F
 * hold the block upper triangular factor (diagonal blocks of order 1 or 2,
 * zeros below set explicitly), J holds the row-permuted signature (its
 * leading n entries are the shortened J), perm[j] is the original index of
 * column j (the permutation P2), and *n2x2 counts the 2x2 pivots.
 * Requires m >= n.  Returns P24_OK or P24_ERR_BREAKDOWN (reading R12).
 */
int p24_jqr(long m, long n, zc *F, long ldf, signed char *J, long *perm, long *n2x2)
{
    if (m < n || n < 1 || ldf < m) return P24_ERR_ARG;
    const double alpha = (1.0 + sqrt(17.0)) / 8.0;
    double *h = (double *)malloc(sizeof(double) * n);
    double *mag = (double *)malloc(sizeof(double) * n);
    zc *s = (zc *)malloc(sizeof(zc) * m);
    int rc = P24_OK;
    for (long j = 0; j < n; ++j) perm[j] = j;
    *n2x2 = 0;
    long k = 0;
    while (k < n && rc == P24_OK) {
        /* diagonal pivoting: the column of the largest |h_ii^[k]| */
        for (long i = k; i < n; ++i) h[i] = jnorm2_k(k, m, F + ldf * i, J);
        long jmax = k;
        for (long i = k + 1; i < n; ++i)
            if (fabs(h[i]) > fabs(h[jmax])) jmax = i;
        if (jmax != k) {
            swap_cols(m, F, ldf, k, jmax);
            long t = perm[k]; perm[k] = perm[jmax]; perm[jmax] = t;
            double th = h[k]; h[k] = h[jmax]; h[jmax] = th;
        }
        int two = 0;
        if (k < n - 1) {
            /* partial pivoting (Bunch-Kaufman): h_1j^[k] for j > k */
            long ii = k + 1;
            for (long j = k + 1; j < n; ++j) {
                mag[j] = cabs(jdot_k(k, m, F + ldf * k, F + ldf * j, J));
                if (mag[j] > mag[ii]) ii = j;
            }
            const double lam = mag[ii];
            if (!(fabs(h[k]) >= alpha * lam)) {
                /* sigma = max_{l != i} |h_il^[k]| */
                double sig = 0.0;
                for (long l = k; l < n; ++l) {
                    if (l == ii) continue;
                    const double v = cabs(jdot_k(k, m, F + ldf * ii, F + ldf * l, J));
                    if (v > sig) sig = v;
                }
                if (fabs(h[k]) * sig >= alpha * lam * lam) {
                    /* single pivot: column k */
                } else if (fabs(h[ii]) >= alpha * sig) {
                    swap_cols(m, F, ldf, k, ii);
                    long t = perm[k]; perm[k] = perm[ii]; perm[ii] = t;
                    double th = h[k]; h[k] = h[ii]; h[ii] = th;
                } else {
                    two = 1;
                    if (ii != k + 1) {
                        swap_cols(m, F, ldf, k + 1, ii);
                        long t = perm[k + 1]; perm[k + 1] = perm[ii]; perm[ii] = t;
                        double th = h[k + 1]; h[k + 1] = h[ii]; h[ii] = th;
                    }
                }
            }
        }
        if (!two) {
            rc = reflect(m, n, F, ldf, J, k, k + 1, s);
            k += 1;
            continue;
        }
        /* 2x2 pivot: A12 = [f1 f2]^* J_k [f1 f2], diagonalized by a Jacobi rotation */
        zc *f1 = F + ldf * k, *f2 = F + ldf * (k + 1);
        const double a11 = jnorm2_k(k, m, f1, J), a22 = jnorm2_k(k, m, f2, J);
        const zc a12 = jdot_k(k, m, f1, f2, J);
        const double b = cabs(a12);
        const zc eth = b > 0.0 ? a12 / b : 1.0;         /* a12 = b e^{i theta} */
        double c = 1.0, sn = 0.0;
        if (b > 0.0) {
            const double zeta = (a22 - a11) / (2.0 * b);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
        }
        /* R = diag(1, conj(e^{i theta})) [c s; -s c]:
         *   R = [c, s; -s conj(eth), c conj(eth)] */
        const zc R11 = c, R12 = sn, R21 = -sn * conj(eth), R22 = c * conj(eth);
        for (long i = k; i < m; ++i) {
            const zc x = f1[i], y = f2[i];
            f1[i] = x * R11 + y * R21;
            f2[i] = x * R12 + y * R22;
        }
        rc = reflect(m, n, F, ldf, J, k, k + 1, s);
        if (rc == P24_OK) rc = reflect(m, n, F, ldf, J, k + 1, k + 2, s);
        if (rc == P24_OK) {
            /* multiply the 2x2 block (rows k, k+1) by R^* */
            for (long i = k; i < k + 2; ++i) {
                const zc x = f1[i], y = f2[i];
                f1[i] = x * conj(R11) + y * conj(R12);
                f2[i] = x * conj(R21) + y * conj(R22);
            }
        }
        *n2x2 += 1;
        k += 2;
    }
    free(h); free(mag); free(s);
    return rc;
}

/*
 * Householder QR of the p x n matrix G (p >= n), in place: rows 0..n-1 of G
 * become R (upper triangular, zeros below set explicitly).  Each reflector
 * H = I - beta v v^* maps the column x to alpha e_k, alpha = -x_k/|x_k| ||x||
 * (alpha = -||x|| when x_k = 0).
 */
int p24_qr(long p, long n, zc *G, long ldg)
{
    if (p < n || n < 1 || ldg < p) return P24_ERR_ARG;
    zc *v = (zc *)malloc(sizeof(zc) * p);
    for (long k = 0; k < n; ++k) {
        zc *x = G + ldg * k;
        double nrm2 = 0.0;
        for (long i = k; i < p; ++i) nrm2 += creal(x[i]) * creal(x[i]) + cimag(x[i]) * cimag(x[i]);
        const double nrm = sqrt(nrm2);
        if (nrm == 0.0) continue;
        const double ax = cabs(x[k]);
        const zc ph = ax > 0.0 ? x[k] / ax : 1.0;
        const zc alpha = -ph * nrm;
        for (long i = k; i < p; ++i) v[i] = x[i];
        v[k] -= alpha;                                   /* = ph (|x_k| + ||x||) */
        const double beta = 1.0 / (nrm * (nrm + ax));    /* 2 / (v^* v) */
        for (long j = k + 1; j < n; ++j) {
            zc *g = G + ldg * j;
            zc d = 0.0;
            for (long i = k; i < p; ++i) d += conj(v[i]) * g[i];
            const zc t = beta * d;
            for (long i = k; i < p; ++i) g[i] -= t * v[i];
        }
        x[k] = alpha;
        for (long i = k + 1; i < p; ++i) x[i] = 0.0;
    }
    free(v);
    return P24_OK;
}

/*
 * Gaussian elimination with complete pivoting, in place (Section 7):
 * P A Q = L U with L unit lower triangular (below the diagonal of A) and U
 * upper triangular (on and above it).  rowp[k] / colp[k] record the row and
 * column exchanged with k at step k.  Returns P24_OK or P24_ERR_SINGULAR.
 */
int p24_lu_complete(long n, zc *A, long lda, long *rowp, long *colp)
{
    if (n < 1 || lda < n) return P24_ERR_ARG;
    for (long k = 0; k < n; ++k) {
        long pi = k, pj = k;
        double best = -1.0;
        for (long j = k; j < n; ++j)
            for (long i = k; i < n; ++i)
                if (cabs(A[i + lda * j]) > best) { best = cabs(A[i + lda * j]); pi = i; pj = j; }
        rowp[k] = pi;
        colp[k] = pj;
        swap_rows(n, A, lda, k, pi);
        swap_cols(n, A, lda, k, pj);
        const zc piv = A[k + lda * k];
        if (piv == 0.0) return P24_ERR_SINGULAR;
        for (long i = k + 1; i < n; ++i) A[i + lda * k] /= piv;
        for (long j = k + 1; j < n; ++j) {
            const zc u = A[k + lda * j];
            for (long i = k + 1; i < n; ++i) A[i + lda * j] -= A[i + lda * k] * u;
        }
    }
    return P24_OK;
}

/*
 * X = Z^{-1} from the factors of p24_lu_complete: with P Z Q = L U,
 * X = Q U^{-1} L^{-1} P.  Solves Z X = I column by column.
 */
int p24_inverse(long n, const zc *LU, long lda, const long *rowp, const long *colp, zc *X,
                long ldx)
{
    if (n < 1 || lda < n || ldx < n) return P24_ERR_ARG;
    for (long c = 0; c < n; ++c) {
        zc *x = X + ldx * c;
        for (long i = 0; i < n; ++i) x[i] = (i == c) ? 1.0 : 0.0;
        for (long k = 0; k < n; ++k) {                   /* x <- P x */
            zc t = x[k]; x[k] = x[rowp[k]]; x[rowp[k]] = t;
        }
        for (long k = 0; k < n; ++k)                     /* L y = P e_c */
            for (long i = k + 1; i < n; ++i) x[i] -= LU[i + lda * k] * x[k];
        for (long k = n - 1; k >= 0; --k) {              /* U w = y */
            x[k] /= LU[k + lda * k];
            for (long i = 0; i < k; ++i) x[i] -= LU[i + lda * k] * x[k];
        }
        for (long k = n - 1; k >= 0; --k) {              /* x <- Q w */
            zc t = x[k]; x[k] = x[colp[k]]; x[colp[k]] = t;
        }
    }
    return P24_OK;
}
