/*
 * ghsvd.h -- C ABI of the GB300 (sm_103a) implicit one-sided Hari-Zimmermann
 * solver for the generalized hyperbolic SVD (GHSVD) of a complex pair (F, G)
 * under a signature J (Singer, Di Napoli, Novakovic, Caklovic, "The LAPW
 * method with eigendecomposition based on the Hari-Zimmermann generalized
 * hyperbolic SVD", arXiv 1907.08560).
 *
 * Given F (m x n, m >= n), J = diag(+-1) (m x m) and G (p x n) of full column
 * rank (hence p >= n), the solver computes the generalized eigenvalues and
 * S-orthonormal eigenvectors of the definite pencil (H, S) = (F^* J F, G^* G)
 * (Section 3, Definition 3.1 and eq. 3.2) without forming H or S and without
 * a Cholesky factorization: block column pairs of F and G are transformed in
 * place by the Level-2 block HZ method of Section 6.4 until no "big"
 * transformation remains (Section 6.1.7).
 *
 * Around that iteration: a mixed-precision schedule (GHSVD_PRECISION_MIXED),
 * batched solves of uneven pencils (ghsvd_solve_batched), a learned warm start
 * (ghsvd_mlp_*, ghsvd_s_orthonormalize, ghsvd_solve_from), Phase 2 of the
 * paper (ghsvd_urv, opts.shorten), Phase 4 (ghsvd_inverse, ghsvd_phase4,
 * ghsvd_decomposition_errors) and a solve that allocates nothing
 * (ghsvd_solve_noalloc).
 *
 * Conventions shared by every entry point:
 *   - complex numbers are complex128 (two doubles, real part first);
 *     matrices are column-major with a leading dimension ld >= rows;
 *   - "device" pointers are CUDA device memory of the handle's device,
 *     "host" pointers are ordinary (pageable or pinned) host memory;
 *   - inputs are caller-owned and never modified; outputs are
 *     caller-allocated; the library owns only its working buffers, which it
 *     allocates on the first solve and reuses while the sizes fit;
 *   - every call is ordered on the given CUDA stream (NULL: the legacy
 *     default stream) and returns only after the result is complete, since
 *     the sweep loop reads the transformation counters on the host once per
 *     sweep;
 *   - no C++ exception crosses this boundary; every failure is a status.
 */
#ifndef GHSVD_H
#define GHSVD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ghsvd_ctx *ghsvd_t;

typedef enum {
    GHSVD_OK = 0,
    GHSVD_ERR_INVALID_ARG = 1,     /* bad size, ld, pointer or J entry          */
    GHSVD_ERR_RANK_DEFICIENT = 2,  /* a pivot of G numerically dependent (x >= 1
                                      or g_j^* g_j <= 0), Section 6.4.2       */
    GHSVD_ERR_NONFINITE = 3,       /* NaN/Inf in the inputs or the iteration    */
    GHSVD_ERR_NOT_CONVERGED = 4,   /* max_sweeps reached; outputs still written */
    GHSVD_ERR_CUDA = 5,            /* a CUDA runtime error                      */
    GHSVD_ERR_NOMEM = 6,           /* device allocation failed                  */
    GHSVD_ERR_SCRATCH_TOO_SMALL = 7, /* ghsvd_solve_noalloc: the problem does not
                                      fit GHSVD_NOALLOC_SCRATCH_BYTES          */
    GHSVD_ERR_BREAKDOWN = 8,       /* Phase 2: the hyperbolic QR met a J-isotropic
                                      nonzero pivot column, or no row whose sign
                                      matches its J-norm (Section 5.3)        */
    GHSVD_ERR_TIMEOUT = 9          /* opts.timeout_ms passed; outputs written  */
} ghsvd_status;

/* Orderings of the pivot pairs (Section 6.3).  The paper cites the MM and ME
 * parallel orderings without defining them; the round-robin (circle) ordering
 * is a parallel cyclic strategy in the paper's sense and is the one built. */
#define GHSVD_ORDER_ROUND_ROBIN 0

/* Precision schedules. */
#define GHSVD_PRECISION_FP64 0     /* every sweep in complex128 / FP64            */
#define GHSVD_PRECISION_MIXED 1    /* rounds of complex64 preconditioning sweeps
                                      with FP32 accumulation, each applied to the
                                      FP64 factors by an FP64 product, then FP64
                                      finishing sweeps; the 2x2 parameters,
                                      J-norms and the stopping test are FP64  */

typedef struct {
    int block_width;     /* w: maximal block-column width, 1..32 (Section 6.4.1);
                            default 32; 0: automatic (32 for one pencil, the
                            autotuner for ghsvd_solve_batched)                */
    int inner_sweeps;    /* inner sweeps per block pivot: 1 = BO (default),
                            up to 30 = FB (Section 6.4.2)                     */
    int max_sweeps;      /* C_max for the outer (block) sweeps, default 30
                            (Algorithm 1)                                      */
    int crit_mode;       /* eq. 6.12 reading: 0 = |h_pq| >= sqrt(max) eps
                            sqrt(n) sqrt(min) (default), 1 = as printed       */
    int precision;       /* GHSVD_PRECISION_FP64 (default) or _MIXED           */
    int mixed_max_sweeps;/* at most this many complex64 sweeps (default 24);
                            they count toward max_sweeps.  The two rounds end
                            where their big count levels off: 36 + 12 sweeps
                            for the n = 2048 benchmark pencil, which is solved
                            with 60 and max_sweeps 80                         */
    int sort_ascending;  /* 1: sort lambda ascending and permute V alike;
                            0 (default): column order of the iteration, as in
                            the paper (Section 3)                              */
    int gram_chunk;      /* rows per Gram work unit; 0 = automatic            */
    int timing;          /* 1: time every step kernel with CUDA events on the
                            solve's stream (ghsvd_stats.ms_*); 0 (default): off */
    int ordering;        /* GHSVD_ORDER_ROUND_ROBIN (default; the only one)    */
    double tol_scale;    /* multiplies eps sqrt(n) in eq. 6.12 (default 1.0,
                            > 0; larger values stop earlier, less accurately) */
    int64_t timeout_ms;  /* > 0: stop after the sweep in which this wall time
                            (from the start of the solve) passes and return
                            GHSVD_ERR_TIMEOUT with the outputs of the current
                            factors; 0 (default): no limit                     */
    int mixed_param32;   /* GHSVD_PRECISION_MIXED: 0 (default) computes the 2x2
                            parameters of the complex64 sweeps in FP64, as the
                            method prescribes; 1 computes them in FP32 and
                            counts a rotation as big by the FP64 test
                            (sin phi or sin psi >= 2^-27): faster, the same
                            rounds and accuracy on the benchmark pencils     */
    int shorten;         /* 1: Phase 2 first (Section 5, see ghsvd_urv): the
                            iteration runs on the square factors; lambda is
                            that of the tall pencil and V is returned in the
                            caller's column order (rows permuted back by P2).
                            Not with a warm start.  0 (default): the tall
                            factors.  ghsvd_solve_batched ignores it (and
                            timeout_ms; it uses tol_scale);
                            ghsvd_solve_noalloc rejects shorten = 1 and
                            honours timeout_ms.                                */
    int mixed_tc;        /* GHSVD_PRECISION_MIXED: 1 (default) runs the Grams
                            of the complex64 sweeps on the tensor cores
                            (tcgen05, TF32 operands split into high and low
                            parts, three products per real product, FP32
                            accumulation) and the block update of every pair
                            whose Z^ - I is small (all entries <= 1/2) there
                            too, in the delta form X + X (Z^ - I); pairs with
                            larger rotations are updated on the FP32 CUDA
                            cores.  0: Grams and updates on the CUDA cores.
                            The 2x2 parameters, J-norms and stopping test are
                            FP64 either way.                                  */
    int delta_update;    /* FP64 sweeps: 1 (default) updates every pair whose
                            Z^ - I is small in the delta form X + X (Z^ - I),
                            the sum in FP64: with all entries <= 2^-29 the
                            product from FP32 roundings by FP32 FMAs (error
                            bound about 2^-47 sum_l |x_il| per entry; typical
                            error that of the FP64 product), with all entries
                            <= 2^-11 in double-float arithmetic (FP32 pairs, 48
                            significant bits; bound about 2^-52 sum_l |x_il|;
                            for a row of comparable entries its typical error
                            is far below the FP64 product's).
                            The other pairs, and every pair with 0, by the FP64
                            product                                           */
} ghsvd_opts;

/* Per-solve statistics (Section 6.4.3, "Completing a sweep"). */
typedef struct {
    int sweeps;                    /* outer sweeps run (all precisions)          */
    int sweeps_low;                /* of which complex64 (mixed schedule)        */
    int steps_per_sweep;           /* outer round-robin steps per sweep          */
    int pairs_per_step;            /* block column pairs per step                */
    int block_width;               /* widest block column actually used          */
    long long transforms[64];      /* all transformations, per sweep (first 64)  */
    long long big[64];             /* big transformations, per sweep             */
    double ms_total;               /* wall time of the last solve, ms            */
    long long kernel_launches;     /* kernels this library launched in the solve */
    long long launches_gram, launches_inner, launches_update;
    double ms_gram, ms_inner, ms_update;   /* summed device time (timing = 1)     */
    int rounds_low;                /* complex64 rounds (mixed schedule)          */
    double ms_phase2;              /* wall time of Phase 2 in the solve (shorten) */
    int n2x2;                      /* 2x2 pivots of that Phase 2                 */
    int sweeps_tc;                 /* complex64 sweeps run on the tensor cores   */
    long long batch_ticks;         /* ghsvd_solve_batched: ticks (one outer step
                                      of every active pencil) run on the device  */
    int batch_graph_launches;      /* ghsvd_solve_batched: launches of the solve's
                                      graph (its while loop runs on the device)  */
    double ms_v0;                  /* warm starts: wall time of applying the
                                      starting bases, (F V0, G V0), ms         */
    long long pairs_delta;         /* with opts.delta_update: FP64 pair updates
                                      taken in the delta form, over the solve  */
    long long pairs_fp64;          /* with opts.delta_update: FP64 pair updates
                                      by the FP64 product, over the solve      */
    long long pairs_df;            /* with opts.delta_update: FP64 pair updates
                                      in the delta form with the product in
                                      double-float arithmetic, over the solve  */
} ghsvd_stats;

/* Fill *opts with the defaults listed above. */
ghsvd_status ghsvd_default_opts(ghsvd_opts *opts);

/* Create a solver handle on CUDA device `device` with options `opts`
 * (NULL: defaults).  Allocates nothing on the device yet.  *h receives the
 * handle, or NULL on error. */
ghsvd_status ghsvd_create(ghsvd_t *h, int device, const ghsvd_opts *opts);

/*
 * Solve H z = lambda S z for H = F^* J F, S = G^* G (eq. 3.2).
 *   m, p, n   sizes: m >= n >= 1, p >= n.
 *   F, ldf    device, complex128 m x n, ld ldf >= m; read only.
 *   J         device or host int8, m entries each +1 or -1; or NULL, in which
 *             case J = diag(+1 x n_plus, -1 x (m - n_plus)) ("positives first",
 *             Section 4.5.1); n_plus is ignored when J != NULL.
 *   G, ldg    device, complex128 p x n, ld ldg >= p; read only.
 *   lambda    device, n doubles: the generalized eigenvalues
 *             lambda_j = (f_j^* J f_j) / (g_j^* g_j) of the converged columns
 *             (Section 6.1.7), signs following J.
 *   V, ldv    device, complex128 n x n, ld ldv >= n, or NULL: the eigenvectors
 *             V = Z' diag(1 / ||g'_j||), so that V^* S V = I and
 *             V^* H V = diag(lambda) (the paper's Z up to column scaling).
 *   sweeps    host, may be NULL: number of outer sweeps run.
 *   stream    cudaStream_t (as void *), may be NULL.
 * Returns GHSVD_ERR_NOT_CONVERGED if max_sweeps was reached (outputs written),
 * GHSVD_ERR_RANK_DEFICIENT / _NONFINITE on the failures listed above
 * (outputs undefined).
 */
ghsvd_status ghsvd_solve(ghsvd_t h, int64_t m, int64_t p, int64_t n,
                         const void *F, int64_t ldf, const int8_t *J, int64_t n_plus,
                         const void *G, int64_t ldg, double *lambda, void *V, int64_t ldv,
                         int *sweeps, void *stream);

/*
 * As ghsvd_solve, but the accumulated transformation starts from V0
 * (device, complex128 n x n, ld ldv0, nonsingular) instead of I: the sweeps
 * run on (F V0, G V0) and V0 is the initial Z' (Algorithm 1 allows any
 * initial Z' such as the prescaling D).  Used for warm starts and to resume
 * from a saved V.
 */
ghsvd_status ghsvd_solve_from(ghsvd_t h, int64_t m, int64_t p, int64_t n,
                              const void *F, int64_t ldf, const int8_t *J, int64_t n_plus,
                              const void *G, int64_t ldg, const void *V0, int64_t ldv0,
                              double *lambda, void *V, int64_t ldv, int *sweeps, void *stream);

/*
 * As ghsvd_solve with every array in HOST memory (F, J, G read; lambda, V
 * written): copies in, solves, copies out.  For callers without device
 * buffers; the copies are part of the call.
 */
ghsvd_status ghsvd_solve_host(ghsvd_t h, int64_t m, int64_t p, int64_t n,
                              const void *F, int64_t ldf, const int8_t *J, int64_t n_plus,
                              const void *G, int64_t ldg, double *lambda, void *V, int64_t ldv,
                              int *sweeps, void *stream);

/*
 * After a solve: copy the transformed factors F' (m x n), G' (p x n) and the
 * accumulated Z' (n x n) into device buffers (any may be NULL).  The paper's
 * remaining outputs follow from them (Section 6.1.7): Sigma_F' and
 * Sigma_G' are the J-norms and norms of the columns, U = F' Sigma_F'^{-1},
 * and the left vectors of G are G' Sigma_G'^{-1}.
 */
ghsvd_status ghsvd_get_factors(ghsvd_t h, void *Fp, int64_t ldf, void *Gp, int64_t ldg,
                               void *Zp, int64_t ldz, void *stream);

/* Statistics of the last solve on this handle. */
ghsvd_status ghsvd_get_stats(ghsvd_t h, ghsvd_stats *stats);

/* A static, human-readable description of a status. */
const char *ghsvd_status_string(ghsvd_status s);

/* Release the handle and its device buffers (NULL is allowed). */
void ghsvd_destroy(ghsvd_t h);

/*
 * Batched solves: `batch` independent pencils (F_i, J_i, G_i) of uneven
 * orders, e.g. the k-points of one LAPW computation.  Every pencil follows
 * its own block schedule (Section 6.4.1, 6.3) and stopping rule (no big
 * transformation in its sweep, Section 6.1.7); one outer step of every
 * pencil that has not stopped runs per "tick" (a Gram, an inner and an
 * update kernel over all pencils, and a control kernel on the device).  The
 * whole iteration is one launch of a CUDA graph whose conditional while node
 * repeats the tick; the control kernel decides on the device whether another
 * tick runs (some pencil active, fewer than max_sweeps sweeps of the longest
 * schedule), so the host waits once (ghsvd_stats.batch_ticks,
 * batch_graph_launches).
 *   m, p, n       host arrays [batch]: sizes of pencil i (n_i >= 2).
 *   F, G          host arrays [batch] of device pointers (complex128,
 *                 column-major) with host arrays ldf, ldg [batch].
 *   J             host array [batch] of device int8 pointers (+-1 each), or
 *                 NULL; a NULL array or entry means positives first with
 *                 n_plus[i] leading +1 signs (n_plus NULL: J = I).
 *   V0, ldv0      host arrays [batch] of device pointers (complex128 n_i x n_i,
 *                 nonsingular) and leading dimensions, or NULL V0 / NULL
 *                 entries: the starting Z' of pencil i (as ghsvd_solve_from).
 *   lambda        host array [batch] of device pointers (n_i doubles each).
 *   V, ldv        host arrays [batch] of device pointers and leading
 *                 dimensions, or NULL V (no eigenvectors).
 *   sweeps, status  host arrays [batch] (may be NULL): sweeps run and the
 *                 status of every pencil.
 * The handle's block_width is used for every pencil; block_width = 0 picks
 * it from {8, 16, 32} by timing a few ticks of each (the autotuner); the
 * choice is reported in ghsvd_stats.block_width.
 * Precision: opts.precision FP64 or MIXED (other values: GHSVD_ERR_INVALID_ARG).
 * With MIXED every pencil without a starting basis runs the mixed schedule
 * of ghsvd_solve on its own clock: complex64 rounds (mixed_max_sweeps,
 * mixed_param32 apply; the complex64 Grams and updates run on the CUDA
 * cores, mixed_tc is not used), each ended by the FP64 product W Z'_low in
 * the next tick, then FP64 sweeps to the stopping rule; a pencil given a V0
 * starts its first round from (F V0, G V0).  ghsvd_stats.sweeps_low and
 * rounds_low are the sums over the pencils.  delta_update applies to the
 * FP64 sweeps of every pencil as in ghsvd_solve (the pairs_* statistics are
 * not kept for batched solves).
 * Returns GHSVD_OK when every pencil converged, otherwise the status of the
 * first pencil that failed (or GHSVD_ERR_NOT_CONVERGED).
 */
ghsvd_status ghsvd_solve_batched(ghsvd_t h, int batch, const int64_t *m, const int64_t *p,
                                 const int64_t *n, const void *const *F, const int64_t *ldf,
                                 const int8_t *const *J, const int64_t *n_plus,
                                 const void *const *G, const int64_t *ldg,
                                 const void *const *V0, const int64_t *ldv0,
                                 double *const *lambda, void *const *V, const int64_t *ldv,
                                 int *sweeps, int *status, void *stream);

/* ------------------------------------------------------------------------
 * Learned warm start.  The paper has no learned part; Algorithm 1 admits any
 * starting Z' (the prescaling D in the paper), and ghsvd_solve_from takes
 * one.  For a family of pencils F(t), G(t) a small MLP trained on the
 * solver's own eigenvectors predicts V0(t); ghsvd_s_orthonormalize makes it
 * S-orthonormal; the sweeps then run to the stopping rule of Section 6.1.7.
 * The array arguments of the calls below (but the parameter copies of
 * ghsvd_mlp_get / ghsvd_mlp_set, which take host or device memory) must be
 * device memory of the MLP's device, or of the current device for the calls
 * without an MLP; any other pointer returns GHSVD_ERR_INVALID_ARG before
 * anything is queued.
 * ------------------------------------------------------------------------ */
typedef struct ghsvd_mlp *ghsvd_mlp_t;

/* MLP x (n_in) -> tanh(W1 x + b1) (n_hidden) -> tanh(W2 . + b2) (n_hidden)
 * -> W3 . + b3 (n_out), FP32, parameters initialized from `seed`
 * (uniform in +-1/sqrt(fan_in), zero biases), on CUDA device `device`. */
ghsvd_status ghsvd_mlp_create(ghsvd_mlp_t *m, int device, int n_in, int n_hidden, int n_out,
                              uint64_t seed);
void ghsvd_mlp_destroy(ghsvd_mlp_t m);

/* The flat FP32 parameter vector [W1 (n_hidden x n_in, row-major), b1, W2,
 * b2, W3 (n_out x n_hidden), b3]: its length; a copy of the parameters
 * (what = 0) or of the last gradient (what = 1) into dst (host or device);
 * replacing the parameters from src (host or device). */
ghsvd_status ghsvd_mlp_size(ghsvd_mlp_t m, int64_t *count);
ghsvd_status ghsvd_mlp_get(ghsvd_mlp_t m, int what, float *dst);
ghsvd_status ghsvd_mlp_set(ghsvd_mlp_t m, const float *src);

/* Y (device, batch x n_out, row-major) = MLP(X) for X (device, batch x n_in). */
ghsvd_status ghsvd_mlp_forward(ghsvd_mlp_t m, int batch, const float *X, float *Y, void *stream);

/* loss = mean over batch x n_out of (MLP(X) - T)^2 (host out, may be NULL);
 * its gradient w.r.t. the parameters is left in the gradient vector. */
ghsvd_status ghsvd_mlp_loss_grad(ghsvd_mlp_t m, int batch, const float *X, const float *T,
                                 double *loss, void *stream);

/* Adam (beta 0.9, 0.999, eps 1e-8, learning rate lr) over `epochs` passes of
 * minibatches of `batch` consecutive samples of (X, T) (device, row-major);
 * *final_loss (may be NULL) = mean loss of the last epoch. */
ghsvd_status ghsvd_mlp_train(ghsvd_mlp_t m, int n_samples, const float *X, const float *T,
                             int epochs, int batch, float lr, double *final_loss, void *stream);

/* For each of `count` pairs: V0_i <- V0_i R_i^{-1} with
 * (G_i V0_i)^* (G_i V0_i) = R_i^* R_i (Cholesky of the n x n Gram of G_i V0_i,
 * never of S), so that V0_i^* S_i V0_i = I.  G_i is p x n, V0_i n x n,
 * complex128 column-major device arrays (host arrays of pointers and leading
 * dimensions), n <= 4096; the factorizations run one CTA per pair.
 * GHSVD_ERR_RANK_DEFICIENT if some G_i V0_i is numerically rank deficient. */
ghsvd_status ghsvd_s_orthonormalize(int count, int64_t p, int64_t n, const void *const *G,
                                    const int64_t *ldg, void *const *V0, const int64_t *ldv0,
                                    void *stream);

/* The MLP's training targets from the solver's eigenvectors V_i (device,
 * complex128 n x n column-major, phases aligned with Vref by
 * ghsvd_align_phases, columns in ascending eigenvalue order): row i of T
 * (device FP32, count x 2 n^2, row-major) = vec(V_i - Vref) as (re, im)
 * pairs in column-major order, divided by their root mean square over all
 * rows, which is returned in *rms (host, may be NULL). */
ghsvd_status ghsvd_v0_targets(int count, int64_t n, const void *Vref, int64_t ldr, const void *const *V,
                              const int64_t *ldv, float *T, double *rms, void *stream);

/* The predicted starting bases: V0_i = Vref + scale D_i, D_i the complex n x n
 * matrix (column-major (re, im) pairs) in row i of Y (device FP32,
 * count x 2 n^2, row-major: the MLP's output for parameter vector i); V0 is
 * a host array of `count` device pointers (complex128, leading dimensions
 * ldv0).  Follow with ghsvd_s_orthonormalize. */
ghsvd_status ghsvd_v0_compose(int count, int64_t n, const float *Y, double scale, const void *Vref, int64_t ldr,
                              void *const *V0, const int64_t *ldv0, void *stream);

/* V[:, j] *= conj(c_j)/|c_j|, c_j = Vref[:, j]^* V[:, j] (device, complex128,
 * n x n column-major): aligns the free phase of each eigenvector with a
 * reference set, so that eigenvectors of nearby pencils can be compared. */
ghsvd_status ghsvd_align_phases(int64_t n, const void *Vref, int64_t ldr, void *V, int64_t ldv,
                                void *stream);

/*
 * The tensor-core block operations of the complex64 sweeps (opts.mixed_tc) on
 * one block pair, for verification against a reference: the block-pivot Gram
 * of Section 6.4.2 (eq. 6.1), gram = X^* J X (J = NULL: X^* X), and the block
 * update of Section 6.4.3, X <- X Z, both by tcgen05.mma of kind::tf32 (each
 * real product as hi*hi + hi*lo + lo*hi of TF32 parts, FP32 accumulation;
 * the update in the delta form X + X (Z - I), X added in FP32).
 *   X     device, complex64 (two floats), rows x 64, column-major, ldx = rows,
 *         rows a positive multiple of 64; overwritten by X Z
 *   J     device int8, rows entries +-1, or NULL
 *   Z     device, complex64 64 x 64, column-major (ld 64); a column equal to
 *         e_j leaves column j of X exactly as it was
 *   gram  device, complex64 64 x 64, column-major, written in full (the upper
 *         part computed, the lower part its conjugate transpose)
 * Allocates its small temporaries on `stream`; returns INVALID_ARG for bad
 * sizes or for a pointer that is not device memory of the current device,
 * GHSVD_ERR_CUDA if the tensor-core path is not available or a device-side
 * wait ran out.
 */
ghsvd_status ghsvd_tc_block_ops(int64_t rows, void *X, int64_t ldx, const int8_t *J, const void *Z,
                                void *gram, void *stream);

/*
 * The block update of the FP64 sweeps (Section 6.4.3) on one block pair, by
 * one of its three routes, for verification against a reference:
 * X <- X Z (route 2: the FP64 product, three-multiplication form), or in the
 * delta form X <- X + X (Z - I) with the product in FP32 (route 0, used by
 * the solve when every entry of Z - I is at most 2^-29) or in double-float
 * arithmetic (route 1, at most 2^-11); the route is taken as given, whatever
 * the size of Z - I.
 *   X     device, complex128, rows x 64, column-major with ldx >= rows, rows a
 *         positive multiple of 64; overwritten
 *   Z     device, complex128 64 x 64, column-major (ld 64); in the delta forms
 *         a column equal to e_j leaves column j of X exactly as it was
 * Allocates its small temporaries on `stream`; returns INVALID_ARG for bad
 * sizes or route, or for a pointer that is not device memory of the current
 * device.
 */
ghsvd_status ghsvd_fp64_block_update(int64_t rows, void *X, int64_t ldx, const void *Z, int route,
                                     void *stream);

/* Size of the device array that ghsvd_solve_noalloc works in (32 MiB). */
#define GHSVD_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * The FP64 solve of ghsvd_solve without any device allocation.  The paper has
 * no counterpart: it exists for callers that cannot call cudaMalloc when they
 * solve, e.g. code running inside a host application whose memory pool has
 * already reserved the whole device, or code that by its own rules may not
 * allocate after start-up.
 *
 * All working memory (the stacked factors, Gram partials, block
 * transformations, schedule, counters) lives in one file-scope device array
 * of GHSVD_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads this
 * library holds until the process exits.  No handle is needed; the call runs
 * on the current CUDA device.  Sizes whose working set does not fit the array
 * are rejected with GHSVD_ERR_SCRATCH_TOO_SMALL (for F 1.5n x n and G 2n x n
 * the limit is about n = 640 at block width 32).
 *
 * Arguments as for ghsvd_solve, except:
 *   - F, G, lambda, V and a non-NULL J must be device memory of the current
 *     device (a host J, or memory of another device, is GHSVD_ERR_INVALID_ARG,
 *     returned before anything is queued);
 *   - opts (NULL: defaults) must ask for GHSVD_PRECISION_FP64, the round-robin
 *     ordering and shorten = 0 (Phase 2 needs working memory of its own);
 *     anything else is GHSVD_ERR_INVALID_ARG.  block_width 0 means 32;
 *     timeout_ms is honoured between sweeps as in ghsvd_solve; `timing`,
 *     `mixed_max_sweeps` and `mixed_param32` are ignored.
 * *sweeps (if non-NULL) is written on every return: 0 before the iteration,
 * else the sweeps run.  lambda and V are written on GHSVD_OK,
 * GHSVD_ERR_NOT_CONVERGED and GHSVD_ERR_TIMEOUT.
 *
 * The first call on a device looks up the array's device address and sets
 * the kernels' shared-memory limits for that device; make that first call
 * before any stream capture begins.  Every call waits on `stream` after each
 * sweep to read the sweep's counters.  Every call shares the array and clears
 * the parts that must start at zero; calls that overlap on the GPU (other
 * streams, other host threads) race on it and must be ordered by the caller.
 */
ghsvd_status ghsvd_solve_noalloc(int64_t m, int64_t p, int64_t n,
                                 const void *F, int64_t ldf, const int8_t *J, int64_t n_plus,
                                 const void *G, int64_t ldg, double *lambda, void *V, int64_t ldv,
                                 const ghsvd_opts *opts, int *sweeps, void *stream);

/*
 * Phase 2 (Section 5): the (J, I) URV shortening of the tall pencil
 * (F~, J~, G~) to a square one (F, J, G) with the same eigenvalues.
 *   P1 F~ P2 = Q_F [F; 0] by the hyperbolic QR with the diagonal and the
 *   Bunch-Kaufman partial pivoting of Section 5.2 (alpha = (1 + sqrt 17)/8),
 *   hyperbolic Householder reflectors (Theorem 5.1, Section 5.3) and 2x2
 *   pivots through a Jacobi rotation; G~ P2 = Q_G G by the Householder QR.
 *   Then P2^T F~^* J~ F~ P2 = F^* J F and P2^T G~^* G~ P2 = G^* G, so the
 *   pencils have the same eigenvalues and the eigenvectors of the tall one
 *   are Z~ = P2 Z (Section 5).
 *   m, p, n, F~/ldf, J~/n_plus, G~/ldg  as for ghsvd_solve; F~, G~ and a
 *             non-NULL J~ in device memory, read only.
 *   Fs, ldfs  device, complex128 n x n (ldfs >= n): F, block upper
 *             triangular with diagonal blocks of order 1 or 2.
 *   Js        device, n int8: J, the leading n signs of the row-permuted J~.
 *   Gs, ldgs  device, complex128 n x n (ldgs >= n): G, upper triangular.
 *   perm      device, n int64, or NULL: P2; column j of F~ P2 is column
 *             perm[j] of F~.
 *   n2x2      host, or NULL: the number of 2x2 pivots taken.
 * Allocates its workspace (16 (m + p) n bytes and O(m + p + n)) on the stream
 * and frees it before returning.  Returns GHSVD_ERR_BREAKDOWN if the
 * hyperbolic QR breaks down (outputs undefined).
 */
ghsvd_status ghsvd_urv(int64_t m, int64_t p, int64_t n, const void *F, int64_t ldf,
                       const int8_t *J, int64_t n_plus, const void *G, int64_t ldg,
                       void *Fs, int64_t ldfs, int8_t *Js, void *Gs, int64_t ldgs, int64_t *perm,
                       int *n2x2, void *stream);

/*
 * Phase 4 (Section 7): X = Z^{-1} by Gaussian elimination with complete
 * pivoting, P Z Q = L U, and the solution of Z X = I.
 *   Z, ldz    device, complex128 n x n, read only.
 *   X, ldx    device, complex128 n x n (ldx >= n).
 * n <= 12288.  Allocates its workspace (16 n^2 bytes and O(n^2 / 4096))
 * on the stream.  Returns GHSVD_ERR_RANK_DEFICIENT if a pivot is exactly
 * zero (X undefined).
 */
ghsvd_status ghsvd_inverse(int64_t n, const void *Z, int64_t ldz, void *X, int64_t ldx, void *stream);

/*
 * The full GHSVD (eq. 3.1) from the last successful ghsvd_solve on h: with
 * F', G', Z' the converged columns (Section 6.1.7),
 *   Sigma_F'_j = |f'_j^* J f'_j|^{1/2}, Sigma_G'_j = ||g'_j||,
 *   Sigma_j = (Sigma_F'_j^2 + Sigma_G'_j^2)^{1/2},
 *   Sigma_F = Sigma_F' / Sigma, Sigma_G = Sigma_G' / Sigma (so that
 *   Sigma_F^2 + Sigma_G^2 = I), Z = Z' Sigma^{-1} and X = Z^{-1} (Phase 4);
 * U = F' Sigma_F'^{-1} and V = G' Sigma_G'^{-1} are the columns that
 * ghsvd_get_factors returns, scaled.  Columns follow the iteration's order
 * (not sorted, whatever sort_ascending says).  After a shortened solve they
 * refer to the square pencil of ghsvd_urv.
 *   sigma_f, sigma_g  device, n doubles each, or NULL.
 *   X, ldx    device, complex128 n x n, or NULL.
 * Allocates its workspace on the stream.
 */
ghsvd_status ghsvd_phase4(ghsvd_t h, double *sigma_f, double *sigma_g, void *X, int64_t ldx,
                          void *stream);

/*
 * The relative errors of eq. 7.1 of the GHSVD of the last successful solve
 * on h: err_f = ||F - U Sigma_F X||_F / ||F||_F and
 * err_g = ||G - V Sigma_G X||_F / ||G||_F, with U Sigma_F X = F' Sigma^{-1} X
 * and V Sigma_G X = G' Sigma^{-1} X.
 *   F, ldf, G, ldg  device: the factors that solve was given (m x n, p x n).
 *   X, ldx    device: X from ghsvd_phase4.
 *   err_f, err_g   host.
 */
ghsvd_status ghsvd_decomposition_errors(ghsvd_t h, const void *F, int64_t ldf, const void *G,
                                        int64_t ldg, const void *X, int64_t ldx, double *err_f,
                                        double *err_g, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GHSVD_H */
