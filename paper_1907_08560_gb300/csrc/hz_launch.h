// hz_launch.h -- host-side launchers of the kernels in hz_step.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hz {

constexpr int KKMAX = 64;          // largest block pivot order 2 wb (wb <= 32)
constexpr int ROWPAD = 64;         // row padding of each range of W
constexpr int GRAM_KT = 16;        // rows staged per Gram step
constexpr int UPD_R = 64;          // rows per update tile
constexpr int UPD_LD = KKMAX + 1;  // padded row length of the update's shared tiles
constexpr int INNER_LD = KKMAX + 1;  // padded column length of the inner level's (H^, S^, Z^)

// Dynamic shared memory of an inner-level CTA: H^, S^, Z^ (elem = 16 or 8).
inline size_t inner_smem_bytes(size_t elem) { return 3 * elem * (size_t)KKMAX * INNER_LD; }

// Dynamic shared memory of an update CTA: Z^ [KKMAX][UPD_LD] and the row tile
// [UPD_R][UPD_LD] (elem = 16 for complex128, 8 for complex64); the complex128
// update also keeps the real sums Re + Im of both tiles.
inline size_t update_smem(size_t elem)
{
    return (elem == 16 ? 24 : elem) * (size_t)(KKMAX + UPD_R) * UPD_LD;
}

// Step descriptor passed by value to every step kernel.
struct StepArgs {
    const int *slotcol;     // [npairs][kk] column of each slot, -1 if empty
    int npairs;             // block column pairs in this step
    int kk;                 // block pivot order 2 wb
    int m_pad, p_pad, n_pad;
    long long ld;           // = Mt
    int kc;                 // rows per Gram chunk (multiple of GRAM_KT)
    int chunks_h, chunks_s; // Gram chunks over the F rows and the G rows
};

// Inner-level descriptor.
struct InnerArgs {
    int npairs, kk, cpp, chunks_h;
    int inner_sweeps;                  // 1 = BO, > 1 = FB
    int crit_mode;                     // eq. 6.12 reading
    double tol;                        // eps * sqrt(n)
    int param32;                       // complex64 sweeps: 2x2 parameters in FP32
};

// Threads of a complex64 Gram CTA: 16 per upper-triangular 16 x 16 tile of the kk x kk pivot.
inline int gram_threads(int kk)
{
    const int nt = (kk + 15) / 16;
    const int t = 16 * nt * (nt + 1) / 2;
    return t < 32 ? 32 : t;
}

// Threads of a complex128 Gram CTA: whole warps for the off-diagonal tiles
// (16 threads each) and one warp for the diagonal tiles; 128 at kk = 64.
inline int gram_threads_c128(int kk)
{
    const int nt = (kk + 15) / 16;
    return 32 * ((8 * nt * (nt - 1) + 31) / 32 + 1);
}

// Gram row chunk (a multiple of GRAM_KT): the chunk whose per-step CTAs
// (npairs x chunks) spread over the SMs best, time ~ waves x rows per chunk
// plus the partial sums the inner level reads; ties go to the larger chunk.
// Only chunks giving at least two CTAs per SM compete when any does: with one
// CTA per SM the loads of a staged row block are not hidden behind another
// CTA's FMAs and SMs idle (the 2048 + 2048 rows of a shortened pencil: 1024-row
// chunks, 128 CTAs, Gram 2.46 ms per step; 320-row chunks, 448 CTAs, 1.61 ms).
inline int gram_chunk_rows(int m_pad, int p_pad, int npairs, int sms)
{
    long long best_cost = -1;
    int best = 512;
    for (int pass = 0; pass < 2 && best_cost < 0; ++pass) {
        for (int kc = 128; kc <= 4096; kc += 64) {
            const long long ch = (m_pad + kc - 1) / kc + (p_pad + kc - 1) / kc;
            const long long ctas = ch * npairs;
            if (pass == 0 && ctas < 2LL * sms) continue;
            const long long waves = (ctas + sms - 1) / sms;
            const long long cost = waves * kc + ch * 8;
            if (best_cost < 0 || cost < best_cost || (cost == best_cost && kc > best)) {
                best_cost = cost;
                best = kc;
            }
        }
    }
    return best;
}

// Error flags raised by the device (bitwise or).
constexpr int DEVERR_RANK = 1;
constexpr int DEVERR_NONFINITE = 2;
constexpr int DEVERR_TIMEOUT = 4;     // a bounded device-side wait ran out

// One item of a batched FP64 product C = A B (A rows x n, B n x n, C rows x n,
// column-major); the batched copy uses A as source and C as destination.
struct GemmItem {
    const double2 *A;
    long long lda;
    long long rows;
    const double2 *B;
    long long ldb;
    double2 *C;
    long long ldc;
    int n;
    int accurate;       // 1: compensated sums (error-free products and sums), 0: plain FP64
};

cudaError_t setup_kernels();
cudaError_t launch_gemm_batched(const GemmItem *items, int count, long long max_rows, int max_n,
                                cudaStream_t s);
cudaError_t launch_copy_batched(const GemmItem *items, int count, cudaStream_t s);
cudaError_t launch_v0_kappa(const GemmItem *items, int count, double *kappa, cudaStream_t s);

// A warm-start basis whose estimated condition relative to G exceeds this is
// applied with compensated sums (see gemm_batched_kernel).
constexpr double WARM_ACCURATE_KAPPA = 100.0;
cudaError_t launch_copyin(void *W, bool single, long long ld, int m, int p, int n, int m_pad,
                          int p_pad, int n_pad, const void *F, long long ldf, const void *G,
                          long long ldg, const void *V0, long long ldv0, int *err, cudaStream_t s);
cudaError_t launch_signs(int8_t *Jrow, const int8_t *J, int m, int m_pad, long long n_plus, int *bad,
                         cudaStream_t s);
cudaError_t launch_convert(void *dst, bool dst_single, const void *src, long long count, cudaStream_t s);
cudaError_t launch_gram(const void *W, bool single, const int8_t *Jrow, const StepArgs &a,
                        void *partial, cudaStream_t s);
// zhat: npairs x KKMAX^2 transformations Z^, complex128 for the FP64 sweeps and
// complex64 (in the same storage) for the complex64 sweeps (single).
cudaError_t launch_inner(const void *partial, bool single, const int *slotcol, const InnerArgs &a,
                         double2 *zhat, int *pair_flag, unsigned long long *counters, int *err,
                         cudaStream_t s);
cudaError_t launch_update(void *W, bool single, const StepArgs &a, const double2 *zhat,
                          const int *pair_flag, cudaStream_t s);
cudaError_t launch_gnorm(const double2 *W, long long ld, int g0, int p_pad, int n, double *gcol2,
                         cudaStream_t s);
cudaError_t launch_finalize(const double2 *W, long long ld, const int8_t *Jrow, int m_pad, int p_pad,
                            int n, int sort, double *lam_tmp, double *gscale, double *vnorm2,
                            const double *gcol2, double *kappa, int *rank, double *lam_out,
                            double2 *V, long long ldv, int *err, cudaStream_t s);
cudaError_t launch_gemm(const double2 *A, long long lda, int rows, const void *B, bool b_single,
                        long long ldb, double2 *C, long long ldc, int n, cudaStream_t s);
cudaError_t launch_eye32(void *W, long long ld, int r0, int n, int n_pad, cudaStream_t s);
cudaError_t launch_extract(const double2 *W, long long ld, int r0, int rows, int n, double2 *out,
                           long long ldo, cudaStream_t s);

// Tensor-core (tcgen05 TF32) Gram and update of the complex64 sweeps (hz_tc.cu).
// W32 is the complex64 working copy; partial holds complex64 partials in the
// layout of launch_gram; zhat the complex64 Z^ of launch_inner.  Device waits
// are bounded: a wait that runs out raises DEVERR_TIMEOUT in err[0].
bool tc_supported(int kk, int npairs, long long ld);
int tc_gram_chunk_rows(int m_pad, int p_pad, int npairs, int sms);
cudaError_t tc_setup();
cudaError_t launch_gram_tc(const void *W32, const int8_t *Jrow, const StepArgs &a, int n, void *partial,
                           int *err, cudaStream_t s);
cudaError_t launch_update_tc(void *W32, const StepArgs &a, int n, const double2 *zhat, const int *pair_flag,
                             int *err, int sms, cudaStream_t s);
// tc_flag[p] = 1: pair p goes to launch_update_tc (its Z^ - I is small);
// cc_flag[p] = 1: to the FP32 CUDA-core launch_update; both 0: no transformation.
cudaError_t launch_route(const double2 *zhat, const int *pair_flag, int kk, int npairs, int *tc_flag,
                         int *cc_flag, cudaStream_t s);

// FP64 sweeps: the delta-form update of pairs whose Z^ - I is small
// (hz_delta.cu).  delta_flag[p] = 1: pair p goes to launch_update_delta64
// (FP32 product); df_flag[p] = 1: to launch_update_df64 (double-float
// product); full_flag[p] = 1: to launch_update (FP64 product); count[0],
// count[1], count[2] += the delta, FP64 and double-float pairs.
cudaError_t delta64_setup();
cudaError_t launch_route64(const double2 *zhat, const int *pair_flag, int kk, int npairs, int *delta_flag,
                           int *df_flag, int *full_flag, unsigned long long *count, cudaStream_t s);
cudaError_t launch_update_df64(double2 *W, const StepArgs &a, const double2 *zhat, const int *df_flag,
                               cudaStream_t s);
cudaError_t launch_update_delta64(double2 *W, const StepArgs &a, const double2 *zhat, const int *delta_flag,
                                  cudaStream_t s);

// Phase 2 (hz_urv.cu): the (J, I) URV shortening of Section 5.
size_t urv_workspace_bytes(long long m, long long p, int n);
cudaError_t launch_urv(int m, int p, int n, const double2 *F, long long ldf, const int8_t *J,
                       long long n_plus, const double2 *G, long long ldg, double2 *Fs, long long ldfs,
                       int8_t *Js, double2 *Gs, long long ldgs, long long *perm_out, int *permi,
                       void *ws, int *d_flags, cudaStream_t s);
int urv_launches(int n);

// Phase 4 (hz_phase4.cu): X = Z^{-1} and the pieces of eq. 7.1.
size_t inverse_workspace_bytes(int n);
int inverse_max_n();
cudaError_t launch_inverse(int n, const double2 *Z, long long ldz, double2 *X, long long ldx, void *ws,
                           int *d_flag, cudaStream_t s);
int inverse_launches(int n);
cudaError_t launch_sigma(const double2 *W, long long ld, const int8_t *Jrow, int m_pad, int p_pad, int n,
                         double *sig, double *sf, double *sg, double2 *Zs, long long ldz, cudaStream_t s);
cudaError_t launch_rowscale(const double2 *X, long long ldx, int n, const double *sig, double2 *B,
                            cudaStream_t s);
cudaError_t launch_rel_err(const double2 *A, long long lda, const double2 *C, long long ldc, int rows, int n,
                           double *part, double *out, cudaStream_t s);
cudaError_t launch_permute_rows(const double2 *src, long long lds, int n, const int *perm, double2 *dst,
                                long long ldd, cudaStream_t s);

}  // namespace hz

// Batched solves (hz_batch.cu).
#include "../../include/ghsvd.h"
// What a batched solve reports beside the per-pencil results.
struct HzBatchInfo {
    int w_chosen;               // block width used
    double ms_solve;            // wall time from set-up to the outputs
    long long ticks;            // ticks run on the device
    double ms_v0;               // applying the starting bases
    long long sweeps_low;       // complex64 sweeps over all pencils (mixed schedule)
    long long rounds_low;       // complex64 rounds over all pencils
};
void *hz_batch_new();
void hz_batch_free(void *buffers);
ghsvd_status hz_batch_solve(void *buffers, int device, const ghsvd_opts *opts, int batch,
                            const int64_t *m, const int64_t *p, const int64_t *n,
                            const void *const *F, const int64_t *ldf, const int8_t *const *J,
                            const int64_t *n_plus, const void *const *G, const int64_t *ldg,
                            const void *const *V0, const int64_t *ldv0, double *const *lambda, void *const *V, const int64_t *ldv, int *sweeps,
                            int *status, HzBatchInfo *info, void *stream);
