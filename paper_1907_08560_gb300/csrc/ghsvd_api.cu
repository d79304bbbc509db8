// ghsvd_api.cu -- the C ABI of include/ghsvd.h: handle, validation, working
// buffers, the block schedule and the sweep loop of the Level-2 block
// Hari-Zimmermann method (arXiv 1907.08560, Section 6.4).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#include "../../include/ghsvd.h"
#include "hz_launch.h"
#include "hz_pivot.cuh"

using hz::InnerArgs;
using hz::StepArgs;

// Per-kernel-class CUDA-event timer: events are recorded around every launch
// on the solve's stream and read once per sweep, after the sweep's sync.
struct KTimer {
    std::vector<cudaEvent_t> ev;
    int used = 0;
    cudaError_t reserve(int count)
    {
        while ((int)ev.size() < count) {
            cudaEvent_t e;
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return r;
            ev.push_back(e);
        }
        return cudaSuccess;
    }
    void release()
    {
        for (auto e : ev) cudaEventDestroy(e);
        ev.clear();
        used = 0;
    }
};

struct ghsvd_ctx {
    int device = 0;
    ghsvd_opts opts{};
    int num_sms = 0;
    // sizes of the allocation
    long long cap_w = 0, cap_w32 = 0;   // elements of W / W32
    long long cap_partial = 0;          // elements of the Gram partials
    int cap_pairs = 0, cap_n = 0, cap_mpad = 0, cap_steps = 0;
    // device buffers
    double2 *W = nullptr;               // [Mt x n] FP64 working factors F', G', Z'
    double2 *Wtmp = nullptr;            // [Mt x n] output of W <- W B (warm start, mixed)
    long long cap_wtmp = 0;
    float2 *W32 = nullptr;              // [Mt x n] complex64 copy (mixed schedule)
    void *partial = nullptr;            // Gram partials (FP64 or FP32 pairs)
    double2 *zhat = nullptr;            // [pairs][KKMAX^2] accumulated block transforms
    int *pair_flag = nullptr;           // [pairs]
    int *route = nullptr;               // [3][pairs]: the update route of each pair
    int *slotcol = nullptr;             // [steps][pairs][kk]
    int8_t *Jrow = nullptr;             // [m_pad]
    int8_t *Jdev = nullptr;             // [m] staging of a host J
    unsigned long long *counters = nullptr;   // [5]: all, big, delta, FP64, double-float pairs
    int *err = nullptr;                 // [2]: device error flags, bad J
    double *lam_tmp = nullptr, *gscale = nullptr;
    double *vnorm2 = nullptr, *gcol2 = nullptr, *kappa = nullptr;
    int *rank = nullptr;
    // pinned host mirrors
    unsigned long long *h_counters = nullptr;
    int *h_err = nullptr;
    // state of the last solve
    int m = 0, p = 0, n = 0, m_pad = 0, p_pad = 0, n_pad = 0;
    long long Mt = 0;
    bool solved = false;
    ghsvd_stats stats{};
    KTimer timer;
    void *batch = nullptr;              // working memory of ghsvd_solve_batched
    hz::GemmItem *d_item = nullptr;     // one item of the compensated warm-start product
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
#define CUDA_TRY(x)                                   \
    do {                                              \
        cudaError_t e_ = (x);                         \
        if (e_ != cudaSuccess) return status_of(e_);  \
    } while (0)

static ghsvd_status status_of(cudaError_t e)
{
    if (e == cudaSuccess) return GHSVD_OK;
    if (e == cudaErrorMemoryAllocation) return GHSVD_ERR_NOMEM;
    return GHSVD_ERR_CUDA;
}

static long long round_up(long long x, long long r) { return (x + r - 1) / r * r; }

template <typename T>
static cudaError_t grow(T **ptr, long long count, long long *cap)
{
    if (*ptr && count <= *cap) return cudaSuccess;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc((void **)ptr, sizeof(T) * (size_t)std::max(count, 1LL));
    if (e == cudaSuccess) *cap = count;
    return e;
}

static void free_all(ghsvd_ctx *h)
{
    h->timer.release();
    hz_batch_free(h->batch);
    h->batch = nullptr;
    cudaFree(h->d_item);
    h->d_item = nullptr;
    cudaFree(h->W); cudaFree(h->W32); cudaFree(h->Wtmp); cudaFree(h->partial); cudaFree(h->zhat);
    cudaFree(h->pair_flag); cudaFree(h->route); cudaFree(h->slotcol); cudaFree(h->Jrow); cudaFree(h->Jdev);
    cudaFree(h->counters); cudaFree(h->err); cudaFree(h->lam_tmp); cudaFree(h->gscale);
    cudaFree(h->rank); cudaFree(h->vnorm2); cudaFree(h->gcol2); cudaFree(h->kappa);
    cudaFreeHost(h->h_counters); cudaFreeHost(h->h_err);
    h->W = nullptr; h->W32 = nullptr; h->Wtmp = nullptr; h->partial = nullptr; h->zhat = nullptr;
    h->pair_flag = nullptr; h->route = nullptr; h->slotcol = nullptr; h->Jrow = nullptr; h->Jdev = nullptr;
    h->counters = nullptr; h->err = nullptr; h->lam_tmp = nullptr; h->gscale = nullptr;
    h->rank = nullptr; h->h_counters = nullptr; h->h_err = nullptr;
    h->vnorm2 = nullptr; h->gcol2 = nullptr; h->kappa = nullptr;
}

// Section 6.4.1: nb (even) block columns of width wb or wb - 1, widths
// non-increasing, from the prescribed maximal width w.
static int partition(int n, int w, std::vector<int> &off)
{
    int nb = (n + w - 1) / w;
    if (nb & 1) nb += 1;
    if (nb < 2) nb = 2;
    if (nb > n) nb = n & ~1;
    const int wb = (n + nb - 1) / nb;
    const int wide = n - nb * (wb - 1);
    off.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) off[b + 1] = off[b] + (b < wide ? wb : wb - 1);
    return nb;
}

// Gram chunk: forced by the options, else the balance rule of gram_chunk_rows.
static int choose_chunk(int m_pad, int p_pad, int npairs, int sms, int forced)
{
    if (forced > 0) return (int)round_up(forced, hz::GRAM_KT);
    return hz::gram_chunk_rows(m_pad, p_pad, npairs, sms);
}

static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" {

ghsvd_status ghsvd_default_opts(ghsvd_opts *o)
{
    if (!o) return GHSVD_ERR_INVALID_ARG;
    memset(o, 0, sizeof(*o));
    o->block_width = 32;
    o->inner_sweeps = 1;
    o->max_sweeps = 30;
    o->crit_mode = 0;
    o->precision = GHSVD_PRECISION_FP64;
    o->mixed_max_sweeps = 24;
    o->sort_ascending = 0;
    o->gram_chunk = 0;
    o->timing = 0;
    o->ordering = GHSVD_ORDER_ROUND_ROBIN;
    o->tol_scale = 1.0;
    o->timeout_ms = 0;
    o->shorten = 0;
    o->mixed_tc = 1;
    o->delta_update = 1;
    return GHSVD_OK;
}

const char *ghsvd_status_string(ghsvd_status s)
{
    switch (s) {
    case GHSVD_OK: return "ok";
    case GHSVD_ERR_INVALID_ARG: return "invalid argument";
    case GHSVD_ERR_RANK_DEFICIENT: return "G is numerically rank deficient";
    case GHSVD_ERR_NONFINITE: return "non-finite value in the input or the iteration";
    case GHSVD_ERR_NOT_CONVERGED: return "not converged within max_sweeps";
    case GHSVD_ERR_CUDA: return "CUDA error";
    case GHSVD_ERR_NOMEM: return "out of device memory";
    case GHSVD_ERR_SCRATCH_TOO_SMALL:
        return "problem too large for the no-allocation scratch array (GHSVD_NOALLOC_SCRATCH_BYTES)";
    case GHSVD_ERR_BREAKDOWN: return "hyperbolic QR breakdown (Phase 2)";
    case GHSVD_ERR_TIMEOUT: return "time limit reached; outputs written";
    }
    return "unknown status";
}

ghsvd_status ghsvd_create(ghsvd_t *out, int device, const ghsvd_opts *opts)
{
    if (!out) return GHSVD_ERR_INVALID_ARG;
    *out = nullptr;
    ghsvd_opts o;
    if (opts) o = *opts;
    else ghsvd_default_opts(&o);
    if (o.block_width < 0 || o.block_width > hz::KKMAX / 2 || o.inner_sweeps < 1 ||
        o.inner_sweeps > 30 || o.max_sweeps < 1 || o.max_sweeps > 1000 ||
        (o.crit_mode != 0 && o.crit_mode != 1) ||
        (o.precision != GHSVD_PRECISION_FP64 && o.precision != GHSVD_PRECISION_MIXED) ||
        o.mixed_max_sweeps < 0 || o.gram_chunk < 0 || (o.timing != 0 && o.timing != 1) ||
        (o.shorten != 0 && o.shorten != 1) || o.ordering != GHSVD_ORDER_ROUND_ROBIN ||
        (o.mixed_param32 != 0 && o.mixed_param32 != 1) || (o.mixed_tc != 0 && o.mixed_tc != 1) || (o.delta_update != 0 && o.delta_update != 1) ||
        !(o.tol_scale > 0.0 && o.tol_scale < 1e300) || o.timeout_ms < 0)
        return GHSVD_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GHSVD_ERR_INVALID_ARG;
    }
    ghsvd_ctx *h = new (std::nothrow) ghsvd_ctx();
    if (!h) return GHSVD_ERR_NOMEM;
    h->device = device;
    h->opts = o;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = hz::setup_kernels();
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_counters, 5 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_err, 2 * sizeof(int));
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        free_all(h);
        delete h;
        return status_of(e);
    }
    *out = h;
    return GHSVD_OK;
}

void ghsvd_destroy(ghsvd_t h)
{
    if (!h) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    free_all(h);
    cudaSetDevice(prev);
    delete h;
}

ghsvd_status ghsvd_get_stats(ghsvd_t h, ghsvd_stats *s)
{
    if (!h || !s) return GHSVD_ERR_INVALID_ARG;
    *s = h->stats;
    return GHSVD_OK;
}

}  // extern "C"

// The solver proper.  Dptr arguments are device pointers (validated by the
// callers of this function).
static ghsvd_status solve_impl(ghsvd_t h, int64_t m64, int64_t p64, int64_t n64, const void *F,
                               int64_t ldf, const int8_t *J, int64_t n_plus, const void *G,
                               int64_t ldg, const void *V0, int64_t ldv0, double *lambda, void *V,
                               int64_t ldv, int *sweeps_out, cudaStream_t st)
{
    auto t0 = std::chrono::steady_clock::now();
    const ghsvd_opts &o = h->opts;
    const int m = (int)m64, p = (int)p64, n = (int)n64;
    const int m_pad = (int)round_up(m, hz::ROWPAD), p_pad = (int)round_up(p, hz::ROWPAD);
    const int n_pad = (int)round_up(n, hz::ROWPAD);
    const long long Mt = (long long)m_pad + p_pad + n_pad;
    h->solved = false;
    memset(&h->stats, 0, sizeof(h->stats));

    // schedule (Section 6.3, 6.4.1)
    std::vector<int> off;
    int nb = 0, wb = 1, kk = 2, npairs = 0, nsteps = 0;
    if (n >= 2) {
        const int w = o.block_width > 0 ? o.block_width : 32;   // 0: automatic (32 for one pencil)
        nb = partition(n, std::min(w, n), off);
        wb = off[1] - off[0];
        kk = 2 * wb;
        npairs = nb / 2;
        nsteps = nb - 1;
    }
    const bool mixed = o.precision == GHSVD_PRECISION_MIXED && n >= 2;
    const int kc = n >= 2 ? choose_chunk(m_pad, p_pad, npairs, h->num_sms, o.gram_chunk) : 16;
    const int chunks_h = (m_pad + kc - 1) / kc, chunks_s = (p_pad + kc - 1) / kc;
    // the complex64 sweeps on the tensor cores (opts.mixed_tc) have a row
    // chunk of their own (two Gram CTAs per SM)
    const bool use_tc = mixed && o.mixed_tc && hz::tc_supported(kk, npairs, Mt);
    const int kc_tc = use_tc ? hz::tc_gram_chunk_rows(m_pad, p_pad, npairs, h->num_sms) : kc;
    const int chunks_h_tc = (m_pad + kc_tc - 1) / kc_tc, chunks_s_tc = (p_pad + kc_tc - 1) / kc_tc;
    const int cpp = std::max(chunks_h + chunks_s, chunks_h_tc + chunks_s_tc);

    // buffers
    long long cap;
    CUDA_TRY(grow(&h->W, Mt * n, &h->cap_w));
    if (mixed) CUDA_TRY(grow(&h->W32, Mt * n, &h->cap_w32));
    const long long npart = (long long)std::max(npairs, 1) * cpp * hz::KKMAX * hz::KKMAX;
    {
        double2 *pp = (double2 *)h->partial;
        CUDA_TRY(grow(&pp, npart, &h->cap_partial));
        h->partial = pp;
    }
    if (npairs > h->cap_pairs || h->zhat == nullptr) {
        cudaFree(h->zhat); cudaFree(h->pair_flag); cudaFree(h->route);
        h->zhat = nullptr; h->pair_flag = nullptr; h->route = nullptr;
        CUDA_TRY(cudaMalloc((void **)&h->zhat, sizeof(double2) * std::max(npairs, 1) * hz::KKMAX * hz::KKMAX));
        CUDA_TRY(cudaMalloc((void **)&h->pair_flag, sizeof(int) * std::max(npairs, 1)));
        CUDA_TRY(cudaMalloc((void **)&h->route, 3 * sizeof(int) * std::max(npairs, 1)));
        h->cap_pairs = std::max(npairs, 1);
    }
    cap = (long long)h->cap_steps;
    if ((long long)std::max(nsteps, 1) * std::max(npairs, 1) * kk > cap || !h->slotcol) {
        cudaFree(h->slotcol);
        h->slotcol = nullptr;
        const long long cnt = (long long)std::max(nsteps, 1) * std::max(npairs, 1) * kk;
        CUDA_TRY(cudaMalloc((void **)&h->slotcol, sizeof(int) * cnt));
        h->cap_steps = (int)cnt;
    }
    if (m_pad > h->cap_mpad || !h->Jrow) {
        cudaFree(h->Jrow); cudaFree(h->Jdev);
        h->Jrow = nullptr; h->Jdev = nullptr;
        CUDA_TRY(cudaMalloc((void **)&h->Jrow, m_pad));
        CUDA_TRY(cudaMalloc((void **)&h->Jdev, m_pad));
        h->cap_mpad = m_pad;
    }
    if (n > h->cap_n || !h->lam_tmp) {
        cudaFree(h->lam_tmp); cudaFree(h->gscale); cudaFree(h->rank);
        cudaFree(h->vnorm2); cudaFree(h->gcol2);
        h->lam_tmp = nullptr; h->gscale = nullptr; h->rank = nullptr;
        h->vnorm2 = nullptr; h->gcol2 = nullptr;
        CUDA_TRY(cudaMalloc((void **)&h->vnorm2, sizeof(double) * n));
        CUDA_TRY(cudaMalloc((void **)&h->gcol2, sizeof(double) * n));
        CUDA_TRY(cudaMalloc((void **)&h->lam_tmp, sizeof(double) * n));
        CUDA_TRY(cudaMalloc((void **)&h->gscale, sizeof(double) * n));
        CUDA_TRY(cudaMalloc((void **)&h->rank, sizeof(int) * n));
        h->cap_n = n;
    }
    if (!h->counters) {
        // all, big transformations of the sweep; FP64 pair updates in the
        // delta form and by the FP64 product
        CUDA_TRY(cudaMalloc((void **)&h->counters, 5 * sizeof(unsigned long long)));
        CUDA_TRY(cudaMalloc((void **)&h->err, 2 * sizeof(int)));
        CUDA_TRY(cudaMalloc((void **)&h->kappa, sizeof(double)));
    }

    // slot tables: step r, pair k -> block pair (P, Q) of the round-robin over
    // nb blocks; P's columns in slots [0, |P|), Q's in [wb, wb + |Q|)
    if (n >= 2) {
        std::vector<int> tab((size_t)nsteps * npairs * kk, -1);
        for (int r = 0; r < nsteps; ++r)
            for (int k = 0; k < npairs; ++k) {
                int P, Q;
                hz::rr_pair(nb, r, k, &P, &Q);
                int *row = &tab[((size_t)r * npairs + k) * kk];
                for (int c = off[P]; c < off[P + 1]; ++c) row[c - off[P]] = c;
                for (int c = off[Q]; c < off[Q + 1]; ++c) row[wb + c - off[Q]] = c;
            }
        CUDA_TRY(cudaMemcpyAsync(h->slotcol, tab.data(), sizeof(int) * tab.size(),
                                 cudaMemcpyHostToDevice, st));
    }

    // inputs: J (host or device) -> padded signs; [F; G; V0 or I] -> W
    auto t_v0 = std::chrono::steady_clock::now();
    CUDA_TRY(cudaMemsetAsync(h->err, 0, 2 * sizeof(int), st));
    const int8_t *Jd = nullptr;
    if (J) {
        if (is_device_ptr(J)) Jd = J;
        else {
            CUDA_TRY(cudaMemcpyAsync(h->Jdev, J, (size_t)m, cudaMemcpyHostToDevice, st));
            Jd = h->Jdev;
        }
    }
    CUDA_TRY(hz::launch_signs(h->Jrow, Jd, m, m_pad, n_plus, h->err + 1, st));
    h->stats.kernel_launches += 3;   // signs, copy-in, column norms of G
    CUDA_TRY(hz::launch_copyin(h->W, false, Mt, m, p, n, m_pad, p_pad, n_pad, F, ldf, G, ldg,
                               nullptr, 0, h->err, st));
    CUDA_TRY(hz::launch_gnorm(h->W, Mt, m_pad, p_pad, n, h->gcol2, st));
    if (V0) {
        // warm start: the sweeps run on (F V0, G V0) and start from Z' = V0
        // (Algorithm 1 admits any nonsingular starting Z')
        // (compensated sums: the basis may be ill-conditioned)
        CUDA_TRY(grow(&h->Wtmp, Mt * n, &h->cap_wtmp));
        if (!h->d_item) CUDA_TRY(cudaMalloc((void **)&h->d_item, sizeof(hz::GemmItem) + 8));
        double *d_kap = (double *)(h->d_item + 1);
        const hz::GemmItem probe{(const double2 *)V0, ldv0, n, (const double2 *)h->gcol2, 0, nullptr, 0,
                                 n, 0};
        double kap = 0.0;
        CUDA_TRY(cudaMemcpyAsync(h->d_item, &probe, sizeof(probe), cudaMemcpyHostToDevice, st));
        CUDA_TRY(hz::launch_v0_kappa(h->d_item, 1, d_kap, st));
        CUDA_TRY(cudaMemcpyAsync(&kap, d_kap, 8, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        t_v0 = std::chrono::steady_clock::now();
        // the rows of F and G only: the rows of Z' (= I) become V0 itself
        const long long fg = (long long)m_pad + p_pad;
        const hz::GemmItem item{h->W, Mt, fg, (const double2 *)V0, ldv0, h->Wtmp, Mt, n,
                                !(kap <= hz::WARM_ACCURATE_KAPPA)};
        CUDA_TRY(cudaMemcpyAsync(h->d_item, &item, sizeof(item), cudaMemcpyHostToDevice, st));
        CUDA_TRY(hz::launch_gemm_batched(h->d_item, 1, fg, n, st));
        h->stats.kernel_launches += 1;
        CUDA_TRY(cudaMemcpy2DAsync(h->W, sizeof(double2) * Mt, h->Wtmp, sizeof(double2) * Mt,
                                   sizeof(double2) * fg, n, cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(cudaMemcpy2DAsync(h->W + fg, sizeof(double2) * Mt, V0, sizeof(double2) * ldv0,
                                   sizeof(double2) * n, n, cudaMemcpyDeviceToDevice, st));
    }
    CUDA_TRY(cudaMemcpyAsync(h->h_err, h->err, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (V0)
        h->stats.ms_v0 =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_v0).count();
    if (h->h_err[1]) return GHSVD_ERR_INVALID_ARG;
    if (h->h_err[0] & hz::DEVERR_NONFINITE) return GHSVD_ERR_NONFINITE;

    h->m = m; h->p = p; h->n = n; h->m_pad = m_pad; h->p_pad = p_pad; h->n_pad = n_pad; h->Mt = Mt;
    ghsvd_status status = GHSVD_ERR_NOT_CONVERGED;
    int sweeps = 0, sweeps_low = 0, rounds = 0;
    h->stats.steps_per_sweep = nsteps;
    h->stats.pairs_per_step = npairs;
    h->stats.block_width = wb;

    if (n < 2) {
        status = GHSVD_OK;
    } else {
        StepArgs sa{};
        sa.npairs = npairs; sa.kk = kk; sa.m_pad = m_pad; sa.p_pad = p_pad; sa.n_pad = n_pad;
        sa.ld = Mt; sa.kc = kc; sa.chunks_h = chunks_h; sa.chunks_s = chunks_s;
        StepArgs sa_tc = sa;
        sa_tc.kc = kc_tc; sa_tc.chunks_h = chunks_h_tc; sa_tc.chunks_s = chunks_s_tc;
        InnerArgs ia{};
        ia.npairs = npairs; ia.kk = kk; ia.cpp = chunks_h + chunks_s; ia.chunks_h = chunks_h;
        ia.inner_sweeps = o.inner_sweeps; ia.crit_mode = o.crit_mode;
        ia.param32 = o.mixed_param32;
        const double tol64 = o.tol_scale * ldexp(1.0, -53) * sqrt((double)n);
        // complex64 sweeps: the single-precision unit roundoff in eq. 6.12,
        // so that pivots below the Gram's rounding level are left alone
        const double tol32 = o.tol_scale * ldexp(1.0, -24) * sqrt((double)n);

        // Mixed schedule (iterative refinement): complex64 sweeps run on
        // W32 = fl32(W) with Z' restarted at I until their big transformations
        // stagnate at the complex64 rounding level; the accumulated Z'_low is
        // then applied to the FP64 factors, W <- W Z'_low (an exact congruence
        // of the pencil, in FP64), and, while a round still made progress, a
        // new complex64 round starts from fl32 of the improved W, whose columns
        // are now nearly orthogonal so that rounding them to complex64 no
        // longer perturbs the ill-conditioned directions.  FP64 sweeps finish.
        // Two rounds: a third and fourth (n = 2048 pencil: 7 more complex64
        // sweeps and two more FP64 products) spared one nearly empty FP64
        // sweep and took 0.5 s more than they saved.
        constexpr int kMaxRounds = 2;
        int phase_single = mixed ? 1 : 0;
        int round_sweeps = 0;
        unsigned long long prev_big = ~0ULL;
        const double pivots_per_sweep = (double)nsteps * npairs * (kk / 2) * (kk - 1);
        if (mixed) {
            CUDA_TRY(hz::launch_convert(h->W32, true, h->W, Mt * n, st));
            CUDA_TRY(hz::launch_eye32(h->W32, Mt, m_pad + p_pad, n, n_pad, st));
            h->stats.kernel_launches += 2;
            CUDA_TRY(grow(&h->Wtmp, Mt * n, &h->cap_wtmp));
        }
        while (sweeps < o.max_sweeps) {
            if (o.timeout_ms > 0 && sweeps > 0 &&
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() >=
                    (double)o.timeout_ms) {
                status = GHSVD_ERR_TIMEOUT;
                break;
            }
            const bool single = phase_single != 0;
            const bool tcs = single && use_tc;
            ia.tol = single ? tol32 : tol64;
            ia.cpp = tcs ? chunks_h_tc + chunks_s_tc : chunks_h + chunks_s;
            ia.chunks_h = tcs ? chunks_h_tc : chunks_h;
            CUDA_TRY(cudaMemsetAsync(h->counters, 0, 5 * sizeof(unsigned long long), st));
            const bool timed = o.timing != 0;
            const bool delta = !single && o.delta_update;
            if (timed) CUDA_TRY(h->timer.reserve(6 * nsteps));
            cudaEvent_t *ev = timed ? h->timer.ev.data() : nullptr;
            for (int r = 0; r < nsteps; ++r) {
                void *Wc = single ? (void *)h->W32 : (void *)h->W;
                sa.slotcol = h->slotcol + (size_t)r * npairs * kk;
                if (timed) CUDA_TRY(cudaEventRecord(ev[6 * r + 0], st));
                if (tcs) {
                    sa_tc.slotcol = sa.slotcol;
                    CUDA_TRY(hz::launch_gram_tc(Wc, h->Jrow, sa_tc, n, h->partial, h->err, st));
                } else {
                    CUDA_TRY(hz::launch_gram(Wc, single, h->Jrow, sa, h->partial, st));
                }
                if (timed) CUDA_TRY(cudaEventRecord(ev[6 * r + 1], st));
                if (timed) CUDA_TRY(cudaEventRecord(ev[6 * r + 2], st));
                CUDA_TRY(hz::launch_inner(h->partial, single, sa.slotcol, ia, h->zhat, h->pair_flag,
                                          h->counters, h->err, st));
                if (timed) CUDA_TRY(cudaEventRecord(ev[6 * r + 3], st));
                if (timed) CUDA_TRY(cudaEventRecord(ev[6 * r + 4], st));
                if (tcs) {
                    // pairs with small rotations on the tensor cores, the others on
                    // the CUDA cores (launch_route)
                    int *tcf = h->route, *ccf = h->route + npairs;
                    CUDA_TRY(hz::launch_route(h->zhat, h->pair_flag, kk, npairs, tcf, ccf, st));
                    CUDA_TRY(hz::launch_update_tc(Wc, sa, n, h->zhat, tcf, h->err, h->num_sms, st));
                    CUDA_TRY(hz::launch_update(Wc, true, sa, h->zhat, ccf, st));
                } else if (delta) {
                    // pairs whose Z^ - I is small in the delta form (FP32 or
                    // double-float product, hz_delta.cu), the others by the
                    // FP64 product
                    int *dl = h->route, *ff = h->route + npairs, *dd = h->route + 2 * npairs;
                    CUDA_TRY(hz::launch_route64(h->zhat, h->pair_flag, kk, npairs, dl, dd, ff, h->counters + 2,
                                                st));
                    CUDA_TRY(hz::launch_update_delta64(h->W, sa, h->zhat, dl, st));
                    CUDA_TRY(hz::launch_update_df64(h->W, sa, h->zhat, dd, st));
                    CUDA_TRY(hz::launch_update(Wc, false, sa, h->zhat, ff, st));
                } else {
                    CUDA_TRY(hz::launch_update(Wc, single, sa, h->zhat, h->pair_flag, st));
                }
                if (timed) CUDA_TRY(cudaEventRecord(ev[6 * r + 5], st));
            }
            h->stats.launches_gram += nsteps;
            h->stats.launches_inner += nsteps;
            h->stats.launches_update += nsteps;
            h->stats.kernel_launches += (delta ? 6LL : tcs ? 5LL : 3LL) * nsteps;
            CUDA_TRY(cudaMemcpyAsync(h->h_counters, h->counters, 5 * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaMemcpyAsync(h->h_err, h->err, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            if (timed) {
                for (int r = 0; r < nsteps; ++r) {
                    float a = 0, b = 0, c = 0;
                    CUDA_TRY(cudaEventElapsedTime(&a, ev[6 * r + 0], ev[6 * r + 1]));
                    CUDA_TRY(cudaEventElapsedTime(&b, ev[6 * r + 2], ev[6 * r + 3]));
                    CUDA_TRY(cudaEventElapsedTime(&c, ev[6 * r + 4], ev[6 * r + 5]));
                    h->stats.ms_gram += a;
                    h->stats.ms_inner += b;
                    h->stats.ms_update += c;
                }
            }
            if (sweeps < 64) {
                h->stats.transforms[sweeps] = (long long)h->h_counters[0];
                h->stats.big[sweeps] = (long long)h->h_counters[1];
            }
            ++sweeps;
            if (single) ++sweeps_low;
            if (tcs) ++h->stats.sweeps_tc;
            if (delta) {
                h->stats.pairs_delta += (long long)h->h_counters[2];
                h->stats.pairs_fp64 += (long long)h->h_counters[3];
                h->stats.pairs_df += (long long)h->h_counters[4];
            }
            if (h->h_err[0] & hz::DEVERR_TIMEOUT) { status = GHSVD_ERR_CUDA; break; }
            if (h->h_err[0] & hz::DEVERR_RANK) { status = GHSVD_ERR_RANK_DEFICIENT; break; }
            if (h->h_err[0] & hz::DEVERR_NONFINITE) { status = GHSVD_ERR_NONFINITE; break; }
            if (single) {
                ++round_sweeps;
                const unsigned long long all = h->h_counters[0], big = h->h_counters[1];
                // stagnation: fewer than 10 % of the pivots still rotate
                // "big" and that number no longer falls by a fifth per sweep
                // (the convergent phase of a round falls by 20-60 % per sweep
                // once below a quarter of the pivots; the complex64 floor of
                // small pencils lies between 1 and 10 %)
                const bool plateau = round_sweeps >= 2 && (double)big > 0.8 * (double)prev_big &&
                                     (double)big < 0.1 * pivots_per_sweep;
                prev_big = big;
                const bool budget = sweeps_low >= o.mixed_max_sweeps;
                if (all == 0 || plateau || budget) {
                    const float2 *zlow = h->W32 + (m_pad + p_pad);
                    CUDA_TRY(hz::launch_gemm(h->W, Mt, (int)Mt, zlow, true, Mt, h->Wtmp, Mt, n, st));
                    CUDA_TRY(cudaMemcpyAsync(h->W, h->Wtmp, sizeof(double2) * Mt * n,
                                             cudaMemcpyDeviceToDevice, st));
                    h->stats.kernel_launches += 1;
                    ++rounds;
                    if (budget || all == 0 || round_sweeps <= 3 || rounds >= kMaxRounds) {
                        phase_single = 0;            // FP64 finishing sweeps
                    } else {                         // next complex64 round
                        CUDA_TRY(hz::launch_convert(h->W32, true, h->W, Mt * n, st));
                        CUDA_TRY(hz::launch_eye32(h->W32, Mt, m_pad + p_pad, n, n_pad, st));
                        h->stats.kernel_launches += 2;
                        round_sweeps = 0;
                        prev_big = ~0ULL;
                    }
                }
                continue;
            }
            if (h->h_counters[1] == 0) { status = GHSVD_OK; break; }
        }
    }
    h->stats.sweeps = sweeps;
    h->stats.sweeps_low = sweeps_low;
    h->stats.rounds_low = rounds;
    if (status == GHSVD_ERR_RANK_DEFICIENT || status == GHSVD_ERR_NONFINITE || status == GHSVD_ERR_CUDA)
        return status;

    // outputs (Section 6.1.7)
    CUDA_TRY(hz::launch_finalize(h->W, Mt, h->Jrow, m_pad, p_pad, n, o.sort_ascending, h->lam_tmp,
                                 h->gscale, h->vnorm2, h->gcol2, h->kappa, h->rank, lambda,
                                 (double2 *)V, ldv, h->err, st));
    h->stats.kernel_launches += 4;   // column norms, rank check, order, emit
    CUDA_TRY(cudaMemcpyAsync(h->h_err, h->err, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (h->h_err[0] & hz::DEVERR_RANK) return GHSVD_ERR_RANK_DEFICIENT;
    if (h->h_err[0] & hz::DEVERR_NONFINITE) return GHSVD_ERR_NONFINITE;
    h->solved = true;
    if (sweeps_out) *sweeps_out = sweeps;
    h->stats.ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return status;
}

static ghsvd_status validate(ghsvd_t h, int64_t m, int64_t p, int64_t n, const void *F, int64_t ldf,
                             const int8_t *J, int64_t n_plus, const void *G, int64_t ldg,
                             double *lambda, const void *V, int64_t ldv)
{
    if (!h || !F || !G || !lambda) return GHSVD_ERR_INVALID_ARG;
    if (n < 1 || m < n || p < n) return GHSVD_ERR_INVALID_ARG;
    if (m > (1LL << 30) || p > (1LL << 30) || n > (1 << 20)) return GHSVD_ERR_INVALID_ARG;
    if (ldf < m || ldg < p) return GHSVD_ERR_INVALID_ARG;
    if (V && ldv < n) return GHSVD_ERR_INVALID_ARG;
    if (!J && (n_plus < 0 || n_plus > m)) return GHSVD_ERR_INVALID_ARG;
    return GHSVD_OK;
}

// Phase 2 then the iteration on the square pencil (opts.shorten), else the
// iteration on the given factors.  Device pointers, except a host J.
static ghsvd_status solve_entry(ghsvd_t h, int64_t m, int64_t p, int64_t n, const void *F, int64_t ldf,
                                const int8_t *J, int64_t n_plus, const void *G, int64_t ldg,
                                const void *V0, int64_t ldv0, double *lambda, void *V, int64_t ldv,
                                int *sweeps, cudaStream_t st)
{
    if (!h->opts.shorten)
        return solve_impl(h, m, p, n, F, ldf, J, n_plus, G, ldg, V0, ldv0, lambda, V, ldv, sweeps, st);
    if (V0) return GHSVD_ERR_INVALID_ARG;
    auto t0 = std::chrono::steady_clock::now();
    const size_t wsb = hz::urv_workspace_bytes(m, p, (int)n);
    void *ws = nullptr, *Fs = nullptr, *Gs = nullptr, *Vs = nullptr;
    int8_t *Js = nullptr, *Jd = nullptr;
    int *permi = nullptr, *dflags = nullptr;
    int hflags[3] = {0, 0, 0};
    cudaError_t e = cudaMallocAsync(&ws, wsb, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&Fs, 16ull * n * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&Gs, 16ull * n * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&Js, (size_t)n, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&permi, 4ull * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dflags, 16, st);
    if (e == cudaSuccess && V) e = cudaMallocAsync(&Vs, 16ull * n * n, st);
    if (e == cudaSuccess && J && !is_device_ptr(J)) {
        e = cudaMallocAsync((void **)&Jd, (size_t)m, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Jd, J, (size_t)m, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess)
        e = hz::launch_urv((int)m, (int)p, (int)n, (const double2 *)F, ldf, Jd ? Jd : J, n_plus,
                           (const double2 *)G, ldg, (double2 *)Fs, n, Js, (double2 *)Gs, n, nullptr, permi,
                           ws, dflags, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hflags, dflags, 12, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const double ms2 =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    ghsvd_status s = status_of(e);
    if (s == GHSVD_OK && hflags[2]) s = GHSVD_ERR_INVALID_ARG;
    if (s == GHSVD_OK && hflags[0]) s = GHSVD_ERR_BREAKDOWN;
    if (s == GHSVD_OK) {
        s = solve_impl(h, n, n, n, Fs, n, Js, 0, Gs, n, nullptr, 0, lambda, Vs, n, sweeps, st);
        if (V && (s == GHSVD_OK || s == GHSVD_ERR_NOT_CONVERGED || s == GHSVD_ERR_TIMEOUT)) {
            e = hz::launch_permute_rows((const double2 *)Vs, n, (int)n, permi, (double2 *)V, ldv, st);
            if (e != cudaSuccess) s = status_of(e);
            h->stats.kernel_launches += 1;
        }
        h->stats.kernel_launches += hz::urv_launches((int)n);
        h->stats.ms_phase2 = ms2;
        h->stats.n2x2 = hflags[1];
    }
    cudaFreeAsync(ws, st); cudaFreeAsync(Fs, st); cudaFreeAsync(Gs, st); cudaFreeAsync(Js, st);
    cudaFreeAsync(permi, st); cudaFreeAsync(dflags, st);
    if (Vs) cudaFreeAsync(Vs, st);
    if (Jd) cudaFreeAsync(Jd, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (s == GHSVD_OK && e2 != cudaSuccess) s = status_of(e2);
    h->stats.ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return s;
}

extern "C" {

ghsvd_status ghsvd_solve_from(ghsvd_t h, int64_t m, int64_t p, int64_t n, const void *F, int64_t ldf,
                              const int8_t *J, int64_t n_plus, const void *G, int64_t ldg,
                              const void *V0, int64_t ldv0, double *lambda, void *V, int64_t ldv,
                              int *sweeps, void *stream)
{
    ghsvd_status s = validate(h, m, p, n, F, ldf, J, n_plus, G, ldg, lambda, V, ldv);
    if (s != GHSVD_OK) return s;
    if (V0 && ldv0 < n) return GHSVD_ERR_INVALID_ARG;
    if (!is_device_ptr(F) || !is_device_ptr(G) || !is_device_ptr(lambda) ||
        (V && !is_device_ptr(V)) || (V0 && !is_device_ptr(V0)))
        return GHSVD_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(h->device) != cudaSuccess) return GHSVD_ERR_CUDA;
    s = solve_entry(h, m, p, n, F, ldf, J, n_plus, G, ldg, V0, ldv0, lambda, V, ldv, sweeps,
                    (cudaStream_t)stream);
    cudaSetDevice(prev);
    return s;
}

ghsvd_status ghsvd_solve(ghsvd_t h, int64_t m, int64_t p, int64_t n, const void *F, int64_t ldf,
                         const int8_t *J, int64_t n_plus, const void *G, int64_t ldg, double *lambda,
                         void *V, int64_t ldv, int *sweeps, void *stream)
{
    return ghsvd_solve_from(h, m, p, n, F, ldf, J, n_plus, G, ldg, nullptr, 0, lambda, V, ldv,
                            sweeps, stream);
}

ghsvd_status ghsvd_solve_host(ghsvd_t h, int64_t m, int64_t p, int64_t n, const void *F,
                              int64_t ldf, const int8_t *J, int64_t n_plus, const void *G,
                              int64_t ldg, double *lambda, void *V, int64_t ldv, int *sweeps,
                              void *stream)
{
    ghsvd_status s = validate(h, m, p, n, F, ldf, J, n_plus, G, ldg, lambda, V, ldv);
    if (s != GHSVD_OK) return s;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(h->device) != cudaSuccess) return GHSVD_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    void *dF = nullptr, *dG = nullptr, *dV = nullptr;
    double *dl = nullptr;
    int8_t *dJ = nullptr;
    cudaError_t e = cudaMallocAsync(&dF, sizeof(double2) * (size_t)m * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dG, sizeof(double2) * (size_t)p * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dl, sizeof(double) * (size_t)n, st);
    if (e == cudaSuccess && V) e = cudaMallocAsync(&dV, sizeof(double2) * (size_t)n * n, st);
    if (e == cudaSuccess && J) e = cudaMallocAsync((void **)&dJ, (size_t)m, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(dF, sizeof(double2) * m, F, sizeof(double2) * ldf, sizeof(double2) * m, n,
                              cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(dG, sizeof(double2) * p, G, sizeof(double2) * ldg, sizeof(double2) * p, n,
                              cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && J) e = cudaMemcpyAsync(dJ, J, (size_t)m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        s = solve_entry(h, m, p, n, dF, m, J ? dJ : nullptr, n_plus, dG, p, nullptr, 0, dl, dV, n,
                        sweeps, st);
        if (s == GHSVD_OK || s == GHSVD_ERR_NOT_CONVERGED || s == GHSVD_ERR_TIMEOUT) {
            e = cudaMemcpyAsync(lambda, dl, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && V)
                e = cudaMemcpy2DAsync(V, sizeof(double2) * ldv, dV, sizeof(double2) * n,
                                      sizeof(double2) * n, n, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
    } else {
        s = status_of(e);
    }
    cudaFreeAsync(dF, st); cudaFreeAsync(dG, st); cudaFreeAsync(dl, st);
    if (dV) cudaFreeAsync(dV, st);
    if (dJ) cudaFreeAsync(dJ, st);
    cudaStreamSynchronize(st);
    cudaSetDevice(prev);
    if (e != cudaSuccess && s == GHSVD_OK) s = status_of(e);
    return s;
}

ghsvd_status ghsvd_get_factors(ghsvd_t h, void *Fp, int64_t ldf, void *Gp, int64_t ldg, void *Zp,
                               int64_t ldz, void *stream)
{
    if (!h || !h->solved) return GHSVD_ERR_INVALID_ARG;
    if ((Fp && ldf < h->m) || (Gp && ldg < h->p) || (Zp && ldz < h->n)) return GHSVD_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(h->device) != cudaSuccess) return GHSVD_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (Fp) e = hz::launch_extract(h->W, h->Mt, 0, h->m, h->n, (double2 *)Fp, ldf, st);
    if (e == cudaSuccess && Gp) e = hz::launch_extract(h->W, h->Mt, h->m_pad, h->p, h->n, (double2 *)Gp, ldg, st);
    if (e == cudaSuccess && Zp)
        e = hz::launch_extract(h->W, h->Mt, h->m_pad + h->p_pad, h->n, h->n, (double2 *)Zp, ldz, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaSetDevice(prev);
    return status_of(e);
}

}  // extern "C"

extern "C" ghsvd_status ghsvd_solve_batched(ghsvd_t h, int batch, const int64_t *m, const int64_t *p,
                                           const int64_t *n, const void *const *F, const int64_t *ldf,
                                           const int8_t *const *J, const int64_t *n_plus,
                                           const void *const *G, const int64_t *ldg,
                                           const void *const *V0, const int64_t *ldv0,
                                           double *const *lambda, void *const *V, const int64_t *ldv,
                                           int *sweeps, int *status, void *stream)
{
    if (!h || batch < 1 || !m || !p || !n || !F || !ldf || !G || !ldg || !lambda)
        return GHSVD_ERR_INVALID_ARG;
    if (h->opts.precision != GHSVD_PRECISION_FP64 && h->opts.precision != GHSVD_PRECISION_MIXED)
        return GHSVD_ERR_INVALID_ARG;
    for (int i = 0; i < batch; ++i) {
        const int8_t *Ji = J ? J[i] : nullptr;
        const int64_t np_ = n_plus ? n_plus[i] : m[i];
        ghsvd_status s = validate(h, m[i], p[i], n[i], F[i], ldf[i], Ji, np_, G[i], ldg[i], lambda[i],
                                  V ? V[i] : nullptr, ldv ? ldv[i] : n[i]);
        if (s != GHSVD_OK) return s;
        if (n[i] < 2 || n[i] > (1 << 20)) return GHSVD_ERR_INVALID_ARG;
        if (!is_device_ptr(F[i]) || !is_device_ptr(G[i]) || !is_device_ptr(lambda[i]) ||
            (V && V[i] && !is_device_ptr(V[i])) || (Ji && !is_device_ptr(Ji)))
            return GHSVD_ERR_INVALID_ARG;
        if (V0 && V0[i] && (!ldv0 || ldv0[i] < n[i] || !is_device_ptr(V0[i])))
            return GHSVD_ERR_INVALID_ARG;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(h->device) != cudaSuccess) return GHSVD_ERR_CUDA;
    if (!h->batch) h->batch = hz_batch_new();
    if (!h->batch) { cudaSetDevice(prev); return GHSVD_ERR_NOMEM; }
    memset(&h->stats, 0, sizeof(h->stats));
    HzBatchInfo info{};
    ghsvd_status s = hz_batch_solve(h->batch, h->device, &h->opts, batch, m, p, n, F, ldf, J, n_plus,
                                    G, ldg, V0, ldv0, lambda, V, ldv, sweeps, status, &info, stream);
    h->stats.ms_v0 = info.ms_v0;
    h->stats.block_width = info.w_chosen;
    h->stats.ms_total = info.ms_solve;
    h->stats.batch_ticks = info.ticks;
    h->stats.batch_graph_launches = info.ticks > 0 ? 1 : 0;
    h->stats.sweeps_low = (int)info.sweeps_low;
    h->stats.rounds_low = (int)info.rounds_low;
    h->solved = false;          // ghsvd_get_factors refers to single solves
    cudaSetDevice(prev);
    return s;
}

// ---------------------------------------------------------------------------
// Phase 2 and Phase 4 (Sections 5 and 7)
// ---------------------------------------------------------------------------
extern "C" {

ghsvd_status ghsvd_urv(int64_t m, int64_t p, int64_t n, const void *F, int64_t ldf, const int8_t *J,
                       int64_t n_plus, const void *G, int64_t ldg, void *Fs, int64_t ldfs, int8_t *Js,
                       void *Gs, int64_t ldgs, int64_t *perm, int *n2x2, void *stream)
{
    if (!F || !G || !Fs || !Js || !Gs || n < 1 || m < n || p < n || ldf < m || ldg < p || ldfs < n ||
        ldgs < n || m > (1LL << 30) || p > (1LL << 30) || n > (1 << 20))
        return GHSVD_ERR_INVALID_ARG;
    if (!J && (n_plus < 0 || n_plus > m)) return GHSVD_ERR_INVALID_ARG;
    if (!is_device_ptr(F) || !is_device_ptr(G) || !is_device_ptr(Fs) || !is_device_ptr(Js) ||
        !is_device_ptr(Gs) || (perm && !is_device_ptr(perm)) || (J && !is_device_ptr(J)))
        return GHSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    void *ws = nullptr;
    int *dflags = nullptr;
    int hflags[3] = {0, 0, 0};
    cudaError_t e = cudaMallocAsync(&ws, hz::urv_workspace_bytes(m, p, (int)n), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dflags, 16, st);
    if (e == cudaSuccess)
        e = hz::launch_urv((int)m, (int)p, (int)n, (const double2 *)F, ldf, J, n_plus, (const double2 *)G,
                           ldg, (double2 *)Fs, ldfs, Js, (double2 *)Gs, ldgs, (long long *)perm, nullptr,
                           ws, dflags, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hflags, dflags, 12, cudaMemcpyDeviceToHost, st);
    if (ws) cudaFreeAsync(ws, st);
    if (dflags) cudaFreeAsync(dflags, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return status_of(e);
    if (n2x2) *n2x2 = hflags[1];
    if (hflags[2]) return GHSVD_ERR_INVALID_ARG;
    return hflags[0] ? GHSVD_ERR_BREAKDOWN : GHSVD_OK;
}

ghsvd_status ghsvd_inverse(int64_t n, const void *Z, int64_t ldz, void *X, int64_t ldx, void *stream)
{
    if (!Z || !X || n < 1 || n > hz::inverse_max_n() || ldz < n || ldx < n) return GHSVD_ERR_INVALID_ARG;
    if (!is_device_ptr(Z) || !is_device_ptr(X)) return GHSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    void *ws = nullptr;
    int *dflag = nullptr;
    int hflag = 0;
    cudaError_t e = cudaMallocAsync(&ws, hz::inverse_workspace_bytes((int)n), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dflag, 4, st);
    if (e == cudaSuccess)
        e = hz::launch_inverse((int)n, (const double2 *)Z, ldz, (double2 *)X, ldx, ws, dflag, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, dflag, 4, cudaMemcpyDeviceToHost, st);
    if (ws) cudaFreeAsync(ws, st);
    if (dflag) cudaFreeAsync(dflag, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return status_of(e);
    return hflag ? GHSVD_ERR_RANK_DEFICIENT : GHSVD_OK;
}

ghsvd_status ghsvd_phase4(ghsvd_t h, double *sigma_f, double *sigma_g, void *X, int64_t ldx, void *stream)
{
    if (!h || !h->solved) return GHSVD_ERR_INVALID_ARG;
    const int n = h->n;
    if (X && (ldx < n || n > hz::inverse_max_n())) return GHSVD_ERR_INVALID_ARG;
    if ((sigma_f && !is_device_ptr(sigma_f)) || (sigma_g && !is_device_ptr(sigma_g)) ||
        (X && !is_device_ptr(X)))
        return GHSVD_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(h->device) != cudaSuccess) return GHSVD_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    double *sig = nullptr;
    double2 *Zs = nullptr;
    void *ws = nullptr;
    int *dflag = nullptr;
    int hflag = 0;
    cudaError_t e = cudaMallocAsync((void **)&sig, 8ull * n, st);
    if (e == cudaSuccess && X) e = cudaMallocAsync((void **)&Zs, 16ull * n * n, st);
    if (e == cudaSuccess && X) e = cudaMallocAsync(&ws, hz::inverse_workspace_bytes(n), st);
    if (e == cudaSuccess && X) e = cudaMallocAsync((void **)&dflag, 4, st);
    if (e == cudaSuccess)
        e = hz::launch_sigma(h->W, h->Mt, h->Jrow, h->m_pad, h->p_pad, n, sig, sigma_f, sigma_g, Zs, n, st);
    if (e == cudaSuccess && X) e = hz::launch_inverse(n, Zs, n, (double2 *)X, ldx, ws, dflag, st);
    if (e == cudaSuccess && X) e = cudaMemcpyAsync(&hflag, dflag, 4, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(sig, st);
    if (Zs) cudaFreeAsync(Zs, st);
    if (ws) cudaFreeAsync(ws, st);
    if (dflag) cudaFreeAsync(dflag, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaSetDevice(prev);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return status_of(e);
    return hflag ? GHSVD_ERR_RANK_DEFICIENT : GHSVD_OK;
}

ghsvd_status ghsvd_decomposition_errors(ghsvd_t h, const void *F, int64_t ldf, const void *G, int64_t ldg,
                                        const void *X, int64_t ldx, double *err_f, double *err_g,
                                        void *stream)
{
    if (!h || !h->solved || !F || !G || !X || !err_f || !err_g) return GHSVD_ERR_INVALID_ARG;
    const int n = h->n, m = h->m, p = h->p;
    if (ldf < m || ldg < p || ldx < n) return GHSVD_ERR_INVALID_ARG;
    if (!is_device_ptr(F) || !is_device_ptr(G) || !is_device_ptr(X)) return GHSVD_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(h->device) != cudaSuccess) return GHSVD_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const long long rows = (long long)h->m_pad + h->p_pad;
    double *sig = nullptr, *part = nullptr, *out = nullptr;
    double2 *B = nullptr, *C = nullptr;
    hz::GemmItem *item = nullptr;
    double hout[2] = {0.0, 0.0};
    cudaError_t e = cudaMallocAsync((void **)&sig, 8ull * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&B, 16ull * n * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&C, 16ull * rows * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&part, 16ull * 304, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&out, 16, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&item, sizeof(hz::GemmItem), st);
    // B = Sigma^{-1} X; C = [F'; G'] B = [U Sigma_F X; V Sigma_G X]
    if (e == cudaSuccess)
        e = hz::launch_sigma(h->W, h->Mt, h->Jrow, h->m_pad, h->p_pad, n, sig, nullptr, nullptr, nullptr, 0,
                             st);
    if (e == cudaSuccess) e = hz::launch_rowscale((const double2 *)X, ldx, n, sig, B, st);
    const hz::GemmItem it{h->W, h->Mt, rows, B, n, C, rows, n, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(item, &it, sizeof(it), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = hz::launch_gemm_batched(item, 1, rows, n, st);
    if (e == cudaSuccess)
        e = hz::launch_rel_err((const double2 *)F, ldf, C, rows, m, n, part, out, st);
    if (e == cudaSuccess)
        e = hz::launch_rel_err((const double2 *)G, ldg, C + h->m_pad, rows, p, n, part, out + 1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hout, out, 16, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(sig, st);
    if (B) cudaFreeAsync(B, st);
    if (C) cudaFreeAsync(C, st);
    if (part) cudaFreeAsync(part, st);
    if (out) cudaFreeAsync(out, st);
    if (item) cudaFreeAsync(item, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaSetDevice(prev);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return status_of(e);
    *err_f = hout[0];
    *err_g = hout[1];
    return GHSVD_OK;
}

}  // extern "C"
