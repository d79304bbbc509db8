// hz_batch.cu -- batched solves: many independent pencils of uneven order
// (k-points of an LAPW computation) advanced together, one outer step of
// every active pencil per "tick" of the Level-2 block HZ method (Section 6.4).
//
// Each pencil keeps its own working buffers, schedule (block partition and
// round-robin tables, Section 6.3, 6.4.1), transformation counters and state
// (current outer step, sweep, active flag, phase).  A tick is the Gram, inner
// and update kernels over the work items of every pencil (CTAs of inactive
// pencils return at once), and a control kernel that advances each pencil's
// step and, at the end of its sweep, applies the stopping rule of Section
// 6.1.7 to that pencil's own counters.  With the mixed schedule a tick also
// holds the complex64 instances of the three step kernels (each pencil runs
// the instance of its phase) and, first, the FP64 products W Z'_low of the
// pencils whose complex64 round ended in the previous tick.  The whole
// iteration is one launch of a CUDA graph whose conditional while node
// repeats the tick: the control kernel sets the loop condition on the
// device, and the host waits once, when no pencil is active any more.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#include "../../include/ghsvd.h"
#include "hz_gemm.cuh"
#include "hz_gram.cuh"
#include "hz_inner.cuh"
#include "hz_update.cuh"
#include "hz_delta.cuh"
#include "hz_launch.h"

namespace hz {

// Per-pencil device descriptor.
struct BPencil {
    double2 *W;                 // [ld x n] stacked F', G', Z'
    float2 *W32;                // [ld x n] complex64 copy (mixed schedule), or null
    double2 *Wtmp;              // [ld x n] product W Z'_low (mixed schedule), or null
    long long ld;               // Mt
    const int8_t *Jrow;         // [m_pad]
    const int *slot;            // [nsteps][npairs][kk]
    double2 *partial;           // [npairs][cpp][KKMAX^2]
    double2 *zhat;              // [npairs][KKMAX^2]
    int *flag;                  // [npairs]
    int *route;                 // [npairs]: FP64 update route (route_class) of this step
    unsigned long long *cnt;    // [2]: all, big of the current sweep
    int *err;                   // [2]
    int m_pad, p_pad, n_pad, n;
    int kk, npairs, nsteps, kc, chunks_h, chunks_s;
    double tol;                 // eps sqrt(n) of eq. 6.12 (FP64 sweeps)
    double tol32;               // the same with the complex64 unit roundoff
    double pivots_per_sweep;    // 2x2 pivots of one sweep
};

// Per-pencil state, advanced by the control kernel.  phase 1: complex64
// rounds of the mixed schedule, phase 0: FP64 sweeps.  pending != 0: the
// round just ended; the next tick applies Z'_low to the FP64 factors
// (1: another complex64 round follows, 2: the FP64 sweeps) and the pencil's
// step kernels skip that tick.
struct BState {
    int step, sweep, active, status;
    int phase, pending, rounds, round_sweeps, sweeps_low;
    unsigned long long prev_big;
};

// Pencils whose round ended: ctl[2] of them, listed in pend[0..), with the
// product's 64 x 64 tiles numbered from toff[j] (toff[ctl[2]] = ctl[3] tiles).

// Status codes the control kernel writes (mirror ghsvd_status).
constexpr int BST_RUNNING = -1;

template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 128 : 160, 3)
gram_batched(const BPencil *__restrict__ P, const BState *__restrict__ S, const int4 *__restrict__ work)
{
    const int4 w = work[blockIdx.x];
    const BState st = S[w.x];
    if (!st.active || st.pending || st.phase != (sizeof(T) == 4)) return;
    const BPencil &p = P[w.x];
    const int r = st.step;
    const int c = w.z;
    const bool isH = c < p.chunks_h;
    const int r0 = isH ? c * p.kc : p.m_pad + (c - p.chunks_h) * p.kc;
    const int r1 = isH ? min(r0 + p.kc, p.m_pad) : min(r0 + p.kc, p.m_pad + p.p_pad);
    const int cpp = p.chunks_h + p.chunks_s;
    using T2 = typename cplx<T>::t;
    const T2 *Wt = sizeof(T) == 8 ? (const T2 *)p.W : (const T2 *)p.W32;
    gram_body<T>(Wt, p.ld, p.Jrow, p.slot + ((long long)r * p.npairs + w.y) * p.kk, p.kk, r0, r1, isH,
                 (T2 *)p.partial + ((long long)w.y * cpp + c) * (KKMAX * KKMAX));
}

template <typename T>
__global__ void __launch_bounds__(1024)
inner_batched(const BPencil *__restrict__ P, const BState *__restrict__ S, const int4 *__restrict__ work,
              int inner_sweeps, int crit_mode, int param32)
{
    extern __shared__ unsigned char smraw_inner[];
    const int4 w = work[blockIdx.x];
    const BState st = S[w.x];
    if (!st.active || st.pending || st.phase != (sizeof(T) == 4)) return;
    const BPencil &p = P[w.x];
    const int r = st.step;
    InnerArgs a{};
    a.npairs = p.npairs;
    a.kk = p.kk;
    a.cpp = p.chunks_h + p.chunks_s;
    a.chunks_h = p.chunks_h;
    a.inner_sweeps = inner_sweeps;
    a.crit_mode = crit_mode;
    a.tol = sizeof(T) == 8 ? p.tol : p.tol32;
    a.param32 = param32;
    using T2 = typename cplx<T>::t;
    inner_body<T, T>((const T2 *)p.partial + (long long)w.y * a.cpp * (KKMAX * KKMAX),
                     p.slot + ((long long)r * p.npairs + w.y) * p.kk, a,
                     (T2 *)p.zhat + (long long)w.y * KKMAX * KKMAX, p.flag + w.y, p.cnt, p.err, smraw_inner);
}

template <typename T>
__global__ void __launch_bounds__(256)
update_batched(const BPencil *__restrict__ P, const BState *__restrict__ S, const int4 *__restrict__ work)
{
    extern __shared__ unsigned char smraw[];
    const int4 w = work[blockIdx.x];
    const BState st = S[w.x];
    if (!st.active || st.pending || st.phase != (sizeof(T) == 4)) return;
    const BPencil &p = P[w.x];
    if (!p.flag[w.y]) return;
    const int r = st.step;
    using T2 = typename cplx<T>::t;
    T2 *Wt = sizeof(T) == 8 ? (T2 *)p.W : (T2 *)p.W32;
    const int *slot = p.slot + ((long long)r * p.npairs + w.y) * p.kk;
    const long long row0 = (long long)w.z * UPD_R;
    if constexpr (sizeof(T) == 8) {
        // FP64 sweeps: the delta forms for pairs whose Z^ - I is small
        const double2 *zp = p.zhat + (long long)w.y * KKMAX * KKMAX;
        const int c = p.route[w.y];
        if (c == 0) {
            delta64_tile(p.W, p.ld, slot, p.kk, row0, zp, smraw);
            return;
        }
        if (c == 1) {
            df64_tile(p.W, p.ld, slot, p.kk, row0, zp, smraw);
            __syncthreads();                    // the first half's shared buffers are free
            df64_tile(p.W, p.ld, slot, p.kk, row0 + DF_R, zp, smraw);
            return;
        }
    }
    update_body<T, T>(Wt, p.ld, slot, p.kk, row0, (const T2 *)p.zhat + (long long)w.y * KKMAX * KKMAX, smraw);
}

// The update route of every transformed pair of the pencils in FP64 sweeps
// (route_class; 2 = the FP64 product for every pair when enable is 0).
__global__ void route_batched(const BPencil *__restrict__ P, const BState *__restrict__ S,
                              const int4 *__restrict__ work, int enable)
{
    const int4 w = work[blockIdx.x];
    const BState st = S[w.x];
    if (!st.active || st.pending || st.phase != 0) return;
    const BPencil &p = P[w.x];
    if (!p.flag[w.y]) return;
    const int c = enable ? route_class(p.zhat + (long long)w.y * KKMAX * KKMAX, p.kk) : 2;
    if (threadIdx.x == 0) p.route[w.y] = c;
}

// The round products W_i Z'_low,i -> Wtmp_i of the pencils listed in pend
// (Z'_low: the complex64 rows of Z' in W32), one 64 x 64 tile per CTA
// iteration over all their tiles.
__global__ void __launch_bounds__(256)
round_product_batched(const BPencil *__restrict__ P, const int *__restrict__ ctl, const int *__restrict__ pend,
                      const int *__restrict__ toff)
{
    const int np = ctl[2], total = ctl[3];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int j = 0;
        while (j + 1 < np && toff[j + 1] <= t) ++j;
        const BPencil &p = P[pend[j]];
        const int local = t - toff[j];
        const int rt = (int)(p.ld / 64);
        const long long row0 = (long long)(local % rt) * 64;
        const int col0 = (local / rt) * 64;
        const float2 *zlow = p.W32 + (p.m_pad + p.p_pad);
        gemm_tile_3m<float2>(p.W, p.ld, zlow, p.ld, p.Wtmp, p.ld, p.n, row0, col0);
    }
}

// After the products: W_i <- Wtmp_i, and for a pencil that starts another
// complex64 round W32_i <- fl32(W_i) with Z' reset to I (pending 1).
__global__ void round_finish_batched(const BPencil *__restrict__ P, const BState *__restrict__ S,
                                     const int *__restrict__ ctl, const int *__restrict__ pend)
{
    const int np = ctl[2];
    for (int j = blockIdx.y; j < np; j += gridDim.y) {
        const int i = pend[j];
        const BPencil &p = P[i];
        const bool again = S[i].pending == 1;
        const long long total = p.ld * p.n;
        const long long z0 = p.m_pad + p.p_pad;
        for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
             e += (long long)gridDim.x * blockDim.x) {
            const double2 v = p.Wtmp[e];
            p.W[e] = v;
            if (again) {
                const long long r = e % p.ld, c = e / p.ld;
                float2 f = make_float2((float)v.x, (float)v.y);
                if (r >= z0) f = make_float2((r - z0) == c ? 1.0f : 0.0f, 0.0f);
                p.W32[e] = f;
            }
        }
    }
}

// One thread per pencil: advance the step; at the end of a sweep apply the
// stopping rule (no big transformation, Section 6.1.7) or C_max, record the
// sweep's counts, reset the counters.  ctl[0] = pencils still running,
// ctl[1] = ticks run.  Inside the solve's graph (loop != 0) the kernel also
// decides on the device whether the graph's while loop runs another tick:
// while some pencil is active and fewer than max_ticks ticks have run.
//
// Mixed schedule (the rules of the single solve): a complex64 round ends when
// its big count levels off (more than 0.8 of the previous sweep's and below
// 10 % of the pivots), when no pivot rotated, or at the complex64 sweep
// budget; the pencil then waits one tick for the product W Z'_low and either
// starts another round (at most two) or continues with FP64 sweeps.  The
// pencils waiting for a product are listed for the next tick.
__global__ void control_batched(const BPencil *__restrict__ P, BState *__restrict__ S, int batch,
                                int max_sweeps, int mixed_max_sweeps, long long *__restrict__ hist,
                                int hist_len, int *__restrict__ ctl, int *__restrict__ pend,
                                int *__restrict__ toff, cudaGraphConditionalHandle loop_handle, int loop,
                                long long max_ticks)
{
    constexpr int kMaxRounds = 2;
    __shared__ int count;
    if (threadIdx.x == 0) count = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < batch; i += blockDim.x) {
        BState st = S[i];
        if (st.active) {
            const BPencil &p = P[i];
            if (st.pending) {
                // this tick applied the round's product: resume
                if (st.pending == 2) st.phase = 0;
                st.pending = 0;
                st.round_sweeps = 0;
                st.prev_big = ~0ULL;
            } else if (p.err[0] & DEVERR_RANK) { st.active = 0; st.status = GHSVD_ERR_RANK_DEFICIENT; }
            else if (p.err[0] & DEVERR_NONFINITE) { st.active = 0; st.status = GHSVD_ERR_NONFINITE; }
            else if (st.step == p.nsteps - 1) {
                const unsigned long long all = p.cnt[0], big = p.cnt[1];
                if (st.sweep < hist_len) {
                    hist[((long long)i * hist_len + st.sweep) * 2] = (long long)all;
                    hist[((long long)i * hist_len + st.sweep) * 2 + 1] = (long long)big;
                }
                st.sweep += 1;
                p.cnt[0] = 0;
                p.cnt[1] = 0;
                st.step = 0;
                if (st.phase == 1) {
                    st.sweeps_low += 1;
                    st.round_sweeps += 1;
                    const bool plateau = st.round_sweeps >= 2 && (double)big > 0.8 * (double)st.prev_big &&
                                         (double)big < 0.1 * p.pivots_per_sweep;
                    st.prev_big = big;
                    const bool budget = st.sweeps_low >= mixed_max_sweeps;
                    if (all == 0 || plateau || budget) {
                        st.rounds += 1;
                        st.pending = (budget || all == 0 || st.round_sweeps <= 3 || st.rounds >= kMaxRounds) ? 2 : 1;
                    }
                    if (st.sweep >= max_sweeps && !st.pending) { st.active = 0; st.status = GHSVD_ERR_NOT_CONVERGED; }
                } else if (big == 0) { st.active = 0; st.status = GHSVD_OK; }
                else if (st.sweep >= max_sweeps) { st.active = 0; st.status = GHSVD_ERR_NOT_CONVERGED; }
            } else {
                st.step += 1;
            }
            S[i] = st;
        }
        if (st.active) atomicAdd(&count, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // the pencils whose round just ended, with the tile offsets of their products
        int np = 0, tiles = 0;
        for (int i = 0; i < batch; ++i) {
            if (!S[i].active || !S[i].pending) continue;
            const BPencil &p = P[i];
            pend[np] = i;
            toff[np] = tiles;
            tiles += (int)(p.ld / 64) * ((p.n + 63) / 64);
            ++np;
        }
        toff[np] = tiles;
        ctl[2] = np;
        ctl[3] = tiles;
        ctl[0] = count;
        const int ticks = ctl[1] + 1;
        ctl[1] = ticks;
        if (loop) cudaGraphSetConditional(loop_handle, (count > 0 && ticks < max_ticks) ? 1u : 0u);
    }
}

__global__ void state_init(const BPencil *__restrict__ P, BState *S, int batch)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < batch) {
        BState st{};
        st.active = 1;
        st.status = BST_RUNNING;
        st.phase = P[i].W32 != nullptr;
        st.prev_big = ~0ULL;
        S[i] = st;
    }
}

}  // namespace hz

using hz::BPencil;
using hz::BState;

namespace {

long long rup(long long x, long long r) { return (x + r - 1) / r * r; }
long long a256(long long x) { return rup(x, 256); }

// Host-side plan of one pencil.
struct PlanP {
    int m, p, n, m_pad, p_pad, n_pad, nb, wb, kk, npairs, nsteps, kc, chunks_h, chunks_s;
    long long Mt;
    long long oW, oPart, oZhat, oFlag, oRoute, oSlot, oJrow, oCnt, oErr, oLam, oGsc, oVn, oGc, oKap, oRank;
    long long oTmp;             // W V0 (warm start) or W Z'_low (mixed schedule), or -1
    long long oW32;             // complex64 copy of W (mixed schedule), or -1
    int mixed;                  // this pencil runs the mixed schedule
};

struct Plan {
    int w;
    std::vector<PlanP> pp;
    long long bytes;
    long long oItems;           // GemmItem[batch] for the warm-start products
    long long oKap0;            // double[batch]: condition estimates of the V0
    int gram_work, inner_work, update_work;
};

int partition(int n, int w, std::vector<int> &off)
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

Plan make_plan(int batch, const int64_t *m, const int64_t *p, const int64_t *n, int w, int sms,
               const void *const *V0, bool mixed)
{
    const bool with_v0 = V0 != nullptr;
    Plan pl;
    pl.w = w;
    pl.bytes = 0;
    pl.gram_work = pl.inner_work = pl.update_work = 0;
    // one Gram row chunk for the whole batch: about 4 Gram CTAs per SM per tick
    long long pair_rows = 0;
    for (int i = 0; i < batch; ++i) {
        std::vector<int> off;
        const int nbi = partition((int)n[i], std::min<int>(w, (int)n[i]), off);
        pair_rows += (long long)(nbi / 2) * (rup(m[i], hz::ROWPAD) + rup(p[i], hz::ROWPAD));
    }
    // (the complex64 sweeps of the mixed schedule sum their Gram partials in
    // FP32: chunks of at most 512 rows keep that rounding noise near the
    // single-pencil solve's, so that their rounds level off as there)
    const long long kc_cap = mixed ? 512 : 4096;
    const int kc_all = (int)std::min<long long>(kc_cap, std::max<long long>(256, rup(pair_rows / (4LL * sms), 64)));
    for (int i = 0; i < batch; ++i) {
        PlanP q{};
        q.m = (int)m[i]; q.p = (int)p[i]; q.n = (int)n[i];
        q.m_pad = (int)rup(q.m, hz::ROWPAD); q.p_pad = (int)rup(q.p, hz::ROWPAD);
        q.n_pad = (int)rup(q.n, hz::ROWPAD);
        q.Mt = (long long)q.m_pad + q.p_pad + q.n_pad;
        std::vector<int> off;
        q.nb = partition(q.n, std::min(w, q.n), off);
        q.wb = off[1] - off[0];
        q.kk = 2 * q.wb;
        q.npairs = q.nb / 2;
        q.nsteps = q.nb - 1;
        q.kc = kc_all;
        q.chunks_h = (q.m_pad + q.kc - 1) / q.kc;
        q.chunks_s = (q.p_pad + q.kc - 1) / q.kc;
        const int cpp = q.chunks_h + q.chunks_s;
        auto carve = [&](long long b) { long long at = pl.bytes; pl.bytes += a256(b); return at; };
        q.oW = carve(16LL * q.Mt * q.n);
        q.oPart = carve(16LL * q.npairs * cpp * hz::KKMAX * hz::KKMAX);
        q.oZhat = carve(16LL * q.npairs * hz::KKMAX * hz::KKMAX);
        q.oFlag = carve(4LL * q.npairs);
        q.oRoute = carve(4LL * q.npairs);
        q.oSlot = carve(4LL * q.nsteps * q.npairs * q.kk);
        q.oJrow = carve(q.m_pad);
        q.oCnt = carve(16);
        q.oErr = carve(8);
        q.oLam = carve(8LL * q.n); q.oGsc = carve(8LL * q.n); q.oVn = carve(8LL * q.n);
        q.oGc = carve(8LL * q.n); q.oKap = carve(8); q.oRank = carve(4LL * q.n);
        // the mixed schedule for every pencil (a starting basis is applied first)
        q.mixed = mixed && q.n >= 2;
        q.oTmp = (with_v0 || q.mixed) ? carve(16LL * q.Mt * q.n) : -1;
        q.oW32 = q.mixed ? carve(8LL * q.Mt * q.n) : -1;
        pl.gram_work += q.npairs * cpp;
        pl.inner_work += q.npairs;
        pl.update_work += q.npairs * (int)(q.Mt / hz::UPD_R);
        pl.pp.push_back(q);
    }
    pl.oItems = pl.bytes;
    pl.bytes += a256((long long)sizeof(hz::GemmItem) * 2 * batch);   // products, then two copies each
    pl.oKap0 = pl.bytes;
    pl.bytes += a256(8LL * batch);
    return pl;
}

}  // namespace

// Batched working memory, owned by a handle and reused between calls.
struct BatchBuffers {
    unsigned char *arena = nullptr;
    long long arena_bytes = 0;
    BPencil *d_pen = nullptr;
    BState *d_state = nullptr;
    int4 *d_work = nullptr;
    long long *d_hist = nullptr;
    int *d_active = nullptr;            // ctl[4]: active pencils, ticks, pending pencils, their tiles
    int *d_pend = nullptr;              // [batch] pending pencils, [batch + 1] their tile offsets
    int cap_batch = 0;
    long long cap_work = 0;
};

static void free_batch(BatchBuffers &b)
{
    cudaFree(b.arena); cudaFree(b.d_pen); cudaFree(b.d_state); cudaFree(b.d_work);
    cudaFree(b.d_hist); cudaFree(b.d_active); cudaFree(b.d_pend);
    b = BatchBuffers();
}

#define BT_TRY(x)                                               \
    do {                                                        \
        cudaError_t e_ = (x);                                   \
        if (e_ != cudaSuccess) {                                \
            free_batch(bb);                                     \
            return e_ == cudaErrorMemoryAllocation ? GHSVD_ERR_NOMEM : GHSVD_ERR_CUDA; \
        }                                                       \
    } while (0)

constexpr int kHistLen = 64;

// Set up the working buffers of every pencil for plan pl (copy-in, signs,
// schedule); returns the device descriptors.
static ghsvd_status setup_batch(BatchBuffers &bb, const Plan &pl, int batch, const void *const *F,
                                const int64_t *ldf, const int8_t *const *J, const int64_t *n_plus,
                                const void *const *G, const int64_t *ldg, const void *const *V0,
                                const int64_t *ldv0, cudaStream_t st, double tol_scale,
                                double *ms_v0 = nullptr)
{
    if (pl.bytes > bb.arena_bytes) {
        cudaFree(bb.arena);
        bb.arena = nullptr;
        bb.arena_bytes = 0;
        BT_TRY(cudaMalloc((void **)&bb.arena, pl.bytes));
        bb.arena_bytes = pl.bytes;
    }
    if (batch > bb.cap_batch) {
        cudaFree(bb.d_pen); cudaFree(bb.d_state); cudaFree(bb.d_hist); cudaFree(bb.d_pend);
        bb.d_pen = nullptr; bb.d_state = nullptr; bb.d_hist = nullptr; bb.d_pend = nullptr;
        BT_TRY(cudaMalloc((void **)&bb.d_pen, sizeof(BPencil) * batch));
        BT_TRY(cudaMalloc((void **)&bb.d_state, sizeof(BState) * batch));
        BT_TRY(cudaMalloc((void **)&bb.d_hist, sizeof(long long) * 2 * kHistLen * batch));
        BT_TRY(cudaMalloc((void **)&bb.d_pend, sizeof(int) * (2 * batch + 1)));
        bb.cap_batch = batch;
    }
    if (!bb.d_active) BT_TRY(cudaMalloc((void **)&bb.d_active, 4 * sizeof(int)));
    BT_TRY(cudaMemsetAsync(bb.d_active, 0, 4 * sizeof(int), st));
    const long long nwork = (long long)pl.gram_work + pl.inner_work + pl.update_work;
    if (nwork > bb.cap_work) {
        cudaFree(bb.d_work);
        bb.d_work = nullptr;
        BT_TRY(cudaMalloc((void **)&bb.d_work, sizeof(int4) * nwork));
        bb.cap_work = nwork;
    }
    std::vector<BPencil> hp(batch);
    std::vector<int4> work;
    work.reserve(nwork);
    for (int i = 0; i < batch; ++i) {
        const PlanP &q = pl.pp[i];
        unsigned char *base = bb.arena;
        BPencil d{};
        d.W = (double2 *)(base + q.oW);
        d.ld = q.Mt;
        d.Jrow = (const int8_t *)(base + q.oJrow);
        d.slot = (const int *)(base + q.oSlot);
        d.partial = (double2 *)(base + q.oPart);
        d.zhat = (double2 *)(base + q.oZhat);
        d.flag = (int *)(base + q.oFlag);
        d.route = (int *)(base + q.oRoute);
        d.cnt = (unsigned long long *)(base + q.oCnt);
        d.err = (int *)(base + q.oErr);
        d.m_pad = q.m_pad; d.p_pad = q.p_pad; d.n_pad = q.n_pad; d.n = q.n;
        d.kk = q.kk; d.npairs = q.npairs; d.nsteps = q.nsteps; d.kc = q.kc;
        d.chunks_h = q.chunks_h; d.chunks_s = q.chunks_s;
        d.tol = tol_scale * ldexp(1.0, -53) * sqrt((double)q.n);
        d.tol32 = tol_scale * ldexp(1.0, -24) * sqrt((double)q.n);
        d.pivots_per_sweep = (double)q.nsteps * q.npairs * (q.kk / 2) * (q.kk - 1);
        d.W32 = q.mixed ? (float2 *)(base + q.oW32) : nullptr;
        d.Wtmp = q.oTmp >= 0 ? (double2 *)(base + q.oTmp) : nullptr;
        hp[i] = d;
        // schedule tables (host-built, as for a single pencil)
        std::vector<int> off;
        partition(q.n, std::min(pl.w, q.n), off);
        std::vector<int> tab((size_t)q.nsteps * q.npairs * q.kk, -1);
        for (int r = 0; r < q.nsteps; ++r)
            for (int k = 0; k < q.npairs; ++k) {
                int P, Q;
                hz::rr_pair(q.nb, r, k, &P, &Q);
                int *row = &tab[((size_t)r * q.npairs + k) * q.kk];
                for (int c = off[P]; c < off[P + 1]; ++c) row[c - off[P]] = c;
                for (int c = off[Q]; c < off[Q + 1]; ++c) row[q.wb + c - off[Q]] = c;
            }
        BT_TRY(cudaMemcpyAsync((void *)d.slot, tab.data(), sizeof(int) * tab.size(),
                               cudaMemcpyHostToDevice, st));
        BT_TRY(cudaMemsetAsync(d.cnt, 0, 16, st));
        BT_TRY(cudaMemsetAsync(d.err, 0, 8, st));
        BT_TRY(cudaMemsetAsync(d.flag, 0, 4LL * q.npairs, st));
        BT_TRY(hz::launch_signs((int8_t *)d.Jrow, J ? J[i] : nullptr, q.m, q.m_pad,
                                n_plus ? n_plus[i] : q.m, d.err + 1, st));
        BT_TRY(hz::launch_copyin(d.W, false, q.Mt, q.m, q.p, q.n, q.m_pad, q.p_pad, q.n_pad, F[i],
                                 ldf[i], G[i], ldg[i], nullptr, 0, d.err, st));
        BT_TRY(hz::launch_gnorm(d.W, q.Mt, q.m_pad, q.p_pad, q.n, (double *)(base + q.oGc), st));
    }
    // warm starts: (F V0, G V0) with Z' = V0 for every pencil that has a V0,
    // as one batched FP64 product and one batched copy
    if (V0) {
        std::vector<hz::GemmItem> items, back, probe;
        long long max_rows = 0;
        int max_n = 0;
        hz::GemmItem *d_items = (hz::GemmItem *)(bb.arena + pl.oItems);
        double *d_kap = (double *)(bb.arena + pl.oKap0);
        // condition estimate of every basis: compensated products only where needed
        for (int i = 0; i < batch; ++i)
            if (V0[i])
                probe.push_back({(const double2 *)V0[i], ldv0[i], pl.pp[i].n,
                                 (const double2 *)(bb.arena + pl.pp[i].oGc), 0, nullptr, 0,
                                 pl.pp[i].n, 0});
        std::vector<double> kap(probe.size(), 0.0);
        if (!probe.empty()) {
            BT_TRY(cudaMemcpyAsync(d_items, probe.data(), sizeof(hz::GemmItem) * probe.size(),
                                   cudaMemcpyHostToDevice, st));
            BT_TRY(hz::launch_v0_kappa(d_items, (int)probe.size(), d_kap, st));
            BT_TRY(cudaMemcpyAsync(kap.data(), d_kap, 8 * kap.size(), cudaMemcpyDeviceToHost, st));
            BT_TRY(cudaStreamSynchronize(st));
        }
        size_t kidx = 0;
        for (int i = 0; i < batch; ++i) {
            if (!V0[i]) continue;
            const PlanP &q = pl.pp[i];
            double2 *Wi = (double2 *)(bb.arena + q.oW);
            double2 *Ti = (double2 *)(bb.arena + q.oTmp);
            const int acc = !(kap[kidx++] <= hz::WARM_ACCURATE_KAPPA);
            // the rows of F and G only; the rows of Z' (= I) become V0 itself
            const long long fg = (long long)q.m_pad + q.p_pad;
            items.push_back({Wi, q.Mt, fg, (const double2 *)V0[i], ldv0[i], Ti, q.Mt, q.n, acc});
            back.push_back({Ti, q.Mt, fg, nullptr, 0, Wi, q.Mt, q.n, 0});
            back.push_back({(const double2 *)V0[i], ldv0[i], q.n, nullptr, 0, Wi + fg, q.Mt, q.n, 0});
            max_rows = std::max(max_rows, fg);
            max_n = std::max(max_n, q.n);
        }
        if (!items.empty()) {
            auto tv = std::chrono::steady_clock::now();
            BT_TRY(cudaMemcpyAsync(d_items, items.data(), sizeof(hz::GemmItem) * items.size(),
                                   cudaMemcpyHostToDevice, st));
            BT_TRY(hz::launch_gemm_batched(d_items, (int)items.size(), max_rows, max_n, st));
            BT_TRY(cudaMemcpyAsync(d_items, back.data(), sizeof(hz::GemmItem) * back.size(),
                                   cudaMemcpyHostToDevice, st));
            BT_TRY(hz::launch_copy_batched(d_items, (int)back.size(), st));
            if (ms_v0) {
                BT_TRY(cudaStreamSynchronize(st));
                *ms_v0 = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tv).count();
            }
        }
    }
    // the first complex64 round of a pencil on the mixed schedule starts from
    // fl32(W) (after its starting basis, if any) with Z' = I
    for (int i = 0; i < batch; ++i) {
        const PlanP &q = pl.pp[i];
        if (!q.mixed) continue;
        BT_TRY(hz::launch_convert(hp[i].W32, true, hp[i].W, q.Mt * q.n, st));
        BT_TRY(hz::launch_eye32(hp[i].W32, q.Mt, q.m_pad + q.p_pad, q.n, q.n_pad, st));
    }
    for (int i = 0; i < batch; ++i) {
        const PlanP &q = pl.pp[i];
        const int cpp = q.chunks_h + q.chunks_s;
        for (int k = 0; k < q.npairs; ++k)
            for (int c = 0; c < cpp; ++c) work.push_back(make_int4(i, k, c, 0));
    }
    for (int i = 0; i < batch; ++i)
        for (int k = 0; k < pl.pp[i].npairs; ++k) work.push_back(make_int4(i, k, 0, 0));
    for (int i = 0; i < batch; ++i) {
        const PlanP &q = pl.pp[i];
        for (int t = 0; t < (int)(q.Mt / hz::UPD_R); ++t)
            for (int k = 0; k < q.npairs; ++k) work.push_back(make_int4(i, k, t, 0));
    }
    BT_TRY(cudaMemcpyAsync(bb.d_pen, hp.data(), sizeof(BPencil) * batch, cudaMemcpyHostToDevice, st));
    BT_TRY(cudaMemcpyAsync(bb.d_work, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice,
                           st));
    BT_TRY(cudaMemsetAsync(bb.d_hist, 0, sizeof(long long) * 2 * kHistLen * batch, st));
    hz::state_init<<<(batch + 127) / 128, 128, 0, st>>>(bb.d_pen, bb.d_state, batch);
    BT_TRY(cudaGetLastError());
    return GHSVD_OK;
}

static cudaError_t enqueue_tick(const BatchBuffers &bb, const Plan &pl, int batch, const ghsvd_opts &o,
                                int max_sweeps, cudaStream_t st, cudaGraphConditionalHandle loop_handle = 0,
                                int loop = 0, long long max_ticks = 0)
{
    const int4 *wg = bb.d_work;
    const int4 *wi = wg + pl.gram_work;
    const int4 *wu = wi + pl.inner_work;
    int kkmax = 2;
    bool mixed = false;
    for (const PlanP &q : pl.pp) {
        kkmax = std::max(kkmax, q.kk);
        mixed |= q.mixed != 0;
    }
    int *pend = bb.d_pend, *toff = bb.d_pend + batch;
    if (mixed) {
        // the products of the rounds that ended in the previous tick
        int sms = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        hz::round_product_batched<<<2 * sms, 256, 0, st>>>(bb.d_pen, bb.d_active, pend, toff);
        hz::round_finish_batched<<<dim3(64, std::min(batch, 64)), 256, 0, st>>>(bb.d_pen, bb.d_state, bb.d_active,
                                                                               pend);
    }
    hz::gram_batched<double><<<pl.gram_work, hz::gram_threads_c128(kkmax), 0, st>>>(bb.d_pen, bb.d_state, wg);
    if (mixed)
        hz::gram_batched<float><<<pl.gram_work, hz::gram_threads(kkmax), 0, st>>>(bb.d_pen, bb.d_state, wg);
    hz::inner_batched<double><<<pl.inner_work, 1024, hz::inner_smem_bytes(sizeof(double2)), st>>>(
        bb.d_pen, bb.d_state, wi, o.inner_sweeps, o.crit_mode, 0);
    if (mixed)
        hz::inner_batched<float><<<pl.inner_work, 1024, hz::inner_smem_bytes(sizeof(float2)), st>>>(
            bb.d_pen, bb.d_state, wi, o.inner_sweeps, o.crit_mode, o.mixed_param32);
    hz::route_batched<<<pl.inner_work, 256, 0, st>>>(bb.d_pen, bb.d_state, wi, o.delta_update);
    hz::update_batched<double><<<pl.update_work, 256, hz::update_smem(sizeof(double2)), st>>>(
        bb.d_pen, bb.d_state, wu);
    if (mixed)
        hz::update_batched<float><<<pl.update_work, 256, hz::update_smem(sizeof(float2)), st>>>(
            bb.d_pen, bb.d_state, wu);
    hz::control_batched<<<1, 128, 0, st>>>(bb.d_pen, bb.d_state, batch, max_sweeps, o.mixed_max_sweeps, bb.d_hist, kHistLen,
                                           bb.d_active, pend, toff, loop_handle, loop, max_ticks);
    return cudaGetLastError();
}

static cudaError_t batch_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(hz::inner_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)hz::inner_smem_bytes(sizeof(double2)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(hz::inner_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)hz::inner_smem_bytes(sizeof(float2)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(hz::update_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)hz::update_smem(sizeof(double2)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(hz::update_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)hz::update_smem(sizeof(float2)));
    return e;
}

// Run ticks until no pencil is active, as one graph launch: the graph is a
// conditional while node whose body is one tick (Gram, inner level, update,
// control); the control kernel sets the loop condition on the device, so the
// host waits once for the whole solve.  Returns the number of ticks run.
static ghsvd_status run_ticks(BatchBuffers &bb, const Plan &pl, int batch, const ghsvd_opts &o,
                              cudaStream_t st, long long max_ticks, long long *ticks_out)
{
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraphConditionalHandle handle = 0;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = handle;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t ec = enqueue_tick(bb, pl, batch, o, o.max_sweeps, cs, handle, 1, max_ticks);
            cudaGraph_t captured = nullptr;
            e = cudaStreamEndCapture(cs, &captured);
            if (e == cudaSuccess) e = ec;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    int ctl[2] = {batch, 0};
    if (e == cudaSuccess) e = cudaMemsetAsync(bb.d_active + 1, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctl, bb.d_active, sizeof(ctl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    if (ticks_out) *ticks_out = ctl[1];
    if (e != cudaSuccess) return GHSVD_ERR_CUDA;
    return GHSVD_OK;
}

void *hz_batch_new() { return new (std::nothrow) BatchBuffers(); }

void hz_batch_free(void *p)
{
    if (!p) return;
    BatchBuffers *b = (BatchBuffers *)p;
    free_batch(*b);
    delete b;
}

ghsvd_status hz_batch_solve(void *buffers, int device, const ghsvd_opts *opts, int batch, const int64_t *m,
                            const int64_t *p, const int64_t *n, const void *const *F, const int64_t *ldf,
                            const int8_t *const *J, const int64_t *n_plus, const void *const *G,
                            const int64_t *ldg, const void *const *V0, const int64_t *ldv0,
                            double *const *lambda, void *const *V, const int64_t *ldv, int *sweeps, int *status,
                            HzBatchInfo *info, void *stream)
{
    BatchBuffers &bb = *(BatchBuffers *)buffers;
    const ghsvd_opts &o = *opts;
    const bool mixed = o.precision == GHSVD_PRECISION_MIXED;
    HzBatchInfo dummy{};
    if (!info) info = &dummy;
    *info = HzBatchInfo{};
    cudaStream_t st = (cudaStream_t)stream;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return GHSVD_ERR_CUDA;
    if (batch_attributes() != cudaSuccess) return GHSVD_ERR_CUDA;

    // block width: given, or autotuned from a few timed ticks per candidate
    int w = o.block_width;
    if (w <= 0) {
        const int cands[] = {8, 16, 32};
        double best = 1e300;
        w = 32;
        for (int c : cands) {
            Plan pl = make_plan(batch, m, p, n, c, sms, V0, mixed);
            ghsvd_status s = setup_batch(bb, pl, batch, F, ldf, J, n_plus, G, ldg, V0, ldv0, st, opts->tol_scale);
            if (s != GHSVD_OK) return s;
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            const int probe = 4;
            // warm-up tick, then time `probe` ticks
            enqueue_tick(bb, pl, batch, o, 1 << 30, st);
            cudaEventRecord(e0, st);
            for (int t = 0; t < probe; ++t) enqueue_tick(bb, pl, batch, o, 1 << 30, st);
            cudaEventRecord(e1, st);
            cudaError_t e = cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (e != cudaSuccess) return GHSVD_ERR_CUDA;
            // time of one sweep of every pencil ~ ticks per sweep x tick time
            int tps = 0;
            for (const PlanP &q : pl.pp) tps = std::max(tps, q.nsteps);
            const double sweep_ms = (double)ms / probe * tps;
            if (sweep_ms < best) { best = sweep_ms; w = c; }
        }
    }
    info->w_chosen = w;
    Plan pl = make_plan(batch, m, p, n, w, sms, V0, mixed);
    auto t0 = std::chrono::steady_clock::now();
    ghsvd_status s = setup_batch(bb, pl, batch, F, ldf, J, n_plus, G, ldg, V0, ldv0, st, opts->tol_scale,
                                 &info->ms_v0);
    if (s != GHSVD_OK) return s;
    // bad J entries or non-finite inputs
    std::vector<int> herr(2 * batch, 0);
    for (int i = 0; i < batch; ++i)
        if (cudaMemcpyAsync(&herr[2 * i], bb.arena + pl.pp[i].oErr, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return GHSVD_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GHSVD_ERR_CUDA;
    for (int i = 0; i < batch; ++i) {
        if (herr[2 * i + 1]) return GHSVD_ERR_INVALID_ARG;
        if (herr[2 * i] & hz::DEVERR_NONFINITE) return GHSVD_ERR_NONFINITE;
    }
    long long max_ticks = 0;
    for (const PlanP &q : pl.pp) max_ticks = std::max<long long>(max_ticks, (long long)q.nsteps * o.max_sweeps);
    long long ticks = 0;
    // + one tick per round product of the mixed schedule
    s = run_ticks(bb, pl, batch, o, st, max_ticks + 16, &ticks);
    if (s != GHSVD_OK) return s;
    info->ticks = ticks;
    std::vector<BState> hs(batch);
    if (cudaMemcpyAsync(hs.data(), bb.d_state, sizeof(BState) * batch, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return GHSVD_ERR_CUDA;
    // outputs per pencil (Section 6.1.7)
    for (int i = 0; i < batch; ++i) {
        const PlanP &q = pl.pp[i];
        unsigned char *b = bb.arena;
        cudaError_t e = hz::launch_finalize(
            (const double2 *)(b + q.oW), q.Mt, (const int8_t *)(b + q.oJrow), q.m_pad, q.p_pad, q.n,
            o.sort_ascending, (double *)(b + q.oLam), (double *)(b + q.oGsc), (double *)(b + q.oVn),
            (const double *)(b + q.oGc), (double *)(b + q.oKap), (int *)(b + q.oRank), lambda[i],
            V ? (double2 *)V[i] : nullptr, ldv ? ldv[i] : q.n, (int *)(b + q.oErr), st);
        if (e != cudaSuccess) return GHSVD_ERR_CUDA;
    }
    for (int i = 0; i < batch; ++i)
        if (cudaMemcpyAsync(&herr[2 * i], bb.arena + pl.pp[i].oErr, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return GHSVD_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GHSVD_ERR_CUDA;
    info->ms_solve = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    ghsvd_status worst = GHSVD_OK;
    for (int i = 0; i < batch; ++i) {
        int stt = hs[i].status;
        if (stt == hz::BST_RUNNING) stt = GHSVD_ERR_NOT_CONVERGED;
        if (herr[2 * i] & hz::DEVERR_RANK) stt = GHSVD_ERR_RANK_DEFICIENT;
        if (herr[2 * i] & hz::DEVERR_NONFINITE) stt = GHSVD_ERR_NONFINITE;
        if (status) status[i] = stt;
        if (sweeps) sweeps[i] = hs[i].sweep;
        info->sweeps_low += hs[i].sweeps_low;
        info->rounds_low += hs[i].rounds;
        if (stt != GHSVD_OK && (worst == GHSVD_OK || worst == GHSVD_ERR_NOT_CONVERGED))
            worst = (ghsvd_status)stt;
    }
    return worst;
}
