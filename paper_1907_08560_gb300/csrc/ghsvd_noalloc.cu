// ghsvd_noalloc.cu -- ghsvd_solve_noalloc: the FP64 solve without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Some callers cannot allocate device memory at the time they solve: a host
// application whose memory pool has already reserved the whole device, or
// code that by its own rules may not allocate after start-up (real-time or
// certified code paths).  This entry point runs the same kernels as
// ghsvd_solve, but every working buffer -- the stacked factors, the split-K
// Gram partials, the block transformations, the schedule, the counters --
// lives in one file-scope device array of GHSVD_NOALLOC_SCRATCH_BYTES bytes.
// Every GPU that loads this library holds that array until the process
// exits.  The caller still passes its inputs and outputs.
//
// The array is shared by every call and keeps the last call's contents; each
// call clears what must start at zero (counters, flags).  Calls that overlap
// on the GPU (on different streams, or from different host threads) race on
// the array: the caller must order them.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <mutex>

#include "../../include/ghsvd.h"
#include "hz_launch.h"
#include "hz_pivot.cuh"

namespace {

// The scratch array.  In host code its name is only a stand-in for the
// device symbol: host code must use the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[GHSVD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};   // device address of g_scratch, per device
bool g_ready[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// array and the kernels' shared-memory limits.
ghsvd_status setup_device(int dev, unsigned char **base)
{
    if (dev < 0 || dev >= kMaxDevices) return GHSVD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_ready[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || ptr == nullptr) return GHSVD_ERR_CUDA;
        e = hz::setup_kernels();
        if (e != cudaSuccess) return GHSVD_ERR_CUDA;
        g_scratch_ptr[dev] = ptr;
        g_ready[dev] = true;
    }
    *base = (unsigned char *)g_scratch_ptr[dev];
    return GHSVD_OK;
}

long long align256(long long x) { return (x + 255) / 256 * 256; }

// Slot table of the round-robin block schedule, built on the device: step r,
// pair k, slot s -> column, with block b at offset b (wb - 1) + min(b, wide)
// and width wb for b < wide, wb - 1 otherwise (the partition of Section 6.4.1).
__global__ void noalloc_slots_kernel(int *slotcol, int nb, int wb, int wide)
{
    const int kk = 2 * wb, np = nb / 2;
    const int total = (nb - 1) * np * kk;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += gridDim.x * blockDim.x) {
        const int s = idx % kk, k = (idx / kk) % np, r = idx / (kk * np);
        int P, Q;
        hz::rr_pair(nb, r, k, &P, &Q);
        const int b = s < wb ? P : Q;
        const int j = s < wb ? s : s - wb;
        const int off = b * (wb - 1) + min(b, wide);
        const int width = b < wide ? wb : wb - 1;
        slotcol[idx] = j < width ? off + j : -1;
    }
}

}  // namespace

extern "C" ghsvd_status ghsvd_solve_noalloc(int64_t m64, int64_t p64, int64_t n64, const void *F,
                                            int64_t ldf, const int8_t *J, int64_t n_plus,
                                            const void *G, int64_t ldg, double *lambda, void *V,
                                            int64_t ldv, const ghsvd_opts *opts, int *sweeps_out,
                                            void *stream)
{
    auto t0 = std::chrono::steady_clock::now();
    if (sweeps_out) *sweeps_out = 0;             // written on every return
    ghsvd_opts o;
    if (opts) o = *opts;
    else ghsvd_default_opts(&o);
    if (o.block_width == 0) o.block_width = 32;  // automatic: 32 for one pencil
    if (!F || !G || !lambda) return GHSVD_ERR_INVALID_ARG;
    if (n64 < 1 || m64 < n64 || p64 < n64 || ldf < m64 || ldg < p64 || (V && ldv < n64))
        return GHSVD_ERR_INVALID_ARG;
    if (!J && (n_plus < 0 || n_plus > m64)) return GHSVD_ERR_INVALID_ARG;
    if (m64 > (1 << 24) || p64 > (1 << 24) || n64 > (1 << 16)) return GHSVD_ERR_SCRATCH_TOO_SMALL;
    // shorten (Phase 2) needs working memory of its own: not available here
    if (o.block_width < 1 || o.block_width > hz::KKMAX / 2 || o.inner_sweeps < 1 ||
        o.inner_sweeps > 30 || o.max_sweeps < 1 || o.max_sweeps > 1000 ||
        (o.crit_mode != 0 && o.crit_mode != 1) || o.precision != GHSVD_PRECISION_FP64 ||
        o.ordering != GHSVD_ORDER_ROUND_ROBIN || o.shorten != 0 || o.timeout_ms < 0 ||
        o.gram_chunk < 0 || !(o.tol_scale > 0.0 && o.tol_scale < 1e300))
        return GHSVD_ERR_INVALID_ARG;
    const int m = (int)m64, p = (int)p64, n = (int)n64;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GHSVD_ERR_CUDA;
    // every pointer, J included, must be device memory of the current device;
    // checked before anything is queued or the shared array is touched
    cudaPointerAttributes pa;
    for (const void *ptr : {F, G, (const void *)lambda, (const void *)V, (const void *)J}) {
        if (!ptr) continue;
        if (cudaPointerGetAttributes(&pa, ptr) != cudaSuccess || pa.type != cudaMemoryTypeDevice ||
            pa.device != dev) {
            cudaGetLastError();
            return GHSVD_ERR_INVALID_ARG;
        }
    }

    // sizes of the schedule (Section 6.4.1) and of every carved buffer
    const int m_pad = (m + hz::ROWPAD - 1) / hz::ROWPAD * hz::ROWPAD;
    const int p_pad = (p + hz::ROWPAD - 1) / hz::ROWPAD * hz::ROWPAD;
    const int n_pad = (n + hz::ROWPAD - 1) / hz::ROWPAD * hz::ROWPAD;
    const long long Mt = (long long)m_pad + p_pad + n_pad;
    int nb = 2, wb = 1, wide = 1, kk = 2, npairs = 1, nsteps = 1;
    if (n >= 2) {
        const int w = o.block_width < n ? o.block_width : n;
        nb = (n + w - 1) / w;
        if (nb & 1) nb += 1;
        if (nb < 2) nb = 2;
        if (nb > n) nb = n & ~1;
        wb = (n + nb - 1) / nb;
        wide = n - nb * (wb - 1);
        kk = 2 * wb;
        npairs = nb / 2;
        nsteps = nb - 1;
    }
    // Gram row chunk: the same balance rule as ghsvd_solve
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GHSVD_ERR_CUDA;
    int kc = 512;
    if (o.gram_chunk > 0) {
        kc = (o.gram_chunk + hz::GRAM_KT - 1) / hz::GRAM_KT * hz::GRAM_KT;
    } else {
        kc = hz::gram_chunk_rows(m_pad, p_pad, npairs, sms);
    }
    const int chunks_h = (m_pad + kc - 1) / kc, chunks_s = (p_pad + kc - 1) / kc;
    const int cpp = chunks_h + chunks_s;
    long long off = 0;
    auto carve = [&](long long bytes) { long long at = off; off += align256(bytes); return at; };
    const long long oW = carve(16LL * Mt * n);
    const long long oPart = carve(16LL * npairs * cpp * hz::KKMAX * hz::KKMAX);
    const long long oZhat = carve(16LL * npairs * hz::KKMAX * hz::KKMAX);
    const long long oFlag = carve(4LL * npairs);
    const long long oSlot = carve(4LL * nsteps * npairs * kk);
    const long long oJrow = carve(m_pad);
    const long long oCnt = carve(16);
    const long long oErr = carve(8);
    const long long oLam = carve(8LL * n), oGsc = carve(8LL * n), oVn = carve(8LL * n);
    const long long oGc = carve(8LL * n), oKap = carve(8), oRank = carve(4LL * n);
    if (off > (long long)GHSVD_NOALLOC_SCRATCH_BYTES) return GHSVD_ERR_SCRATCH_TOO_SMALL;

    unsigned char *base = nullptr;
    ghsvd_status s = setup_device(dev, &base);
    if (s != GHSVD_OK) return s;
    double2 *W = (double2 *)(base + oW);
    void *partial = base + oPart;
    double2 *zhat = (double2 *)(base + oZhat);
    int *pair_flag = (int *)(base + oFlag);
    int *slotcol = (int *)(base + oSlot);
    int8_t *Jrow = (int8_t *)(base + oJrow);
    unsigned long long *counters = (unsigned long long *)(base + oCnt);
    int *err = (int *)(base + oErr);
    double *lam_tmp = (double *)(base + oLam), *gscale = (double *)(base + oGsc);
    double *vnorm2 = (double *)(base + oVn), *gcol2 = (double *)(base + oGc);
    double *kappa = (double *)(base + oKap);
    int *rank = (int *)(base + oRank);

#define NA_TRY(x)                                       \
    do {                                                \
        if ((x) != cudaSuccess) return GHSVD_ERR_CUDA;  \
    } while (0)

    // what must start at zero
    NA_TRY(cudaMemsetAsync(err, 0, 8, st));
    NA_TRY(cudaMemsetAsync(counters, 0, 16, st));
    NA_TRY(cudaMemsetAsync(pair_flag, 0, 4LL * npairs, st));
    if (n >= 2) {
        const int total = nsteps * npairs * kk;
        noalloc_slots_kernel<<<(total + 255) / 256, 256, 0, st>>>(slotcol, nb, wb, wide);
        NA_TRY(cudaGetLastError());
    }
    NA_TRY(hz::launch_signs(Jrow, J, m, m_pad, n_plus, err + 1, st));
    NA_TRY(hz::launch_copyin(W, false, Mt, m, p, n, m_pad, p_pad, n_pad, F, ldf, G, ldg, nullptr, 0,
                             err, st));
    NA_TRY(hz::launch_gnorm(W, Mt, m_pad, p_pad, n, gcol2, st));
    int herr[2] = {0, 0};
    NA_TRY(cudaMemcpyAsync(herr, err, 8, cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
    if (herr[1]) return GHSVD_ERR_INVALID_ARG;
    if (herr[0] & hz::DEVERR_NONFINITE) return GHSVD_ERR_NONFINITE;

    ghsvd_status status = GHSVD_ERR_NOT_CONVERGED;
    int sweeps = 0;
    if (n < 2) {
        status = GHSVD_OK;
    } else {
        hz::StepArgs sa{};
        sa.npairs = npairs; sa.kk = kk; sa.m_pad = m_pad; sa.p_pad = p_pad; sa.n_pad = n_pad;
        sa.ld = Mt; sa.kc = kc; sa.chunks_h = chunks_h; sa.chunks_s = chunks_s;
        hz::InnerArgs ia{};
        ia.npairs = npairs; ia.kk = kk; ia.cpp = cpp; ia.chunks_h = chunks_h;
        ia.inner_sweeps = o.inner_sweeps; ia.crit_mode = o.crit_mode;
        ia.tol = o.tol_scale * ldexp(1.0, -53) * sqrt((double)n);
        while (sweeps < o.max_sweeps) {
            // the wall-time limit, checked between sweeps as in ghsvd_solve
            if (o.timeout_ms > 0 && sweeps > 0 &&
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                        .count() >= (double)o.timeout_ms) {
                status = GHSVD_ERR_TIMEOUT;
                break;
            }
            NA_TRY(cudaMemsetAsync(counters, 0, 16, st));
            for (int r = 0; r < nsteps; ++r) {
                sa.slotcol = slotcol + (size_t)r * npairs * kk;
                NA_TRY(hz::launch_gram(W, false, Jrow, sa, partial, st));
                NA_TRY(hz::launch_inner(partial, false, sa.slotcol, ia, zhat, pair_flag, counters,
                                        err, st));
                NA_TRY(hz::launch_update(W, false, sa, zhat, pair_flag, st));
            }
            unsigned long long hc[2] = {0, 0};
            NA_TRY(cudaMemcpyAsync(hc, counters, 16, cudaMemcpyDeviceToHost, st));
            NA_TRY(cudaMemcpyAsync(herr, err, 8, cudaMemcpyDeviceToHost, st));
            NA_TRY(cudaStreamSynchronize(st));
            ++sweeps;
            if (sweeps_out) *sweeps_out = sweeps;
            if (herr[0] & hz::DEVERR_RANK) return GHSVD_ERR_RANK_DEFICIENT;
            if (herr[0] & hz::DEVERR_NONFINITE) return GHSVD_ERR_NONFINITE;
            if (hc[1] == 0) { status = GHSVD_OK; break; }
        }
    }
    NA_TRY(hz::launch_finalize(W, Mt, Jrow, m_pad, p_pad, n, o.sort_ascending, lam_tmp, gscale,
                               vnorm2, gcol2, kappa, rank, lambda, (double2 *)V, ldv, err, st));
    NA_TRY(cudaMemcpyAsync(herr, err, 8, cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
#undef NA_TRY
    if (herr[0] & hz::DEVERR_RANK) return GHSVD_ERR_RANK_DEFICIENT;
    if (herr[0] & hz::DEVERR_NONFINITE) return GHSVD_ERR_NONFINITE;
    if (sweeps_out) *sweeps_out = sweeps;
    return status;
}
