// hz_step.cu -- instantiation and launch of the step kernels, plus the
// set-up (copy-in), finalization (Section 6.1.7 outputs) and ordering
// kernels.  Host code calls only the launch_* functions of hz_launch.h.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include "hz_gemm.cuh"
#include "hz_gram.cuh"
#include "hz_inner.cuh"
#include "hz_update.cuh"
#include "hz_launch.h"

namespace hz {

// ----------------------------------------------------------------------------
// Copy-in: W <- [F; G; Z0] with zero padding rows, J -> padded sign rows.
// One CTA row-block per column; flags non-finite input entries.
// ----------------------------------------------------------------------------
template <typename T2out>
__global__ void copyin_kernel(T2out *__restrict__ W, long long ld, int m, int p, int n,
                              int m_pad, int p_pad, int n_pad,
                              const double2 *__restrict__ F, long long ldf,
                              const double2 *__restrict__ G, long long ldg,
                              const double2 *__restrict__ V0, long long ldv0, int *err)
{
    const int j = blockIdx.y;
    const long long Mt = (long long)m_pad + p_pad + n_pad;
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Mt;
         i += (long long)gridDim.x * blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        if (i < m_pad) {
            if (i < m) v = F[i + ldf * j];
        } else if (i < m_pad + p_pad) {
            const long long r = i - m_pad;
            if (r < p) v = G[r + ldg * j];
        } else {
            const long long r = i - m_pad - p_pad;
            if (r < n) {
                if (V0) v = V0[r + ldv0 * j];
                else v = make_double2(r == j ? 1.0 : 0.0, 0.0);
            }
        }
        if (!isfinite(v.x) || !isfinite(v.y)) bad = true;
        T2out o;
        o.x = v.x;
        o.y = v.y;
        W[i + ld * j] = o;
    }
    if (bad) atomicOr(err, DEVERR_NONFINITE);
}

// Jrow[i] = J[i] (validated +-1) for i < m, +1 on padding rows; or positives
// first: +1 for i < n_plus.
__global__ void signs_kernel(int8_t *__restrict__ Jrow, const int8_t *__restrict__ J, int m,
                             int m_pad, long long n_plus, int *bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m_pad; i += gridDim.x * blockDim.x) {
        int8_t s = 1;
        if (i < m) {
            if (J) {
                s = J[i];
                if (s != 1 && s != -1) { atomicOr(bad, 1); s = 1; }
            } else {
                s = i < n_plus ? 1 : -1;
            }
        }
        Jrow[i] = s;
    }
}

// Copy W (either precision) into the other precision, rows [0, Mt) of n columns.
template <typename A, typename B>
__global__ void convert_kernel(B *__restrict__ dst, const A *__restrict__ src, long long count)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        B o;
        o.x = src[i].x;
        o.y = src[i].y;
        dst[i] = o;
    }
}

// ----------------------------------------------------------------------------
// Outputs (Section 6.1.7, eq. 3.2): per column j,
//   hf_j = f_j^* J f_j,  gg_j = g_j^* g_j,  lambda_j = hf_j / gg_j,
//   V[:, j] = Z'[:, j] / sqrt(gg_j).
// One CTA per column; fixed-order block reduction (deterministic).
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
colnorm_kernel(const double2 *__restrict__ W, long long ld, const int8_t *__restrict__ Jrow,
               int m_pad, int p_pad, int n, double *__restrict__ lam, double *__restrict__ gscale,
               double *__restrict__ vnorm2, int *err)
{
    __shared__ double red[3][256];
    const int j = blockIdx.x, tid = threadIdx.x;
    const double2 *col = W + ld * j;
    double hf = 0.0, gg = 0.0;
    for (int i = tid; i < m_pad; i += 256) {
        const double2 v = col[i];
        const double a = fma(v.x, v.x, v.y * v.y);
        hf += Jrow[i] < 0 ? -a : a;
    }
    for (int i = tid; i < p_pad; i += 256) {
        const double2 v = col[m_pad + i];
        gg = fma(v.x, v.x, fma(v.y, v.y, gg));
    }
    double zz = 0.0;
    for (int i = tid; i < n; i += 256) {
        const double2 v = col[m_pad + p_pad + i];
        zz = fma(v.x, v.x, fma(v.y, v.y, zz));
    }
    red[0][tid] = hf;
    red[1][tid] = gg;
    red[2][tid] = zz;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (tid < s) {
            red[0][tid] += red[0][tid + s];
            red[1][tid] += red[1][tid + s];
            red[2][tid] += red[2][tid + s];
        }
        __syncthreads();
    }
    if (tid == 0) {
        const double h = red[0][0], g = red[1][0];
        if (!(g > 0.0)) atomicOr(err, DEVERR_RANK);
        if (!isfinite(h) || !isfinite(g)) atomicOr(err, DEVERR_NONFINITE);
        lam[j] = h / g;
        gscale[j] = 1.0 / sqrt(g);
        vnorm2[j] = red[2][0] / g;
    }
}

// gcol2[j] = ||g_j||^2 of the G rows of W (called on the input G).
__global__ void __launch_bounds__(256)
gnorm_kernel(const double2 *__restrict__ W, long long ld, int g0, int p_pad, double *__restrict__ gcol2)
{
    __shared__ double red[256];
    const int j = blockIdx.x, tid = threadIdx.x;
    const double2 *col = W + ld * j + g0;
    double s = 0.0;
    for (int i = tid; i < p_pad; i += 256) s = fma(col[i].x, col[i].x, fma(col[i].y, col[i].y, s));
    red[tid] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (tid < k) red[tid] += red[tid + k];
        __syncthreads();
    }
    if (tid == 0) gcol2[j] = red[0];
}

// Numerical rank of G (the end-of-iteration form of the rank-deficiency
// stop of Section 6.4.2): G V has orthonormal columns, so
// kappa_est = ||G||_F max_j ||v_j|| estimates cond(G) within sqrt(n);
// kappa_est > 1 / (8 eps sqrt(n)), eps = 2^-53, is a rank-deficient G.
// vnorm2[j] = ||v_j||^2.  One CTA; fixed-order sums.
__global__ void __launch_bounds__(256)
rankcheck_kernel(const double *__restrict__ gcol2, const double *__restrict__ vnorm2, int n,
                 double *__restrict__ kappa, int *err)
{
    __shared__ double rs[256], rm[256];
    const int tid = threadIdx.x;
    double s = 0.0, mx = 0.0;
    for (int j = tid; j < n; j += 256) { s += gcol2[j]; mx = fmax(mx, vnorm2[j]); }
    rs[tid] = s;
    rm[tid] = mx;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (tid < k) { rs[tid] += rs[tid + k]; rm[tid] = fmax(rm[tid], rm[tid + k]); }
        __syncthreads();
    }
    if (tid == 0) {
        const double k = sqrt(rs[0]) * sqrt(rm[0]);
        *kappa = k;
        if (!(k <= 0.125 / (ldexp(1.0, -53) * sqrt((double)n)))) atomicOr(err, DEVERR_RANK);
    }
}

// rank[j] = position of lambda_j in ascending order (ties by index), or j.
__global__ void rank_kernel(const double *__restrict__ lam, int n, int sort, int *__restrict__ rank)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (!sort) { rank[j] = j; return; }
    const double x = lam[j];
    int r = 0;
    for (int k = 0; k < n; ++k) {
        const double y = lam[k];
        r += (y < x) || (y == x && k < j);
    }
    rank[j] = r;
}

// lambda_out[rank_j] = lambda_j; V[:, rank_j] = Z'[:, j] * gscale_j.
__global__ void emit_kernel(const double2 *__restrict__ W, long long ld, int zrow0, int n,
                            const double *__restrict__ lam, const double *__restrict__ gscale,
                            const int *__restrict__ rank, double *__restrict__ lam_out,
                            double2 *__restrict__ V, long long ldv)
{
    const int j = blockIdx.y;
    const int rj = rank[j];
    if (blockIdx.x == 0 && threadIdx.x == 0) lam_out[rj] = lam[j];
    if (!V) return;
    const double sc = gscale[j];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double2 z = W[zrow0 + i + ld * j];
        V[i + ldv * rj] = make_double2(z.x * sc, z.y * sc);
    }
}

// Copy rows [r0, r0 + rows) of W's n columns into a column-major buffer.
__global__ void extract_kernel(const double2 *__restrict__ W, long long ld, int r0, int rows, int n,
                               double2 *__restrict__ out, long long ldo)
{
    const int j = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x)
        out[i + ldo * j] = W[r0 + i + ld * j];
}

// C = A B for a column-major A (rows x n, rows a multiple of 64) and a square
// B (n x n, complex128 or complex64 promoted to FP64): one 64 x 64 tile per
// CTA (gemm_tile_3m, hz_gemm.cuh).  Used once per solve to apply a starting
// transformation (warm start) or the transformation accumulated by the
// complex64 sweeps to the FP64 factors.
template <typename TB>
__global__ void __launch_bounds__(256)
gemm_kernel(const double2 *__restrict__ A, long long lda, const TB *__restrict__ B, long long ldb,
            double2 *__restrict__ C, long long ldc, int n)
{
    gemm_tile_3m<TB>(A, lda, B, ldb, C, ldc, n, (long long)blockIdx.x * 64, blockIdx.y * 64);
}

// s + c += x * y without losing the rounding errors of the product and of
// the sum: the product by fma (TwoProduct) and the sum by Knuth's TwoSum, the
// errors accumulated in c (the compensated dot product of Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005).
__device__ __forceinline__ void acc2(double &s, double &c, double x, double y)
{
    const double h = x * y;
    const double l = fma(x, y, -h);
    const double t = s + h;
    const double z = t - s;
    const double e = (s - (t - z)) + (h - z);
    s = t;
    c += e + l;
}

// Batched form of the same product over independent items (one per pencil),
// with row and column bounds (any row count): C_i = A_i B_i.  Items marked
// accurate accumulate with compensated sums, so that the computed product is
// close to the correctly rounded one even when B_i is ill-conditioned (used
// to apply a warm-start basis: a plain product would put a backward error of
// the order of cond(B_i) eps into the factors).
__global__ void __launch_bounds__(256)
gemm_batched_kernel(const GemmItem *__restrict__ items)
{
    const GemmItem it = items[blockIdx.z];
    const long long row0 = (long long)blockIdx.x * 64;
    const int col0 = blockIdx.y * 64;
    if (row0 >= it.rows || col0 >= it.n) return;
    __shared__ double2 as[64][17];
    __shared__ double2 bs[16][64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int n = it.n;
    double accr[4][4], acci[4][4], corr[4][4], cori[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { accr[i][j] = 0; acci[i][j] = 0; corr[i][j] = 0; cori[i][j] = 0; }
    for (int k0 = 0; k0 < n; k0 += 16) {
        __syncthreads();
        for (int e = tid; e < 64 * 16; e += 256) {
            const int r = e % 64, k = e / 64;
            as[r][k] = (k0 + k < n && row0 + r < it.rows) ? it.A[row0 + r + it.lda * (k0 + k)]
                                                          : make_double2(0.0, 0.0);
        }
        for (int e = tid; e < 16 * 64; e += 256) {
            const int k = e % 16, c = e / 16;
            bs[k][c] = (k0 + k < n && col0 + c < n) ? it.B[(k0 + k) + it.ldb * (col0 + c)]
                                                   : make_double2(0.0, 0.0);
        }
        __syncthreads();
        if (it.accurate) {
            for (int k = 0; k < 16; ++k) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const double2 x = as[ty + 16 * i][k];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const double2 z = bs[k][tx + 16 * j];
                        acc2(accr[i][j], corr[i][j], x.x, z.x);
                        acc2(accr[i][j], corr[i][j], -x.y, z.y);
                        acc2(acci[i][j], cori[i][j], x.x, z.y);
                        acc2(acci[i][j], cori[i][j], x.y, z.x);
                    }
                }
            }
        } else {
#pragma unroll 4
            for (int k = 0; k < 16; ++k) {
                double2 x[4], z[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) x[i] = as[ty + 16 * i][k];
#pragma unroll
                for (int j = 0; j < 4; ++j) z[j] = bs[k][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        accr[i][j] = fma(x[i].x, z[j].x, accr[i][j]);
                        accr[i][j] = fma(-x[i].y, z[j].y, accr[i][j]);
                        acci[i][j] = fma(x[i].x, z[j].y, acci[i][j]);
                        acci[i][j] = fma(x[i].y, z[j].x, acci[i][j]);
                    }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long r = row0 + ty + 16 * i;
            const int c = col0 + tx + 16 * j;
            if (r < it.rows && c < n)
                it.C[r + it.ldc * c] = make_double2(accr[i][j] + corr[i][j], acci[i][j] + cori[i][j]);
        }
}

// kappa[i] = ||G_i||_F max_j ||(V0_i)_j||, an estimate of the condition of a
// warm-start basis relative to G_i (item fields: A = V0_i, lda, n; B holds the
// squared column norms of G_i as doubles).  One CTA per item.
__global__ void __launch_bounds__(256)
v0_kappa_kernel(const GemmItem *__restrict__ items, double *__restrict__ kappa)
{
    __shared__ double rg[8], rv[8];
    const GemmItem it = items[blockIdx.x];
    const double *gcol2 = (const double *)it.B;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double g = 0.0, vmax = 0.0;
    for (int j = warp; j < it.n; j += 8) {          // one warp per column, lanes over rows
        double v = 0.0;
        for (int i = lane; i < it.n; i += 32) {
            const double2 a = it.A[i + it.lda * j];
            v = fma(a.x, a.x, fma(a.y, a.y, v));
        }
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        vmax = fmax(vmax, v);
        if (lane == 0) g += gcol2[j];
    }
    if (lane == 0) { rg[warp] = g; rv[warp] = vmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double gs = 0.0, vm = 0.0;
        for (int k = 0; k < 8; ++k) { gs += rg[k]; vm = fmax(vm, rv[k]); }
        kappa[blockIdx.x] = sqrt(gs) * sqrt(vm);
    }
}

// Batched copy of column-major blocks: dst_i (rows x n, ldd) <- src_i (lds).
__global__ void copy_batched_kernel(const GemmItem *__restrict__ items)
{
    // item fields reused: A = source (lda), C = destination (ldc), rows, n
    const GemmItem it = items[blockIdx.y];
    const long long total = (long long)it.rows * it.n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e % it.rows, c = e / it.rows;
        it.C[r + it.ldc * c] = it.A[r + it.lda * c];
    }
}

// Identity into rows [r0, r0 + n_pad) of an n-column complex64 buffer.
__global__ void eye32_kernel(float2 *__restrict__ W, long long ld, int r0, int n, int n_pad)
{
    const int j = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x)
        W[r0 + i + ld * j] = make_float2(i == j ? 1.0f : 0.0f, 0.0f);
}

// ----------------------------------------------------------------------------
// Launchers
// ----------------------------------------------------------------------------
static unsigned grid1d(long long work, int threads, int cap = 4096)
{
    long long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

cudaError_t launch_copyin(void *W, bool single, long long ld, int m, int p, int n, int m_pad,
                          int p_pad, int n_pad, const void *F, long long ldf, const void *G,
                          long long ldg, const void *V0, long long ldv0, int *err, cudaStream_t s)
{
    const long long Mt = (long long)m_pad + p_pad + n_pad;
    dim3 grid(grid1d(Mt, 256, 64), n);
    if (single)
        copyin_kernel<float2><<<grid, 256, 0, s>>>((float2 *)W, ld, m, p, n, m_pad, p_pad, n_pad,
                                                   (const double2 *)F, ldf, (const double2 *)G, ldg,
                                                   (const double2 *)V0, ldv0, err);
    else
        copyin_kernel<double2><<<grid, 256, 0, s>>>((double2 *)W, ld, m, p, n, m_pad, p_pad, n_pad,
                                                    (const double2 *)F, ldf, (const double2 *)G, ldg,
                                                    (const double2 *)V0, ldv0, err);
    return cudaGetLastError();
}

cudaError_t launch_signs(int8_t *Jrow, const int8_t *J, int m, int m_pad, long long n_plus, int *bad,
                         cudaStream_t s)
{
    signs_kernel<<<grid1d(m_pad, 256, 256), 256, 0, s>>>(Jrow, J, m, m_pad, n_plus, bad);
    return cudaGetLastError();
}

cudaError_t launch_convert(void *dst, bool dst_single, const void *src, long long count, cudaStream_t s)
{
    if (dst_single)
        convert_kernel<double2, float2><<<grid1d(count, 256, 8192), 256, 0, s>>>(
            (float2 *)dst, (const double2 *)src, count);
    else
        convert_kernel<float2, double2><<<grid1d(count, 256, 8192), 256, 0, s>>>(
            (double2 *)dst, (const float2 *)src, count);
    return cudaGetLastError();
}

cudaError_t launch_gram(const void *W, bool single, const int8_t *Jrow, const StepArgs &a,
                        void *partial, cudaStream_t s)
{
    const int grid = a.npairs * (a.chunks_h + a.chunks_s);
    const int threads = single ? gram_threads(a.kk) : gram_threads_c128(a.kk);
    if (single)
        gram_kernel<float><<<grid, threads, 0, s>>>((const float2 *)W, Jrow, a, (float2 *)partial);
    else
        gram_kernel<double><<<grid, threads, 0, s>>>((const double2 *)W, Jrow, a, (double2 *)partial);
    return cudaGetLastError();
}

static size_t inner_smem(bool single)
{
    return inner_smem_bytes(single ? sizeof(float2) : sizeof(double2));
}

// Cluster widths of the inner level usable on this device (bit CL set: a
// cluster of CL CTAs with the inner kernel's shared memory can be resident).
static int g_cluster_mask = -1;

template <typename TP, typename TU, int CL>
static cudaError_t setup_cluster(bool single, int *mask)
{
    auto k = inner_cluster_kernel<TP, TU, CL>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)inner_smem(single));
    if (e != cudaSuccess) { cudaGetLastError(); return cudaSuccess; }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = inner_smem(single);
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = CL;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg);
    if (e != cudaSuccess) { cudaGetLastError(); return cudaSuccess; }
    if (nclusters > 0) *mask |= CL;
    return cudaSuccess;
}

cudaError_t setup_kernels()
{
    cudaError_t e;
    e = cudaFuncSetAttribute(inner_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)inner_smem(false));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(inner_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)inner_smem(true));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(update_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)update_smem(sizeof(double2)));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(update_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)update_smem(sizeof(float2)));
    if (e != cudaSuccess) return e;
    e = tc_setup();
    if (e != cudaSuccess) return e;
    e = delta64_setup();
    if (e != cudaSuccess) return e;
    if (g_cluster_mask < 0) {
        int m64 = 0, m32 = 0;
        const char *env = getenv("GHSVD_INNER_CLUSTER");
        if (!(env && env[0] == '0')) {
            setup_cluster<double, double, 2>(false, &m64);
            setup_cluster<double, double, 4>(false, &m64);
            setup_cluster<float, float, 2>(true, &m32);
            setup_cluster<float, float, 4>(true, &m32);
        }
        g_cluster_mask = m64 & m32;
    }
    return cudaSuccess;
}

template <typename TP, typename TU, int CL>
static cudaError_t launch_inner_cluster(const void *partial, const int *slotcol, const InnerArgs &a,
                                        double2 *zhat, int *pair_flag, unsigned long long *counters,
                                        int *err, cudaStream_t s, bool single)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.npairs * CL);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = inner_smem(single);
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = CL;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, inner_cluster_kernel<TP, TU, CL>,
                              (const typename cplx<TP>::t *)partial, slotcol, a,
                              (typename cplx<TU>::t *)zhat, pair_flag, counters, err);
}

cudaError_t launch_inner(const void *partial, bool single, const int *slotcol, const InnerArgs &a,
                         double2 *zhat, int *pair_flag, unsigned long long *counters, int *err,
                         cudaStream_t s)
{
    // FP64 sweeps: spread each block pivot over a cluster of 4 (or 2) SMs
    // when the step's pairs leave SMs idle (for the complex64 sweeps the
    // cluster's barriers and remote stores cost more than they save: 0.69
    // against 0.50 ms per step at n = 2048)
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int mask = (g_cluster_mask < 0 || single) ? 0 : g_cluster_mask;
    if ((mask & 4) && a.npairs * 4 <= sms) {
        return single ? launch_inner_cluster<float, float, 4>(partial, slotcol, a, zhat, pair_flag,
                                                              counters, err, s, true)
                      : launch_inner_cluster<double, double, 4>(partial, slotcol, a, zhat, pair_flag,
                                                                counters, err, s, false);
    }
    if ((mask & 2) && a.npairs * 2 <= sms) {
        return single ? launch_inner_cluster<float, float, 2>(partial, slotcol, a, zhat, pair_flag,
                                                              counters, err, s, true)
                      : launch_inner_cluster<double, double, 2>(partial, slotcol, a, zhat, pair_flag,
                                                                counters, err, s, false);
    }
    if (single)
        inner_kernel<float, float><<<a.npairs, 1024, inner_smem(true), s>>>(
            (const float2 *)partial, slotcol, a, (float2 *)zhat, pair_flag, counters, err);
    else
        inner_kernel<double, double><<<a.npairs, 1024, inner_smem(false), s>>>(
            (const double2 *)partial, slotcol, a, zhat, pair_flag, counters, err);
    return cudaGetLastError();
}

cudaError_t launch_update(void *W, bool single, const StepArgs &a, const double2 *zhat,
                          const int *pair_flag, cudaStream_t s)
{
    const long long Mt = (long long)a.m_pad + a.p_pad + a.n_pad;
    dim3 grid((unsigned)(Mt / UPD_R), a.npairs);
    if (single)     // complex64 sweeps: Z^ is complex64 (the inner level's own precision)
        update_kernel<float, float><<<grid, 256, update_smem(sizeof(float2)), s>>>(
            (float2 *)W, a, (const float2 *)zhat, pair_flag);
    else
        update_kernel<double, double><<<grid, 256, update_smem(sizeof(double2)), s>>>(
            (double2 *)W, a, zhat, pair_flag);
    return cudaGetLastError();
}

cudaError_t launch_gnorm(const double2 *W, long long ld, int g0, int p_pad, int n, double *gcol2,
                         cudaStream_t s)
{
    gnorm_kernel<<<n, 256, 0, s>>>(W, ld, g0, p_pad, gcol2);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double2 *W, long long ld, const int8_t *Jrow, int m_pad, int p_pad,
                            int n, int sort, double *lam_tmp, double *gscale, double *vnorm2,
                            const double *gcol2, double *kappa, int *rank, double *lam_out,
                            double2 *V, long long ldv, int *err, cudaStream_t s)
{
    colnorm_kernel<<<n, 256, 0, s>>>(W, ld, Jrow, m_pad, p_pad, n, lam_tmp, gscale, vnorm2, err);
    rankcheck_kernel<<<1, 256, 0, s>>>(gcol2, vnorm2, n, kappa, err);
    rank_kernel<<<(n + 255) / 256, 256, 0, s>>>(lam_tmp, n, sort, rank);
    dim3 grid(grid1d(n, 256, 64), n);
    emit_kernel<<<grid, 256, 0, s>>>(W, ld, m_pad + p_pad, n, lam_tmp, gscale, rank, lam_out, V, ldv);
    return cudaGetLastError();
}

cudaError_t launch_gemm(const double2 *A, long long lda, int rows, const void *B, bool b_single,
                        long long ldb, double2 *C, long long ldc, int n, cudaStream_t s)
{
    dim3 grid((unsigned)(rows / 64), (unsigned)((n + 63) / 64));
    if (b_single)
        gemm_kernel<float2><<<grid, 256, 0, s>>>(A, lda, (const float2 *)B, ldb, C, ldc, n);
    else
        gemm_kernel<double2><<<grid, 256, 0, s>>>(A, lda, (const double2 *)B, ldb, C, ldc, n);
    return cudaGetLastError();
}

cudaError_t launch_gemm_batched(const GemmItem *items, int count, long long max_rows, int max_n,
                                cudaStream_t s)
{
    dim3 grid((unsigned)((max_rows + 63) / 64), (unsigned)((max_n + 63) / 64), (unsigned)count);
    gemm_batched_kernel<<<grid, 256, 0, s>>>(items);
    return cudaGetLastError();
}

cudaError_t launch_v0_kappa(const GemmItem *items, int count, double *kappa, cudaStream_t s)
{
    v0_kappa_kernel<<<count, 256, 0, s>>>(items, kappa);
    return cudaGetLastError();
}

cudaError_t launch_copy_batched(const GemmItem *items, int count, cudaStream_t s)
{
    dim3 grid(256, (unsigned)count);
    copy_batched_kernel<<<grid, 256, 0, s>>>(items);
    return cudaGetLastError();
}

cudaError_t launch_eye32(void *W, long long ld, int r0, int n, int n_pad, cudaStream_t s)
{
    dim3 grid(grid1d(n_pad, 256, 64), n);
    eye32_kernel<<<grid, 256, 0, s>>>((float2 *)W, ld, r0, n, n_pad);
    return cudaGetLastError();
}

cudaError_t launch_extract(const double2 *W, long long ld, int r0, int rows, int n, double2 *out,
                           long long ldo, cudaStream_t s)
{
    dim3 grid(grid1d(rows, 256, 64), n);
    extract_kernel<<<grid, 256, 0, s>>>(W, ld, r0, rows, n, out, ldo);
    return cudaGetLastError();
}

}  // namespace hz
