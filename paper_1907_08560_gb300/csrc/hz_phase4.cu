// hz_phase4.cu -- Phase 4 of arXiv 1907.08560 (Section 7): X = Z^{-1} by
// Gaussian elimination with complete pivoting (P Z Q = L U, the paper's
// ZGETC2 step) and a solve of Z X = I (its ZGESC2 step), plus the pieces of
// the full GHSVD (Section 6.1.7 outputs) and of the error measure eq. 7.1.
//
// Elimination: step k is one single-CTA kernel (reduce the partial maxima,
// exchange row and column, divide the pivot column) and one tiled kernel
// (the rank-1 update of the trailing matrix, which also forms the partial
// maxima of the next step).  The solve is one kernel with one CTA per column
// of X, each carrying its column through the permutations and both
// triangular solves in shared memory.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hz_launch.h"

namespace hz {
namespace {

constexpr int LT = 64;          // edge of an update tile
constexpr int NTU = 256;        // threads of an update CTA: 64 rows x 4 column groups
constexpr int NT1 = 1024;
constexpr int NTS = 256;        // threads of a solve CTA

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// a / b by Smith's algorithm (R. L. Smith, CACM 5(8), 1962)
__device__ __forceinline__ double2 cdiv(double2 a, double2 b)
{
    if (fabs(b.x) >= fabs(b.y)) {
        const double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    }
    const double r = b.x / b.y, d = b.x * r + b.y;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}

// larger value wins; equal values go to the smaller column-major index
__device__ __forceinline__ void better(double &v, long long &i, double v2, long long i2)
{
    if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

// The last stage runs in warp 0 and is broadcast through shared memory (a
// warp's FP64 instruction holds its sub-partition's FP64 pipe for 64 cycles,
// so every thread repeating it costs NT/32 times as much); better is a total
// order on the values that can win (NaN never does), so the tree picks what a
// scan in warp order would.
template <int NT>
__device__ void block_argmax(double &v, long long &i, double *shv, long long *shi)
{
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const long long i2 = __shfl_xor_sync(0xffffffffu, i, o);
        better(v, i, v2, i2);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) { shv[w] = v; shi[w] = i; }
    __syncthreads();
    if (w == 0) {
        v = l < NT / 32 ? shv[l] : shv[0];
        i = l < NT / 32 ? shi[l] : shi[0];
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const long long i2 = __shfl_xor_sync(0xffffffffu, i, o);
            better(v, i, v2, i2);
        }
        __syncwarp();
        if (l == 0) { shv[0] = v; shi[0] = i; }
    }
    __syncthreads();
    v = shv[0];
    i = shi[0];
    __syncthreads();
}

// Trailing update of step k (k = -1: none) over [k+1, n)^2 and the partial
// maxima of |a_ij| there; one 64 x 64 tile per CTA.
__global__ void __launch_bounds__(NTU)
lu_update(double2 *__restrict__ A, long long ld, int n, int k, double *__restrict__ pv,
          long long *__restrict__ pi)
{
    __shared__ double2 urow[LT];
    __shared__ double shv[NTU / 32];
    __shared__ long long shi[NTU / 32];
    const int r0 = k + 1;
    const int tiles_r = (n - r0 + LT - 1) / LT;
    const int tr = blockIdx.x % tiles_r, tc = blockIdx.x / tiles_r;
    const int row = r0 + tr * LT + (threadIdx.x % LT);
    const int cbase = r0 + tc * LT;
    if (k >= 0 && threadIdx.x < LT) {
        const int c = cbase + threadIdx.x;
        urow[threadIdx.x] = c < n ? A[k + ld * c] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    double v = -1.0;
    long long idx = (long long)n * n;
    if (row < n) {
        const double2 l = k >= 0 ? A[row + ld * k] : make_double2(0.0, 0.0);
        const int g = threadIdx.x / LT;
        for (int q = 0; q < LT / 4; ++q) {
            const int cl = g * (LT / 4) + q;
            const int c = cbase + cl;
            if (c >= n) break;
            double2 a = A[row + ld * c];
            if (k >= 0) {
                const double2 p = cmul(l, urow[cl]);
                a = make_double2(a.x - p.x, a.y - p.y);
                A[row + ld * c] = a;
            }
            better(v, idx, hypot(a.x, a.y), (long long)c * n + row);
        }
    }
    block_argmax<NTU>(v, idx, shv, shi);
    if (threadIdx.x == 0) {
        pv[blockIdx.x] = v;
        pi[blockIdx.x] = idx;
    }
}

// Step k: the pivot from the partial maxima, the exchanges, the multipliers.
__global__ void __launch_bounds__(NT1)
lu_pivot(double2 *__restrict__ A, long long ld, int n, int k, int nparts, const double *__restrict__ pv,
         const long long *__restrict__ pi, int *__restrict__ rowp, int *__restrict__ colp,
         int *__restrict__ flag)
{
    __shared__ double shv[NT1 / 32];
    __shared__ long long shi[NT1 / 32];
    if (*flag) return;
    double v = -1.0;
    long long idx = (long long)n * n;
    for (int t = threadIdx.x; t < nparts; t += NT1) better(v, idx, pv[t], pi[t]);
    block_argmax<NT1>(v, idx, shv, shi);
    if (idx >= (long long)n * n) {          // no comparable entry (NaN): stop
        if (threadIdx.x == 0) *flag = 1;
        return;
    }
    const int pr = (int)(idx % n), pc = (int)(idx / n);
    if (threadIdx.x == 0) {
        rowp[k] = pr;
        colp[k] = pc;
    }
    if (pr != k)
        for (int c = threadIdx.x; c < n; c += NT1) {
            const double2 t = A[k + ld * c];
            A[k + ld * c] = A[pr + ld * c];
            A[pr + ld * c] = t;
        }
    __syncthreads();
    if (pc != k)
        for (int r = threadIdx.x; r < n; r += NT1) {
            const double2 t = A[r + ld * k];
            A[r + ld * k] = A[r + ld * pc];
            A[r + ld * pc] = t;
        }
    __syncthreads();
    const double2 piv = A[k + ld * k];
    if (piv.x == 0.0 && piv.y == 0.0) {
        if (threadIdx.x == 0) *flag = 1;
        return;
    }
    for (int r = k + 1 + threadIdx.x; r < n; r += NT1) A[r + ld * k] = cdiv(A[r + ld * k], piv);
}

// X[:, c] = Q U^{-1} L^{-1} P e_c, one CTA per column, the column in shared memory.
__global__ void __launch_bounds__(NTS)
lu_solve(const double2 *__restrict__ LU, long long ld, int n, const int *__restrict__ rowp,
         const int *__restrict__ colp, const int *__restrict__ flag, double2 *__restrict__ X, long long ldx)
{
    extern __shared__ double2 x[];
    __shared__ int sfirst;
    if (*flag) return;                          // the elimination stopped: no valid permutation
    const int c = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += NTS) x[i] = make_double2(i == c ? 1.0 : 0.0, 0.0);
    __syncthreads();
    if (threadIdx.x == 0) {
        int pos = c;                              // where the 1 sits
        for (int k = 0; k < n; ++k) {
            const int r = rowp[k];
            const double2 t = x[k]; x[k] = x[r]; x[r] = t;
            if (pos == k) pos = r; else if (pos == r) pos = k;
        }
        sfirst = pos;
    }
    __syncthreads();
    for (int k = sfirst; k < n; ++k) {            // L y = P e_c (entries above the 1 stay zero)
        const double2 xk = x[k];
        const double2 *lk = LU + ld * k;
        for (int i = k + 1 + threadIdx.x; i < n; i += NTS) {
            const double2 p = cmul(lk[i], xk);
            x[i] = make_double2(x[i].x - p.x, x[i].y - p.y);
        }
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {            // U w = y
        const double2 *uk = LU + ld * k;
        const double2 xk = cdiv(x[k], uk[k]);
        __syncthreads();
        if (threadIdx.x == 0) x[k] = xk;
        for (int i = threadIdx.x; i < k; i += NTS) {
            const double2 p = cmul(uk[i], xk);
            x[i] = make_double2(x[i].x - p.x, x[i].y - p.y);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = n - 1; k >= 0; --k) {        // x = Q w
            const int r = colp[k];
            const double2 t = x[k]; x[k] = x[r]; x[r] = t;
        }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += NTS) X[i + ldx * c] = x[i];
}

__global__ void copy_square(const double2 *__restrict__ Z, long long ldz, int n, double2 *__restrict__ A,
                            long long lda)
{
    const int j = blockIdx.x;
    for (int r = threadIdx.x; r < n; r += blockDim.x) A[r + lda * j] = Z[r + ldz * j];
}

// Section 6.1.7: Sigma_F'_j, Sigma_G'_j of the converged columns of W and
// Sigma_j = (Sigma_F'^2 + Sigma_G'^2)^{1/2}; Z = Z' Sigma^{-1} into Zs;
// Sigma_F = Sigma_F' / Sigma, Sigma_G = Sigma_G' / Sigma.  One CTA per column.
__global__ void __launch_bounds__(256)
sigma_kernel(const double2 *__restrict__ W, long long ld, const int8_t *__restrict__ Jrow, int m_pad,
             int p_pad, int n, double *__restrict__ sig, double *__restrict__ sf, double *__restrict__ sg,
             double2 *__restrict__ Zs, long long ldz)
{
    __shared__ double rf[256], rg[256];
    const int j = blockIdx.x;
    const double2 *col = W + ld * j;
    double f = 0.0, g = 0.0;
    for (int r = threadIdx.x; r < m_pad; r += 256) {
        const double2 a = col[r];
        f += (double)Jrow[r] * (a.x * a.x + a.y * a.y);
    }
    for (int r = threadIdx.x; r < p_pad; r += 256) {
        const double2 a = col[m_pad + r];
        g += a.x * a.x + a.y * a.y;
    }
    rf[threadIdx.x] = f;
    rg[threadIdx.x] = g;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) { rf[threadIdx.x] += rf[threadIdx.x + s]; rg[threadIdx.x] += rg[threadIdx.x + s]; }
        __syncthreads();
    }
    const double sfp = sqrt(fabs(rf[0])), sgp = sqrt(rg[0]);
    const double s = sqrt(sfp * sfp + sgp * sgp);
    if (threadIdx.x == 0) {
        sig[j] = s;
        if (sf) sf[j] = sfp / s;
        if (sg) sg[j] = sgp / s;
    }
    if (!Zs) return;
    const double2 *z = col + m_pad + p_pad;
    for (int r = threadIdx.x; r < n; r += 256) Zs[r + ldz * j] = make_double2(z[r].x / s, z[r].y / s);
}

// B = Sigma^{-1} X (row scaling): with F' = F Z' this is Z'^{-1}, so that
// [F'; G'] B = U Sigma_F X and V Sigma_G X of eq. 7.1.
__global__ void rowscale(const double2 *__restrict__ X, long long ldx, int n, const double *__restrict__ sig,
                         double2 *__restrict__ B)
{
    const int j = blockIdx.x;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const double2 a = X[r + ldx * j];
        B[r + (long long)n * j] = make_double2(a.x / sig[r], a.y / sig[r]);
    }
}

// part[2 b] = sum |A - C|^2, part[2 b + 1] = sum |A|^2 over the columns of CTA b
__global__ void __launch_bounds__(256)
err_partial(const double2 *__restrict__ A, long long lda, const double2 *__restrict__ C, long long ldc,
            int rows, int n, double *__restrict__ part)
{
    __shared__ double rd[256], ra[256];
    double d = 0.0, a2 = 0.0;
    for (int j = blockIdx.x; j < n; j += gridDim.x)
        for (int r = threadIdx.x; r < rows; r += 256) {
            const double2 a = A[r + lda * j], c = C[r + ldc * j];
            const double ex = a.x - c.x, ey = a.y - c.y;
            d += ex * ex + ey * ey;
            a2 += a.x * a.x + a.y * a.y;
        }
    rd[threadIdx.x] = d;
    ra[threadIdx.x] = a2;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) { rd[threadIdx.x] += rd[threadIdx.x + s]; ra[threadIdx.x] += ra[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = rd[0]; part[2 * blockIdx.x + 1] = ra[0]; }
}

__global__ void err_final(const double *__restrict__ part, int nparts, double *__restrict__ out)
{
    if (threadIdx.x != 0) return;
    double d = 0.0, a = 0.0;
    for (int b = 0; b < nparts; ++b) { d += part[2 * b]; a += part[2 * b + 1]; }
    out[0] = a > 0.0 ? sqrt(d / a) : 0.0;
}

// dst[perm[i], j] = src[i, j]: eigenvectors of (F~ P2, G~ P2) back to the
// column order of (F~, G~) (Z~ = P2 Z, Section 5)
__global__ void permute_rows(const double2 *__restrict__ src, long long lds, int n, const int *__restrict__ perm,
                             double2 *__restrict__ dst, long long ldd)
{
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[perm[i] + ldd * j] = src[i + lds * j];
}

}  // namespace

cudaError_t launch_permute_rows(const double2 *src, long long lds, int n, const int *perm, double2 *dst,
                                long long ldd, cudaStream_t s)
{
    permute_rows<<<n, 256, 0, s>>>(src, lds, n, perm, dst, ldd);
    return cudaGetLastError();
}

static int lu_tiles(int n, int k)
{
    const int t = (n - (k + 1) + LT - 1) / LT;
    return t * t;
}

size_t inverse_workspace_bytes(int n)
{
    auto a = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t tiles = (size_t)lu_tiles(n, -1);
    return a(16ull * n * n) + a(8 * tiles) + a(8 * tiles) + 2 * a(4ull * n) + a(4);
}

int inverse_max_n() { return 12288; }

// X = Z^{-1}; d_flag (device int) = 1 if a pivot is exactly zero.
cudaError_t launch_inverse(int n, const double2 *Z, long long ldz, double2 *X, long long ldx, void *ws,
                           int *d_flag, cudaStream_t s)
{
    auto a = [](size_t b) { return (b + 255) / 256 * 256; };
    char *base = (char *)ws;
    const size_t tiles = (size_t)lu_tiles(n, -1);
    double2 *A = (double2 *)base; base += a(16ull * n * n);
    double *pv = (double *)base; base += a(8 * tiles);
    long long *pi = (long long *)base; base += a(8 * tiles);
    int *rowp = (int *)base; base += a(4ull * n);
    int *colp = (int *)base; base += a(4ull * n);
    int *flag = (int *)base;
    cudaError_t e;
    if ((e = cudaMemsetAsync(flag, 0, 4, s)) != cudaSuccess) return e;
    copy_square<<<n, 256, 0, s>>>(Z, ldz, n, A, n);
    lu_update<<<lu_tiles(n, -1), NTU, 0, s>>>(A, n, n, -1, pv, pi);
    for (int k = 0; k < n; ++k) {
        lu_pivot<<<1, NT1, 0, s>>>(A, n, n, k, lu_tiles(n, k - 1), pv, pi, rowp, colp, flag);
        if (k + 1 < n) lu_update<<<lu_tiles(n, k), NTU, 0, s>>>(A, n, n, k, pv, pi);
    }
    const size_t smem = 16ull * n;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(lu_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    lu_solve<<<n, NTS, smem, s>>>(A, n, n, rowp, colp, flag, X, ldx);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaMemcpyAsync(d_flag, flag, 4, cudaMemcpyDeviceToDevice, s);
}

int inverse_launches(int n) { return 2 + 2 * n - 1 + 1; }

cudaError_t launch_sigma(const double2 *W, long long ld, const int8_t *Jrow, int m_pad, int p_pad, int n,
                         double *sig, double *sf, double *sg, double2 *Zs, long long ldz, cudaStream_t s)
{
    sigma_kernel<<<n, 256, 0, s>>>(W, ld, Jrow, m_pad, p_pad, n, sig, sf, sg, Zs, ldz);
    return cudaGetLastError();
}

cudaError_t launch_rowscale(const double2 *X, long long ldx, int n, const double *sig, double2 *B,
                            cudaStream_t s)
{
    rowscale<<<n, 256, 0, s>>>(X, ldx, n, sig, B);
    return cudaGetLastError();
}

// out[0] = ||A - C||_F / ||A||_F over rows x n; part: 2 * 304 doubles
cudaError_t launch_rel_err(const double2 *A, long long lda, const double2 *C, long long ldc, int rows, int n,
                           double *part, double *out, cudaStream_t s)
{
    const int nb = n < 304 ? n : 304;
    err_partial<<<nb, 256, 0, s>>>(A, lda, C, ldc, rows, n, part);
    err_final<<<1, 32, 0, s>>>(part, nb, out);
    return cudaGetLastError();
}

}  // namespace hz
