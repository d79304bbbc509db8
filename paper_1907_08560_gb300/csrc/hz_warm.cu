// hz_warm.cu -- learned warm start for families of pencils: a small MLP
// t -> V0(t) trained on the solver's own eigenvectors, the S-inner-product
// re-orthonormalization of a starting V0, and the column phase alignment
// used to make eigenvector targets comparable across pencils.
//
// The paper has no learned component; its Algorithm 1 admits any starting
// Z' (e.g. the prescaling D).  Here the starting Z' = V0 is predicted, and
// the HZ sweeps then run to the paper's stopping rule (Section 6.1.7).
//
// MLP: x (n_in) -> tanh(W1 x + b1) (n_h) -> tanh(W2 . + b2) (n_h) -> W3 . + b3
// (n_out), FP32, row-major activations (one sample per row), parameters in
// one flat vector [W1 (n_h x n_in), b1, W2 (n_h x n_h), b2, W3 (n_out x n_h),
// b3], loss = mean squared error over samples and outputs, Adam.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/ghsvd.h"
#include "hz_launch.h"

namespace {

// ---------------------------------------------------------------------------
// FP32 GEMM: C (M x N, row-major, ldc) = op(A) op(B) [+ C]; op(A) is M x K
// (A stored K x M when ta), op(B) is K x N (B stored N x K when tb).  64 x 64
// tiles, 16-deep K slabs in shared memory, 4 x 4 outputs per thread.  With
// splits > 1 every split of K writes its partial to part[split][M x N] and
// reduce_splits sums them in split order (deterministic).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
sgemm_kernel(int M, int N, int K, const float *__restrict__ A, int lda, int ta,
             const float *__restrict__ B, int ldb, int tb, float *__restrict__ C, int ldc,
             int accumulate, int kchunk, float *__restrict__ part)
{
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int k_begin = blockIdx.z * kchunk, k_end = min(K, k_begin + kchunk);
    float acc[4][4] = {};
    for (int k0 = k_begin; k0 < k_end; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            const int kk = e / 64, mm = e % 64;
            const int k = k0 + kk, mi = m0 + mm;
            float a = 0.f;
            if (k < k_end && mi < M) a = ta ? A[(long long)k * lda + mi] : A[(long long)mi * lda + k];
            As[kk][mm] = a;
            const int nj = n0 + mm;
            float b = 0.f;
            if (k < k_end && nj < N) b = tb ? B[(long long)nj * ldb + k] : B[(long long)k * ldb + nj];
            Bs[kk][mm] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int mi = m0 + ty + 16 * i, nj = n0 + tx + 16 * j;
            if (mi < M && nj < N) {
                if (part) part[(long long)blockIdx.z * M * N + (long long)mi * N + nj] = acc[i][j];
                else C[(long long)mi * ldc + nj] = accumulate ? C[(long long)mi * ldc + nj] + acc[i][j] : acc[i][j];
            }
        }
}

__global__ void reduce_splits(int M, int N, int splits, const float *__restrict__ part,
                              float *__restrict__ C, int ldc, int accumulate)
{
    const long long total = (long long)M * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[(long long)z * total + e];
        const long long mi = e / N, nj = e % N;
        C[mi * ldc + nj] = accumulate ? C[mi * ldc + nj] + s : s;
    }
}

// y = tanh(y + b) (act) or y + b, per row of a B x n matrix.
__global__ void bias_act(float *__restrict__ Y, const float *__restrict__ b, int B, int n, int act)
{
    const long long total = (long long)B * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const float v = Y[e] + b[e % n];
        Y[e] = act ? tanhf(v) : v;
    }
}

// dZ = dA * (1 - A^2) (tanh derivative).
__global__ void tanh_back(float *__restrict__ dA, const float *__restrict__ A, long long total)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        dA[e] *= 1.f - A[e] * A[e];
}

// db[j] = sum over rows of dZ[:, j] (fixed row order).
__global__ void colsum(const float *__restrict__ dZ, int B, int n, float *__restrict__ db)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float s = 0.f;
    for (int r = 0; r < B; ++r) s += dZ[(long long)r * n + j];
    db[j] = s;
}

// dY = 2 (Y - T) / (B n); per-block partial sums of (Y - T)^2 into lpart.
__global__ void mse_grad(const float *__restrict__ Y, const float *__restrict__ T, long long total,
                         float scale, float *__restrict__ dY, double *__restrict__ lpart)
{
    __shared__ double red[256];
    double s = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const float d = Y[e] - T[e];
        if (dY) dY[e] = 2.f * d * scale;
        s += (double)d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
}

__global__ void adam_step(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                          float *__restrict__ v, long long n, float lr, float b1, float b2,
                          float c1, float c2, float eps)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// splitmix64 -> uniform (-a, a): parameter initialization from a seed.
__global__ void init_uniform(float *__restrict__ p, long long n, unsigned long long seed, float a)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        const float u = (float)((z >> 40) * (1.0 / 16777216.0));   // [0, 1)
        p[i] = (2.f * u - 1.f) * a;
    }
}

unsigned grid_for(long long n, int threads = 256, int cap = 4096)
{
    long long g = (n + threads - 1) / threads;
    return (unsigned)std::max<long long>(1, std::min<long long>(g, cap));
}

// ---------------------------------------------------------------------------
// FP64 helpers for the S-orthonormalization and the phase alignment.
// ---------------------------------------------------------------------------

// C = X^* X for X (rows x n, column-major, ld), C n x n column-major (FP64).
__global__ void __launch_bounds__(256)
zgram_full(const double2 *__restrict__ Xs, long long ld, int rows, int n, double2 *__restrict__ Cs)
{
    // item blockIdx.z: X = Xs + z ld n, C = Cs + z n n
    const double2 *X = Xs + (long long)blockIdx.z * ld * n;
    double2 *C = Cs + (long long)blockIdx.z * n * n;
    __shared__ double2 xs[16][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    double ar[4][4] = {}, ai[4][4] = {};
    __shared__ double2 ys[16][65];
    for (int k0 = 0; k0 < rows; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            const int k = e % 16, c = e / 16;
            xs[k][c] = (k0 + k < rows && i0 + c < n) ? X[(long long)(i0 + c) * ld + k0 + k] : make_double2(0, 0);
            ys[k][c] = (k0 + k < rows && j0 + c < n) ? X[(long long)(j0 + c) * ld + k0 + k] : make_double2(0, 0);
        }
        __syncthreads();
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const double2 x = xs[k][ty + 16 * a];
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const double2 y = ys[k][tx + 16 * b];
                    ar[a][b] = fma(x.x, y.x, fma(x.y, y.y, ar[a][b]));
                    ai[a][b] = fma(x.x, y.y, fma(-x.y, y.x, ai[a][b]));
                }
            }
        }
        __syncthreads();
    }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
            if (i < n && j < n) C[(long long)j * n + i] = make_double2(ar[a][b], ai[a][b]);
        }
}

// In one CTA: C = L L^* (lower triangle, in place, column-major n x n), then
// Xbuf = L^{-1} (thread j forms column j by forward substitution) and
// Binv = (L^{-1})^* (upper triangular, column-major), so that
// (G V0 Binv)^* (G V0 Binv) = I.  *bad = 1 if a pivot is not positive.
__global__ void __launch_bounds__(1024)
chol_inv(double2 *__restrict__ Cs, int n, double2 *__restrict__ Xbufs, double2 *__restrict__ Binvs,
         int *bad)
{
    // one CTA per matrix of the batch
    double2 *C = Cs + (long long)blockIdx.x * n * n;
    double2 *Xbuf = Xbufs + (long long)blockIdx.x * n * n;
    double2 *Binv = Binvs + (long long)blockIdx.x * n * n;
    __shared__ double piv;
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double d = C[(long long)k * n + k].x;
            if (!(d > 0.0)) *bad = 1;
            piv = d > 0.0 ? sqrt(d) : 1.0;
            C[(long long)k * n + k] = make_double2(piv, 0.0);
        }
        __syncthreads();
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
            const double2 v = C[(long long)k * n + i];
            C[(long long)k * n + i] = make_double2(v.x / piv, v.y / piv);
        }
        __syncthreads();
        // trailing lower triangle: C[i][j] -= L[i][k] conj(L[j][k]), n > i >= j > k
        const int m = n - k - 1;
        for (long long t = threadIdx.x; t < (long long)m * m; t += blockDim.x) {
            const int ii = (int)(t % m), jj = (int)(t / m);
            if (jj > ii) continue;
            const int i = k + 1 + ii, j = k + 1 + jj;
            const double2 a = C[(long long)k * n + i], b = C[(long long)k * n + j];
            double2 c = C[(long long)j * n + i];
            c.x -= a.x * b.x + a.y * b.y;
            c.y -= a.y * b.x - a.x * b.y;
            C[(long long)j * n + i] = c;
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        for (int i = 0; i < j; ++i) Xbuf[(long long)j * n + i] = make_double2(0.0, 0.0);
        for (int i = j; i < n; ++i) {
            double sr = i == j ? 1.0 : 0.0, si = 0.0;
            for (int q = j; q < i; ++q) {
                const double2 l = C[(long long)q * n + i], x = Xbuf[(long long)j * n + q];
                sr -= l.x * x.x - l.y * x.y;
                si -= l.x * x.y + l.y * x.x;
            }
            const double d = C[(long long)i * n + i].x;
            Xbuf[(long long)j * n + i] = make_double2(sr / d, si / d);
        }
    }
    __syncthreads();
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        const int r = (int)(t % n), c = (int)(t / n);     // Binv[r][c] = conj(X[c][r])
        const double2 x = Xbuf[(long long)r * n + c];
        Binv[(long long)c * n + r] = make_double2(x.x, -x.y);
    }
}

// Column phases: V[:, j] *= conj(c_j) / |c_j| with c_j = Vref[:, j]^* V[:, j]
// (makes each eigenvector's phase agree with a reference set).
__global__ void __launch_bounds__(256)
align_phases(const double2 *__restrict__ Vref, long long ldr, double2 *__restrict__ V, long long ldv,
             int n)
{
    __shared__ double rr[256], ri[256];
    const int j = blockIdx.x, tid = threadIdx.x;
    double sr = 0.0, si = 0.0;
    for (int i = tid; i < n; i += 256) {
        const double2 a = Vref[(long long)j * ldr + i], b = V[(long long)j * ldv + i];
        sr += a.x * b.x + a.y * b.y;
        si += a.x * b.y - a.y * b.x;
    }
    rr[tid] = sr;
    ri[tid] = si;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (tid < k) { rr[tid] += rr[tid + k]; ri[tid] += ri[tid + k]; }
        __syncthreads();
    }
    const double cr = rr[0], ci = ri[0], a = hypot(cr, ci);
    if (!(a > 0.0)) return;
    const double pr = cr / a, pi = -ci / a;           // conj(c) / |c|
    for (int i = tid; i < n; i += 256) {
        const double2 v = V[(long long)j * ldv + i];
        V[(long long)j * ldv + i] = make_double2(v.x * pr - v.y * pi, v.x * pi + v.y * pr);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// The MLP object
// ---------------------------------------------------------------------------
struct ghsvd_mlp {
    int device = 0;
    int nin = 0, nh = 0, nout = 0;
    long long np = 0;
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;   // params, grads, Adam moments
    long long adam_t = 0;
    int cap_batch = 0;
    float *A1 = nullptr, *A2 = nullptr, *Y = nullptr, *dY = nullptr, *dA2 = nullptr, *dA1 = nullptr;
    float *part = nullptr;
    long long cap_part = 0;
    double *lpart = nullptr;
    // offsets in the flat parameter vector
    long long oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
};

namespace {

void mlp_free_acts(ghsvd_mlp *m)
{
    cudaFree(m->A1); cudaFree(m->A2); cudaFree(m->Y); cudaFree(m->dY); cudaFree(m->dA2);
    cudaFree(m->dA1);
    m->A1 = m->A2 = m->Y = m->dY = m->dA2 = m->dA1 = nullptr;
    m->cap_batch = 0;
}

cudaError_t mlp_acts(ghsvd_mlp *m, int B)
{
    if (B <= m->cap_batch) return cudaSuccess;
    mlp_free_acts(m);
    cudaError_t e = cudaMalloc((void **)&m->A1, sizeof(float) * B * m->nh);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->A2, sizeof(float) * B * m->nh);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->Y, sizeof(float) * (size_t)B * m->nout);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->dY, sizeof(float) * (size_t)B * m->nout);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->dA2, sizeof(float) * B * m->nh);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->dA1, sizeof(float) * B * m->nh);
    if (e == cudaSuccess) m->cap_batch = B;
    return e;
}

// C (M x N) = op(A) op(B) [+ C], split over K when K is long and the output small.
cudaError_t sgemm(ghsvd_mlp *m, int M, int N, int K, const float *A, int lda, int ta, const float *B,
                  int ldb, int tb, float *C, int ldc, int accumulate, cudaStream_t st)
{
    const int tiles = ((M + 63) / 64) * ((N + 63) / 64);
    int splits = 1;
    if (tiles < 152 && K > 1024) splits = (int)std::min<long long>(64, std::max<long long>(1, (long long)304 / tiles));
    int kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + 15) / 16 * 16;
    splits = (K + kchunk - 1) / kchunk;
    dim3 grid((N + 63) / 64, (M + 63) / 64, splits);
    if (splits == 1) {
        sgemm_kernel<<<grid, 256, 0, st>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, accumulate, kchunk,
                                           nullptr);
        return cudaGetLastError();
    }
    const long long need = (long long)splits * M * N;
    if (need > m->cap_part) {
        cudaFree(m->part);
        m->part = nullptr;
        m->cap_part = 0;
        cudaError_t e = cudaMalloc((void **)&m->part, sizeof(float) * need);
        if (e != cudaSuccess) return e;
        m->cap_part = need;
    }
    sgemm_kernel<<<grid, 256, 0, st>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, accumulate, kchunk,
                                       m->part);
    reduce_splits<<<grid_for((long long)M * N), 256, 0, st>>>(M, N, splits, m->part, C, ldc, accumulate);
    return cudaGetLastError();
}

cudaError_t mlp_forward(ghsvd_mlp *m, int B, const float *X, float *Yout, cudaStream_t st)
{
    const float *P = m->P;
    cudaError_t e = sgemm(m, B, m->nh, m->nin, X, m->nin, 0, P + m->oW1, m->nin, 1, m->A1, m->nh, 0, st);
    if (e != cudaSuccess) return e;
    bias_act<<<grid_for((long long)B * m->nh), 256, 0, st>>>(m->A1, P + m->ob1, B, m->nh, 1);
    e = sgemm(m, B, m->nh, m->nh, m->A1, m->nh, 0, P + m->oW2, m->nh, 1, m->A2, m->nh, 0, st);
    if (e != cudaSuccess) return e;
    bias_act<<<grid_for((long long)B * m->nh), 256, 0, st>>>(m->A2, P + m->ob2, B, m->nh, 1);
    e = sgemm(m, B, m->nout, m->nh, m->A2, m->nh, 0, P + m->oW3, m->nh, 1, Yout, m->nout, 0, st);
    if (e != cudaSuccess) return e;
    bias_act<<<grid_for((long long)B * m->nout), 256, 0, st>>>(Yout, P + m->ob3, B, m->nout, 0);
    return cudaGetLastError();
}

// Loss (mean squared error) and its gradient w.r.t. the flat parameters, into m->G.
cudaError_t mlp_loss_grad(ghsvd_mlp *m, int B, const float *X, const float *T, double *loss,
                          cudaStream_t st)
{
    cudaError_t e = mlp_forward(m, B, X, m->Y, st);
    if (e != cudaSuccess) return e;
    const long long tot = (long long)B * m->nout;
    const unsigned gl = grid_for(tot, 256, 1024);
    mse_grad<<<gl, 256, 0, st>>>(m->Y, T, tot, 1.f / (float)tot, m->dY, m->lpart);
    float *G = m->G;
    const float *P = m->P;
    // layer 3
    e = sgemm(m, m->nout, m->nh, B, m->dY, m->nout, 1, m->A2, m->nh, 0, G + m->oW3, m->nh, 0, st);
    if (e != cudaSuccess) return e;
    colsum<<<(m->nout + 255) / 256, 256, 0, st>>>(m->dY, B, m->nout, G + m->ob3);
    e = sgemm(m, B, m->nh, m->nout, m->dY, m->nout, 0, P + m->oW3, m->nh, 0, m->dA2, m->nh, 0, st);
    if (e != cudaSuccess) return e;
    tanh_back<<<grid_for((long long)B * m->nh), 256, 0, st>>>(m->dA2, m->A2, (long long)B * m->nh);
    // layer 2
    e = sgemm(m, m->nh, m->nh, B, m->dA2, m->nh, 1, m->A1, m->nh, 0, G + m->oW2, m->nh, 0, st);
    if (e != cudaSuccess) return e;
    colsum<<<(m->nh + 255) / 256, 256, 0, st>>>(m->dA2, B, m->nh, G + m->ob2);
    e = sgemm(m, B, m->nh, m->nh, m->dA2, m->nh, 0, P + m->oW2, m->nh, 0, m->dA1, m->nh, 0, st);
    if (e != cudaSuccess) return e;
    tanh_back<<<grid_for((long long)B * m->nh), 256, 0, st>>>(m->dA1, m->A1, (long long)B * m->nh);
    // layer 1
    e = sgemm(m, m->nh, m->nin, B, m->dA1, m->nh, 1, X, m->nin, 0, G + m->oW1, m->nin, 0, st);
    if (e != cudaSuccess) return e;
    colsum<<<(m->nh + 255) / 256, 256, 0, st>>>(m->dA1, B, m->nh, G + m->ob1);
    if (loss) {
        std::vector<double> lp(gl);
        e = cudaMemcpyAsync(lp.data(), m->lpart, sizeof(double) * gl, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        double s = 0.0;
        for (double v : lp) s += v;
        *loss = s / (double)tot;
    }
    return cudaGetLastError();
}

// T_i = vec(V_i - Vref) as FP32 (re, im) pairs, column-major (the MLP's
// training targets), and the sum of their squares (FP64, one atomic per CTA).
__global__ void __launch_bounds__(256)
v0_targets_kernel(const double2 *__restrict__ Vref, long long ldr, const double2 *const *__restrict__ V,
                  const long long *__restrict__ ldv, int n, float *__restrict__ T, double *__restrict__ sumsq)
{
    __shared__ double red[8];
    const int i = blockIdx.y;
    const long long nn = (long long)n * n;
    const double2 *Vi = V[i];
    const long long lv = ldv[i];
    double acc = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % n), c = (int)(e / n);
        const double2 v = Vi[r + lv * c], w = Vref[r + ldr * c];
        const float dx = (float)(v.x - w.x), dy = (float)(v.y - w.y);
        T[(long long)i * 2 * nn + 2 * e] = dx;
        T[(long long)i * 2 * nn + 2 * e + 1] = dy;
        acc += (double)dx * dx + (double)dy * dy;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += red[k];
        atomicAdd(sumsq, s);
    }
}

__global__ void scale_f32(float *__restrict__ x, long long count, const double *__restrict__ sumsq, long long total)
{
    const double rms = sqrt(*sumsq / (double)total);
    const float f = rms > 0.0 ? (float)(1.0 / rms) : 1.0f;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x)
        x[e] *= f;
}

// V0_i = Vref + scale * D_i, D_i the FP32 (re, im) pairs of row i of Y
// (column-major n x n, the layout of the training targets).
__global__ void __launch_bounds__(256)
v0_compose_kernel(const float *__restrict__ Y, double scale, const double2 *__restrict__ Vref, long long ldr,
                  double2 *const *__restrict__ V0, const long long *__restrict__ ldv0, int n)
{
    const int i = blockIdx.y;
    const long long nn = (long long)n * n;
    double2 *Vi = V0[i];
    const long long lv = ldv0[i];
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % n), c = (int)(e / n);
        const double2 w = Vref[r + ldr * c];
        const float dx = Y[(long long)i * 2 * nn + 2 * e], dy = Y[(long long)i * 2 * nn + 2 * e + 1];
        Vi[r + lv * c] = make_double2(w.x + scale * dx, w.y + scale * dy);
    }
}

ghsvd_status st_of(cudaError_t e)
{
    if (e == cudaSuccess) return GHSVD_OK;
    return e == cudaErrorMemoryAllocation ? GHSVD_ERR_NOMEM : GHSVD_ERR_CUDA;
}

struct DevGuard {
    int prev = 0;
    bool ok = false;
    explicit DevGuard(int d) { cudaGetDevice(&prev); ok = cudaSetDevice(d) == cudaSuccess; }
    ~DevGuard() { cudaSetDevice(prev); }
};

// p is device (or managed) memory of `device` (-1: the current device).
bool dev_ok(const void *p, int device = -1)
{
    if (!p) return false;
    if (device < 0 && cudaGetDevice(&device) != cudaSuccess) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}

}  // namespace

extern "C" {

ghsvd_status ghsvd_mlp_create(ghsvd_mlp_t *out, int device, int n_in, int n_hidden, int n_out,
                              uint64_t seed)
{
    if (!out || n_in < 1 || n_hidden < 1 || n_out < 1) return GHSVD_ERR_INVALID_ARG;
    *out = nullptr;
    DevGuard g(device);
    if (!g.ok) return GHSVD_ERR_INVALID_ARG;
    ghsvd_mlp *m = new (std::nothrow) ghsvd_mlp();
    if (!m) return GHSVD_ERR_NOMEM;
    m->device = device;
    m->nin = n_in; m->nh = n_hidden; m->nout = n_out;
    m->oW1 = 0;
    m->ob1 = m->oW1 + (long long)n_hidden * n_in;
    m->oW2 = m->ob1 + n_hidden;
    m->ob2 = m->oW2 + (long long)n_hidden * n_hidden;
    m->oW3 = m->ob2 + n_hidden;
    m->ob3 = m->oW3 + (long long)n_out * n_hidden;
    m->np = m->ob3 + n_out;
    cudaError_t e = cudaMalloc((void **)&m->P, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->G, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->M, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->V, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->lpart, sizeof(double) * 1024);
    if (e == cudaSuccess) {
        // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
        init_uniform<<<grid_for(m->ob1), 256>>>(m->P + m->oW1, m->ob1, seed, 1.f / sqrtf((float)n_in));
        init_uniform<<<grid_for(m->ob2 - m->oW2), 256>>>(m->P + m->oW2, m->ob2 - m->oW2, seed + 1,
                                                        1.f / sqrtf((float)n_hidden));
        init_uniform<<<grid_for(m->ob3 - m->oW3), 256>>>(m->P + m->oW3, m->ob3 - m->oW3, seed + 2,
                                                        1.f / sqrtf((float)n_hidden));
        cudaMemset(m->P + m->ob1, 0, sizeof(float) * n_hidden);
        cudaMemset(m->P + m->ob2, 0, sizeof(float) * n_hidden);
        cudaMemset(m->P + m->ob3, 0, sizeof(float) * n_out);
        cudaMemset(m->M, 0, sizeof(float) * m->np);
        cudaMemset(m->V, 0, sizeof(float) * m->np);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        ghsvd_mlp_destroy(m);
        return st_of(e);
    }
    *out = m;
    return GHSVD_OK;
}

void ghsvd_mlp_destroy(ghsvd_mlp_t m)
{
    if (!m) return;
    DevGuard g(m->device);
    mlp_free_acts(m);
    cudaFree(m->P); cudaFree(m->G); cudaFree(m->M); cudaFree(m->V); cudaFree(m->part);
    cudaFree(m->lpart);
    delete m;
}

ghsvd_status ghsvd_mlp_size(ghsvd_mlp_t m, int64_t *count)
{
    if (!m || !count) return GHSVD_ERR_INVALID_ARG;
    *count = m->np;
    return GHSVD_OK;
}

ghsvd_status ghsvd_mlp_get(ghsvd_mlp_t m, int what, float *dst)
{
    if (!m || !dst || (what != 0 && what != 1)) return GHSVD_ERR_INVALID_ARG;
    DevGuard g(m->device);
    return st_of(cudaMemcpy(dst, what ? m->G : m->P, sizeof(float) * m->np, cudaMemcpyDefault));
}

ghsvd_status ghsvd_mlp_set(ghsvd_mlp_t m, const float *src)
{
    if (!m || !src) return GHSVD_ERR_INVALID_ARG;
    DevGuard g(m->device);
    return st_of(cudaMemcpy(m->P, src, sizeof(float) * m->np, cudaMemcpyDefault));
}

ghsvd_status ghsvd_mlp_forward(ghsvd_mlp_t m, int batch, const float *X, float *Y, void *stream)
{
    if (!m || batch < 1 || !dev_ok(X, m->device) || !dev_ok(Y, m->device)) return GHSVD_ERR_INVALID_ARG;
    DevGuard g(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = mlp_acts(m, batch);
    if (e == cudaSuccess) e = mlp_forward(m, batch, X, Y, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return st_of(e);
}

ghsvd_status ghsvd_mlp_loss_grad(ghsvd_mlp_t m, int batch, const float *X, const float *T,
                                 double *loss, void *stream)
{
    if (!m || batch < 1 || !dev_ok(X, m->device) || !dev_ok(T, m->device)) return GHSVD_ERR_INVALID_ARG;
    DevGuard g(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = mlp_acts(m, batch);
    if (e == cudaSuccess) e = mlp_loss_grad(m, batch, X, T, loss, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return st_of(e);
}

ghsvd_status ghsvd_mlp_train(ghsvd_mlp_t m, int n_samples, const float *X, const float *T,
                             int epochs, int batch, float lr, double *final_loss, void *stream)
{
    if (!m || n_samples < 1 || !dev_ok(X, m->device) || !dev_ok(T, m->device) || epochs < 1 || batch < 1 ||
        !(lr > 0.f))
        return GHSVD_ERR_INVALID_ARG;
    DevGuard g(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    batch = std::min(batch, n_samples);
    cudaError_t e = mlp_acts(m, batch);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double loss = 0.0, epoch_loss = 0.0;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        epoch_loss = 0.0;
        for (int s0 = 0; s0 < n_samples && e == cudaSuccess; s0 += batch) {
            const int B = std::min(batch, n_samples - s0);
            const bool last = ep == epochs - 1;
            e = mlp_loss_grad(m, B, X + (long long)s0 * m->nin, T + (long long)s0 * m->nout,
                              last ? &loss : nullptr, st);
            if (e != cudaSuccess) break;
            m->adam_t += 1;
            const float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
            adam_step<<<grid_for(m->np), 256, 0, st>>>(m->P, m->G, m->M, m->V, m->np, lr, b1, b2, c1,
                                                        c2, eps);
            e = cudaGetLastError();
            if (last) epoch_loss += loss * B;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (final_loss) *final_loss = epoch_loss / n_samples;
    return st_of(e);
}

ghsvd_status ghsvd_s_orthonormalize(int count, int64_t p, int64_t n, const void *const *G,
                                    const int64_t *ldg, void *const *V0, const int64_t *ldv0,
                                    void *stream)
{
    if (count < 1 || p < n || n < 1 || n > 4096 || !G || !V0 || !ldg || !ldv0)
        return GHSVD_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (!dev_ok(G[i]) || !dev_ok(V0[i]) || ldg[i] < p || ldv0[i] < n) return GHSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // for every pair: X = G V0 (p x n), C = X^* X = L L^*, V0 <- V0 (L^{-1})^*;
    // each stage is one batched launch over all pairs
    double2 *X = nullptr, *C = nullptr, *Xb = nullptr, *B = nullptr, *Y = nullptr;
    hz::GemmItem *items = nullptr;
    int *bad = nullptr;
    const long long pn = p * n, nn = n * n;
    cudaError_t e = cudaMallocAsync((void **)&X, 16LL * count * pn, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&C, 16LL * count * nn, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&Xb, 16LL * count * nn, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&B, 16LL * count * nn, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&Y, 16LL * count * nn, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&items, sizeof(hz::GemmItem) * count, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&bad, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), st);
    std::vector<hz::GemmItem> it(count);
    for (int i = 0; i < count; ++i)
        it[i] = {(const double2 *)G[i], ldg[i], p, (const double2 *)V0[i], ldv0[i], X + i * pn, p, (int)n, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(items, it.data(), sizeof(hz::GemmItem) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = hz::launch_gemm_batched(items, count, p, (int)n, st);
    if (e == cudaSuccess) {
        dim3 grid((unsigned)((n + 63) / 64), (unsigned)((n + 63) / 64), (unsigned)count);
        zgram_full<<<grid, 256, 0, st>>>(X, p, (int)p, (int)n, C);
        chol_inv<<<count, 1024, 0, st>>>(C, (int)n, Xb, B, bad);
        e = cudaGetLastError();
    }
    for (int i = 0; i < count; ++i)
        it[i] = {(const double2 *)V0[i], ldv0[i], n, B + i * nn, n, Y + i * nn, n, (int)n, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(items, it.data(), sizeof(hz::GemmItem) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = hz::launch_gemm_batched(items, count, n, (int)n, st);
    for (int i = 0; i < count; ++i)
        it[i] = {Y + i * nn, n, n, nullptr, 0, (double2 *)V0[i], ldv0[i], (int)n, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(items, it.data(), sizeof(hz::GemmItem) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = hz::launch_copy_batched(items, count, st);
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(X, st); cudaFreeAsync(C, st); cudaFreeAsync(Xb, st); cudaFreeAsync(B, st);
    cudaFreeAsync(Y, st); cudaFreeAsync(items, st); cudaFreeAsync(bad, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return st_of(e);
    return hbad ? GHSVD_ERR_RANK_DEFICIENT : GHSVD_OK;
}

ghsvd_status ghsvd_v0_targets(int count, int64_t n, const void *Vref, int64_t ldr, const void *const *V,
                              const int64_t *ldv, float *T, double *rms, void *stream)
{
    if (count < 1 || n < 1 || n > 4096 || !dev_ok(Vref) || ldr < n || !V || !ldv || !dev_ok(T))
        return GHSVD_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (!dev_ok(V[i]) || ldv[i] < n) return GHSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const double2 **dV = nullptr;
    long long *dl = nullptr;
    double *sumsq = nullptr;
    std::vector<long long> lv(ldv, ldv + count);
    cudaError_t e = cudaMallocAsync((void **)&dV, sizeof(void *) * count, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dl, sizeof(long long) * count, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&sumsq, sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dV, V, sizeof(void *) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dl, lv.data(), sizeof(long long) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sumsq, 0, sizeof(double), st);
    const long long nn = n * n, total = 2LL * nn * count;
    if (e == cudaSuccess) {
        dim3 grid((unsigned)std::min<long long>((nn + 255) / 256, 1024), (unsigned)count);
        v0_targets_kernel<<<grid, 256, 0, st>>>((const double2 *)Vref, ldr, dV, dl, (int)n, T, sumsq);
        scale_f32<<<1024, 256, 0, st>>>(T, total, sumsq, total);
        e = cudaGetLastError();
    }
    double hs = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, sumsq, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(dV, st);
    cudaFreeAsync(dl, st);
    cudaFreeAsync(sumsq, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (rms) *rms = sqrt(hs / (double)total);
    return st_of(e);
}

ghsvd_status ghsvd_v0_compose(int count, int64_t n, const float *Y, double scale, const void *Vref, int64_t ldr,
                              void *const *V0, const int64_t *ldv0, void *stream)
{
    if (count < 1 || n < 1 || n > 4096 || !dev_ok(Y) || !dev_ok(Vref) || ldr < n || !V0 || !ldv0)
        return GHSVD_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (!dev_ok(V0[i]) || ldv0[i] < n) return GHSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double2 **dV = nullptr;
    long long *dl = nullptr;
    std::vector<long long> lv(ldv0, ldv0 + count);
    cudaError_t e = cudaMallocAsync((void **)&dV, sizeof(void *) * count, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dl, sizeof(long long) * count, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dV, V0, sizeof(void *) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dl, lv.data(), sizeof(long long) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const long long nn = n * n;
        dim3 grid((unsigned)std::min<long long>((nn + 255) / 256, 1024), (unsigned)count);
        v0_compose_kernel<<<grid, 256, 0, st>>>(Y, scale, (const double2 *)Vref, ldr, dV, dl, (int)n);
        e = cudaGetLastError();
    }
    cudaFreeAsync(dV, st);
    cudaFreeAsync(dl, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return st_of(e);
}

ghsvd_status ghsvd_align_phases(int64_t n, const void *Vref, int64_t ldr, void *V, int64_t ldv,
                                void *stream)
{
    if (n < 1 || !dev_ok(Vref) || !dev_ok(V) || ldr < n || ldv < n) return GHSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    align_phases<<<(unsigned)n, 256, 0, st>>>((const double2 *)Vref, ldr, (double2 *)V, ldv, (int)n);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return st_of(e);
}

}  // extern "C"
