// hz_urv.cu -- Phase 2 of arXiv 1907.08560 (Section 5): the optional (J, I)
// URV shortening of the tall factors before the Hari-Zimmermann iteration.
//
//   F~ (m x n, signature J~) is reduced by the hyperbolic QR: at each step the
//   diagonal pivoting and the Bunch-Kaufman partial pivoting of Section 5.2
//   choose one pivot column or two, a row exchange brings a sign equal to the
//   sign of the pivot's J-norm to the top, and hyperbolic Householder
//   reflectors H(s) = I + tau s s^* J_k (Theorem 5.1, Section 5.3) reduce the
//   pivot column(s); a 2x2 pivot is first made J-orthogonal by a Jacobi
//   rotation R_k and its block is multiplied by R_k^* at the end.
//   G~ P2 (p x n) is reduced by the Householder QR.
//
// The column steps are sequential; each is a short chain of kernels whose
// decisions (pivot columns, pivot kind, reflector) live in a device-side
// state, so the host enqueues the whole factorization without synchronizing.
// Single-CTA kernels take the decisions; the reflector is applied by one CTA
// per trailing column, which also forms the column's J-norm for the next
// step's diagonal pivoting.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hz_launch.h"

namespace hz {
namespace {

constexpr int NT1 = 1024;      // threads of a decision kernel (one CTA)
constexpr int NTA = 256;       // threads of a column CTA
constexpr int REG = 16;        // column entries a thread keeps in registers
constexpr double BK_ALPHA = 0.6403882032022076;   // (1 + sqrt(17)) / 8, correctly rounded

struct UrvState {
    int k;          // first column of the current step
    int knext;      // first column of the next step
    int kind;       // 0: no step (finished or failed), 1: single pivot, 2: 2x2 pivot
    int need1;      // the step needs |h_1j| (k < n - 1)
    int need2;      // the Bunch-Kaufman test needs sigma
    int ii;         // column of the largest |h_1j|
    double lam;     // |h_1,ii|
    int err;        // breakdown (reading: the oracle's P24_ERR_BREAKDOWN)
    int n2x2;       // 2x2 pivots taken
    int apply1;     // reflector 1 (rows k.., columns k+1..) is applied
    double tau1;
    int apply2;     // reflector 2 of a 2x2 pivot (rows k+1.., columns k+2..)
    double tau2;
    double2 R[4];   // Jacobi rotation of the 2x2 pivot, row-major
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double abs2(double2 a) { return a.x * a.x + a.y * a.y; }

// ---- block reductions (fixed order: deterministic) -------------------------
// Block reductions.  The last stage runs in one thread (sum, in warp order)
// or one warp (argmax) and is broadcast through shared memory: on GB300 a
// warp's FP64 instruction holds its sub-partition's FP64 pipe for 64 cycles,
// so NT threads each repeating the last stage cost NT/32 times as much.
template <int NT>
__device__ double block_sum(double v, double *sh)
{
    __shared__ double s_sum;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int i = 0; i < NT / 32; ++i) r += sh[i];
        s_sum = r;
    }
    __syncthreads();
    const double r = s_sum;
    __syncthreads();
    return r;
}

template <int NT>
__device__ double2 block_sum2(double2 v, double *sh)
{
    const double a = block_sum<NT>(v.x, sh);
    const double b = block_sum<NT>(v.y, sh);
    return make_double2(a, b);
}

// (value, index) maximum: larger value wins, equal values go to the smaller index.
__device__ __forceinline__ void better(double &v, int &i, double v2, int i2)
{
    if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

// (better is a total order on the values that can win -- NaN never does --
// so the tree in warp 0 picks what a scan in warp order would.)
template <int NT>
__device__ void block_argmax(double &v, int &i, double *shv, int *shi)
{
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
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
            const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
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

__device__ void swap_cols(double2 *F, long long ld, int m, int a, int b)
{
    if (a == b) return;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        const double2 t = F[r + ld * a];
        F[r + ld * a] = F[r + ld * b];
        F[r + ld * b] = t;
    }
}

__device__ void swap_rows(double2 *F, long long ld, int n, int a, int b)
{
    if (a == b) return;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const double2 t = F[a + ld * c];
        F[a + ld * c] = F[b + ld * c];
        F[b + ld * c] = t;
    }
}

// ---- J-norms of all columns over rows k0.. (one warp per column) ----------
__global__ void __launch_bounds__(256)
urv_norms(const double2 *__restrict__ F, long long ld, int m, int n, const int8_t *__restrict__ J,
          int k0, double *__restrict__ h)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < n; c += nw) {
        double s = 0.0;
        for (int r = k0 + lane; r < m; r += 32) s += (double)J[r] * abs2(F[r + ld * c]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) h[c] = s;
    }
}

// ---- step part 1: diagonal pivoting (Section 5.2.1) -----------------------
__global__ void __launch_bounds__(NT1)
urv_select(double2 *__restrict__ F, long long ld, int m, int n, int *__restrict__ perm,
           double *__restrict__ h, UrvState *__restrict__ st)
{
    __shared__ double shv[32];
    __shared__ int shi[32];
    __shared__ int sk;
    if (threadIdx.x == 0) {
        st->k = st->knext;
        sk = (st->err || st->k >= n) ? -1 : st->k;
        st->kind = 0;
        st->need1 = 0;
        st->need2 = 0;
        st->apply1 = 0;
        st->apply2 = 0;
    }
    __syncthreads();
    const int k = sk;
    if (k < 0) return;
    double v = -1.0;
    int idx = n;
    for (int i = k + threadIdx.x; i < n; i += NT1) better(v, idx, fabs(h[i]), i);
    block_argmax<NT1>(v, idx, shv, shi);
    if (idx >= n) idx = k;                  // no comparable norm (NaN): keep the order
    if (idx != k) {
        swap_cols(F, ld, m, k, idx);
        if (threadIdx.x == 0) {
            const int tp = perm[k]; perm[k] = perm[idx]; perm[idx] = tp;
            const double th = h[k]; h[k] = h[idx]; h[idx] = th;
        }
    }
    if (threadIdx.x == 0) {
        st->kind = 1;
        st->need1 = k < n - 1;
    }
}

// ---- |J_k-dot| of a pivot column with the other columns (one warp each) ---
// mode 1: out[j] = |f_k^* J_k f_j|, j > k.  mode 2: out[l] = |f_ii^* J_k f_l|,
// l >= k, l != ii (out[ii] = 0).
__global__ void __launch_bounds__(256)
urv_dots(const double2 *__restrict__ F, long long ld, int m, int n, const int8_t *__restrict__ J,
         const UrvState *__restrict__ st, int mode, double *__restrict__ out)
{
    if (mode == 1 ? !st->need1 : !st->need2) return;
    const int k = st->k;
    const int pc = mode == 1 ? k : st->ii;
    const int c0 = mode == 1 ? k + 1 : k;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const double2 *a = F + ld * pc;
    for (int c = c0 + warp; c < n; c += nw) {
        if (c == pc) {
            if (lane == 0) out[c] = 0.0;
            continue;
        }
        const double2 *b = F + ld * c;
        double sr = 0.0, si = 0.0;
        for (int r = k + lane; r < m; r += 32) {
            const double2 x = a[r], y = b[r];
            const double j = (double)J[r];
            sr += j * (x.x * y.x + x.y * y.y);
            si += j * (x.x * y.y - x.y * y.x);
        }
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) out[c] = hypot(sr, si);
    }
}

// ---- step part 2: the first Bunch-Kaufman test ----------------------------
__global__ void __launch_bounds__(NT1)
urv_bk1(const double *__restrict__ h, const double *__restrict__ mag, int n, UrvState *__restrict__ st)
{
    __shared__ double shv[32];
    __shared__ int shi[32];
    if (!st->need1) return;
    const int k = st->k;
    double v = -1.0;
    int idx = n;
    for (int j = k + 1 + threadIdx.x; j < n; j += NT1) better(v, idx, mag[j], j);
    block_argmax<NT1>(v, idx, shv, shi);
    if (idx >= n) idx = k + 1;              // no comparable product (NaN)
    if (threadIdx.x == 0) {
        st->ii = idx;
        st->lam = v;
        st->need2 = !(fabs(h[k]) >= BK_ALPHA * v);
    }
}

// Reflector of column c over rows r0.. (Section 5.3): row exchange for the
// sign, s = f + c1 e_r0, tau; the column becomes -c1 e_r0.  Returns through
// the state: *apply = 0 for a zero column, st->err on a breakdown.
__device__ void reflect_setup(double2 *__restrict__ F, long long ld, int m, int n, int8_t *__restrict__ J,
                              int c, int r0, double2 *__restrict__ s, UrvState *st, int *apply,
                              double *tau_out, double *sh, int *shi)
{
    double2 *f = F + ld * c;
    double part = 0.0;
    int nz = 0;
    for (int r = r0 + threadIdx.x; r < m; r += blockDim.x) {
        const double2 x = f[r];
        part += (double)J[r] * abs2(x);
        nz |= (x.x != 0.0 || x.y != 0.0);
    }
    const double h = block_sum<NT1>(part, sh);
    nz = __syncthreads_or(nz);
    if (h == 0.0) {
        if (threadIdx.x == 0) {
            *apply = 0;
            if (nz) { st->err = 1; st->knext = n; }
        }
        return;
    }
    const int sg = h > 0.0 ? 1 : -1;
    if (J[r0] != sg) {
        double v = -1.0;
        int idx = m;
        for (int r = r0 + 1 + threadIdx.x; r < m; r += blockDim.x)
            if (J[r] == sg) better(v, idx, hypot(f[r].x, f[r].y), r);
        block_argmax<NT1>(v, idx, sh, shi);
        if (idx >= m) {
            if (threadIdx.x == 0) { *apply = 0; st->err = 1; st->knext = n; }
            return;
        }
        swap_rows(F, ld, n, r0, idx);
        __syncthreads();
        if (threadIdx.x == 0) { const int8_t t = J[r0]; J[r0] = J[idx]; J[idx] = t; }
        __syncthreads();
    }
    const double2 f0 = f[r0];
    const double r1 = hypot(f0.x, f0.y);
    const double2 eid = r1 > 0.0 ? make_double2(f0.x / r1, f0.y / r1) : make_double2(1.0, 0.0);
    const double rh = sqrt(fabs(h));
    const double2 c1 = cscale(eid, rh);
    const double tau = -1.0 / (h + rh * r1 * (double)J[r0]);
    __syncthreads();
    for (int r = r0 + threadIdx.x; r < m; r += blockDim.x) {
        const double2 x = f[r];
        s[r] = r == r0 ? cadd(x, c1) : x;
        f[r] = r == r0 ? make_double2(-c1.x, -c1.y) : make_double2(0.0, 0.0);
    }
    if (threadIdx.x == 0) {
        *apply = 1;
        *tau_out = tau;
    }
}

// ---- step part 3: the rest of Section 5.2, the 2x2 rotation, reflector 1 --
__global__ void __launch_bounds__(NT1)
urv_pivot(double2 *__restrict__ F, long long ld, int m, int n, int8_t *__restrict__ J,
          int *__restrict__ perm, double *__restrict__ h, const double *__restrict__ mag2,
          double2 *__restrict__ s, UrvState *__restrict__ st)
{
    __shared__ double sh[32];
    __shared__ int shi[32];
    __shared__ int skind, sswap_a, sswap_b;
    if (st->kind == 0) return;
    const int k = st->k;
    if (threadIdx.x == 0) { skind = 1; sswap_a = sswap_b = -1; }
    if (st->need2) {
        double v = -1.0;
        int idx = n;
        const int ii = st->ii;
        for (int l = k + threadIdx.x; l < n; l += NT1)
            if (l != ii) better(v, idx, mag2[l], l);
        block_argmax<NT1>(v, idx, sh, shi);
        if (threadIdx.x == 0) {
            const double sig = v, lam = st->lam;
            if (fabs(h[k]) * sig >= BK_ALPHA * lam * lam) {
                // single pivot: column k
            } else if (fabs(h[ii]) >= BK_ALPHA * sig) {
                sswap_a = k; sswap_b = ii;
            } else {
                skind = 2;
                if (ii != k + 1) { sswap_a = k + 1; sswap_b = ii; }
            }
        }
        __syncthreads();
        if (sswap_a >= 0) {
            swap_cols(F, ld, m, sswap_a, sswap_b);
            if (threadIdx.x == 0) {
                const int tp = perm[sswap_a]; perm[sswap_a] = perm[sswap_b]; perm[sswap_b] = tp;
                const double th = h[sswap_a]; h[sswap_a] = h[sswap_b]; h[sswap_b] = th;
            }
            __syncthreads();
        }
    }
    const int kind = skind;
    if (kind == 2) {
        double2 *f1 = F + ld * k, *f2 = F + ld * (k + 1);
        double p11 = 0.0, p22 = 0.0;
        double2 p12 = make_double2(0.0, 0.0);
        for (int r = k + threadIdx.x; r < m; r += NT1) {
            const double2 x = f1[r], y = f2[r];
            const double j = (double)J[r];
            p11 += j * abs2(x);
            p22 += j * abs2(y);
            p12.x += j * (x.x * y.x + x.y * y.y);
            p12.y += j * (x.x * y.y - x.y * y.x);
        }
        const double a11 = block_sum<NT1>(p11, sh);
        const double a22 = block_sum<NT1>(p22, sh);
        const double2 a12 = block_sum2<NT1>(p12, sh);
        const double b = hypot(a12.x, a12.y);
        const double2 eth = b > 0.0 ? make_double2(a12.x / b, a12.y / b) : make_double2(1.0, 0.0);
        double c = 1.0, sn = 0.0;
        if (b > 0.0) {
            const double zeta = (a22 - a11) / (2.0 * b);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
        }
        // R = diag(1, conj(e^{i theta})) [c s; -s c]
        const double2 R11 = make_double2(c, 0.0), R12 = make_double2(sn, 0.0);
        const double2 R21 = cscale(cconj(eth), -sn), R22 = cscale(cconj(eth), c);
        for (int r = k + threadIdx.x; r < m; r += NT1) {
            const double2 x = f1[r], y = f2[r];
            f1[r] = cadd(cmul(x, R11), cmul(y, R21));
            f2[r] = cadd(cmul(x, R12), cmul(y, R22));
        }
        if (threadIdx.x == 0) {
            st->R[0] = R11; st->R[1] = R12; st->R[2] = R21; st->R[3] = R22;
        }
        __syncthreads();
    }
    __shared__ int sapply;
    __shared__ double stau;
    reflect_setup(F, ld, m, n, J, k, k, s, st, &sapply, &stau, sh, shi);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (st->err) {
            st->kind = 0;
            st->apply1 = 0;
        } else {
            st->kind = kind;
            st->apply1 = sapply;
            st->tau1 = stau;
            st->knext = k + kind;
            st->n2x2 += kind == 2;
        }
    }
}

// ---- reflector application: one CTA per trailing column --------------------
// f_j <- f_j + tau s (s^* J f_j) over rows kr.., then h_j = J-norm over rows
// kr+1.. (the next step's diagonal pivoting).  A step whose reflector was
// skipped (a zero pivot column) still refreshes the norms.
__global__ void __launch_bounds__(NTA)
urv_apply(double2 *__restrict__ F, long long ld, int m, int n, const int8_t *__restrict__ J,
          const double2 *__restrict__ s, double *__restrict__ h, const UrvState *__restrict__ st,
          int which)
{
    __shared__ double sh[32];
    const int on = which == 1 ? st->kind != 0 : st->kind == 2;
    if (!on) return;
    const int kr = st->k + which - 1;
    const int first = st->k + (which == 1 ? 1 : 2);
    const int refl = which == 1 ? st->apply1 : st->apply2;
    const double tau = which == 1 ? st->tau1 : st->tau2;
    for (int c = first + blockIdx.x; c < n; c += gridDim.x) {
        double2 *f = F + ld * c;
        double2 v[REG];
        double dr = 0.0, di = 0.0;
#pragma unroll
        for (int t = 0; t < REG; ++t) {
            const int r = kr + threadIdx.x + NTA * t;
            if (r < m) {
                v[t] = f[r];
                if (refl) {
                    const double2 a = s[r];
                    const double j = (double)J[r];
                    dr += j * (a.x * v[t].x + a.y * v[t].y);
                    di += j * (a.x * v[t].y - a.y * v[t].x);
                }
            }
        }
        if (refl)
            for (int r = kr + threadIdx.x + NTA * REG; r < m; r += NTA) {
                const double2 x = f[r], a = s[r];
                const double j = (double)J[r];
                dr += j * (a.x * x.x + a.y * x.y);
                di += j * (a.x * x.y - a.y * x.x);
            }
        double2 t = make_double2(0.0, 0.0);
        if (refl) t = cscale(block_sum2<NTA>(make_double2(dr, di), sh), tau);
        double nn = 0.0;
#pragma unroll
        for (int u = 0; u < REG; ++u) {
            const int r = kr + threadIdx.x + NTA * u;
            if (r < m) {
                double2 x = v[u];
                if (refl) {
                    x = cadd(x, cmul(t, s[r]));
                    f[r] = x;
                }
                if (r > kr) nn += (double)J[r] * abs2(x);
            }
        }
        for (int r = kr + threadIdx.x + NTA * REG; r < m; r += NTA) {
            double2 x = f[r];
            if (refl) {
                x = cadd(x, cmul(t, s[r]));
                f[r] = x;
            }
            nn += (double)J[r] * abs2(x);
        }
        const double hn = block_sum<NTA>(nn, sh);
        if (threadIdx.x == 0) h[c] = hn;
    }
}

// ---- step part 4: the second reflector of a 2x2 pivot and R_k^* -----------
__global__ void __launch_bounds__(NT1)
urv_reflect2(double2 *__restrict__ F, long long ld, int m, int n, int8_t *__restrict__ J,
             double2 *__restrict__ s, UrvState *__restrict__ st)
{
    __shared__ double sh[32];
    __shared__ int shi[32];
    __shared__ int sapply;
    __shared__ double stau;
    if (st->kind != 2) return;
    const int k = st->k;
    reflect_setup(F, ld, m, n, J, k + 1, k + 1, s, st, &sapply, &stau, sh, shi);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (st->err) {
            st->apply2 = 0;
            st->kind = 0;
            return;
        }
        // the 2x2 block (rows k, k+1 of columns k, k+1) times R^*
        double2 *f1 = F + ld * k, *f2 = F + ld * (k + 1);
        const double2 R11 = st->R[0], R12 = st->R[1], R21 = st->R[2], R22 = st->R[3];
        for (int r = k; r < k + 2; ++r) {
            const double2 x = f1[r], y = f2[r];
            f1[r] = cadd(cmul(x, cconj(R11)), cmul(y, cconj(R12)));
            f2[r] = cadd(cmul(x, cconj(R21)), cmul(y, cconj(R22)));
        }
        st->apply2 = sapply;
        st->tau2 = stau;
    }
}

__global__ void urv_init(int n, int *__restrict__ perm, UrvState *__restrict__ st)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) perm[j] = j;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        UrvState z{};
        *st = z;
    }
}

// J~ as signs: the caller's vector, or n_plus positives then negatives
__global__ void urv_signs(const int8_t *__restrict__ J, long long n_plus, int m, int8_t *__restrict__ Jw,
                          int *__restrict__ bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        int8_t v = J ? J[i] : (i < n_plus ? 1 : -1);
        if (v != 1 && v != -1) { *bad = 1; v = 1; }
        Jw[i] = v;
    }
}

// ---- Householder QR of G~ P2 ------------------------------------------------
struct QrState {
    double beta[2];
};

// Gw[:, j] = G[:, perm[j]]
__global__ void qr_gather(const double2 *__restrict__ G, long long ldg, int p, const int *__restrict__ perm,
                          double2 *__restrict__ Gw, long long ldw)
{
    const int j = blockIdx.x;
    const double2 *src = G + ldg * perm[j];
    for (int r = threadIdx.x; r < p; r += blockDim.x) Gw[r + ldw * j] = src[r];
}

// Reflector of column c from its rows c.. held by this CTA (x in registers or
// re-read): v = x - alpha e_c, beta = 1 / (||x|| (||x|| + |x_c|)), column := alpha e_c.
__device__ void qr_make(double2 *__restrict__ g, int c, int p, const double2 *v, double2 *__restrict__ vb,
                        double *beta, double *sh)
{
    double part = 0.0;
#pragma unroll
    for (int t = 0; t < REG; ++t) {
        const int r = c + threadIdx.x + NTA * t;
        if (r < p) part += abs2(v[t]);
    }
    for (int r = c + threadIdx.x + NTA * REG; r < p; r += NTA) part += abs2(g[r]);
    const double nrm2 = block_sum<NTA>(part, sh);
    const double nrm = sqrt(nrm2);
    const double2 xc = g[c];
    __syncthreads();
    if (nrm == 0.0) {
        if (threadIdx.x == 0) *beta = 0.0;
        return;
    }
    const double ax = hypot(xc.x, xc.y);
    const double2 ph = ax > 0.0 ? make_double2(xc.x / ax, xc.y / ax) : make_double2(1.0, 0.0);
    const double2 alpha = make_double2(-ph.x * nrm, -ph.y * nrm);
#pragma unroll
    for (int t = 0; t < REG; ++t) {
        const int r = c + threadIdx.x + NTA * t;
        if (r < p) {
            vb[r] = r == c ? make_double2(v[t].x - alpha.x, v[t].y - alpha.y) : v[t];
            g[r] = r == c ? alpha : make_double2(0.0, 0.0);
        }
    }
    for (int r = c + threadIdx.x + NTA * REG; r < p; r += NTA) {
        vb[r] = g[r];
        g[r] = make_double2(0.0, 0.0);
    }
    if (threadIdx.x == 0) *beta = 1.0 / (nrm * (nrm + ax));
}

__global__ void __launch_bounds__(NTA)
qr_first(double2 *__restrict__ Gw, long long ld, int p, double2 *__restrict__ vb, QrState *__restrict__ qs)
{
    __shared__ double sh[32];
    double2 v[REG];
#pragma unroll
    for (int t = 0; t < REG; ++t) {
        const int r = threadIdx.x + NTA * t;
        v[t] = r < p ? Gw[r] : make_double2(0.0, 0.0);
    }
    qr_make(Gw, 0, p, v, vb, &qs->beta[0], sh);
}

// Step k: apply reflector k (vb[k & 1]) to columns k+1..n-1; the CTA of column
// k+1 then makes reflector k+1 into vb[(k+1) & 1].
__global__ void __launch_bounds__(NTA)
qr_step(double2 *__restrict__ Gw, long long ld, int p, int n, int k, double2 *__restrict__ vbuf,
        long long vstride, QrState *__restrict__ qs)
{
    __shared__ double sh[32];
    const int c = k + 1 + blockIdx.x;
    if (c >= n) return;
    const double2 *vb = vbuf + vstride * (k & 1);
    const double beta = qs->beta[k & 1];
    double2 *g = Gw + ld * c;
    double2 v[REG];
    double dr = 0.0, di = 0.0;
#pragma unroll
    for (int t = 0; t < REG; ++t) {
        const int r = k + threadIdx.x + NTA * t;
        if (r < p) {
            v[t] = g[r];
            const double2 a = vb[r];
            dr += a.x * v[t].x + a.y * v[t].y;
            di += a.x * v[t].y - a.y * v[t].x;
        }
    }
    for (int r = k + threadIdx.x + NTA * REG; r < p; r += NTA) {
        const double2 x = g[r], a = vb[r];
        dr += a.x * x.x + a.y * x.y;
        di += a.x * x.y - a.y * x.x;
    }
    const double2 d = block_sum2<NTA>(make_double2(dr, di), sh);
    const double2 t = cscale(d, beta);
#pragma unroll
    for (int u = 0; u < REG; ++u) {
        const int r = k + threadIdx.x + NTA * u;
        if (r < p) {
            const double2 a = vb[r];
            v[u] = make_double2(v[u].x - (t.x * a.x - t.y * a.y), v[u].y - (t.x * a.y + t.y * a.x));
            g[r] = v[u];
        }
    }
    for (int r = k + threadIdx.x + NTA * REG; r < p; r += NTA) {
        const double2 x = g[r], a = vb[r];
        g[r] = make_double2(x.x - (t.x * a.x - t.y * a.y), x.y - (t.x * a.y + t.y * a.x));
    }
    if (c != k + 1) return;
    __syncthreads();
    // reflector k + 1 from rows k+1.. of this column: shift the register window by one row
    // (entries are re-read from global memory, which this CTA has just written)
    double2 w[REG];
#pragma unroll
    for (int u = 0; u < REG; ++u) {
        const int r = c + threadIdx.x + NTA * u;
        w[u] = r < p ? g[r] : make_double2(0.0, 0.0);
    }
    qr_make(g, c, p, w, vbuf + vstride * ((k + 1) & 1), &qs->beta[(k + 1) & 1], sh);
}

// rows 0..n-1 of the n columns of W -> out (ld lo)
__global__ void urv_extract(const double2 *__restrict__ W, long long ldw, int n, double2 *__restrict__ out,
                            long long lo)
{
    const int j = blockIdx.x;
    for (int r = threadIdx.x; r < n; r += blockDim.x) out[r + lo * j] = W[r + ldw * j];
}

__global__ void urv_finish(const int8_t *__restrict__ Jw, const int *__restrict__ perm, int n,
                           int8_t *__restrict__ Js, long long *__restrict__ perm_out, int *__restrict__ permi)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        Js[j] = Jw[j];
        if (perm_out) perm_out[j] = perm[j];
        if (permi) permi[j] = perm[j];
    }
}

}  // namespace

size_t urv_workspace_bytes(long long m, long long p, int n)
{
    auto a = [](size_t b) { return (b + 255) / 256 * 256; };
    return a(16ull * m * n) + a(16ull * p * n) + a((size_t)m) + a(4ull * n) + 3 * a(8ull * n) +
           a(16ull * m) + a(32ull * p) + a(sizeof(UrvState)) + a(sizeof(QrState)) + a(4);
}

// Phase 2 into caller buffers: Fs (n x n, ldfs), Js (n), Gs (n x n, ldgs),
// perm (n, int64, may be null), permi (n, int32, may be null).
// ws: urv_workspace_bytes(m, p, n) bytes of device memory.
// Returns cudaSuccess and, after the caller's sync, *h_flags = {err, n2x2, bad J}.
cudaError_t launch_urv(int m, int p, int n, const double2 *F, long long ldf, const int8_t *J,
                       long long n_plus, const double2 *G, long long ldg, double2 *Fs, long long ldfs,
                       int8_t *Js, double2 *Gs, long long ldgs, long long *perm_out, int *permi,
                       void *ws, int *d_flags, cudaStream_t s)
{
    auto a = [](size_t b) { return (b + 255) / 256 * 256; };
    char *base = (char *)ws;
    double2 *Fw = (double2 *)base; base += a(16ull * m * n);
    double2 *Gw = (double2 *)base; base += a(16ull * p * n);
    int8_t *Jw = (int8_t *)base; base += a((size_t)m);
    int *perm = (int *)base; base += a(4ull * n);
    double *h = (double *)base; base += a(8ull * n);
    double *mag = (double *)base; base += a(8ull * n);
    double *mag2 = (double *)base; base += a(8ull * n);
    double2 *sv = (double2 *)base; base += a(16ull * m);
    double2 *vb = (double2 *)base; base += a(32ull * p);
    UrvState *st = (UrvState *)base; base += a(sizeof(UrvState));
    QrState *qs = (QrState *)base; base += a(sizeof(QrState));
    int *bad = (int *)base;
    cudaError_t e;
    if ((e = cudaMemsetAsync(bad, 0, 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpy2DAsync(Fw, 16ull * m, F, 16ull * ldf, 16ull * m, n, cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
        return e;
    urv_signs<<<(m + 255) / 256, 256, 0, s>>>(J, n_plus, m, Jw, bad);
    urv_init<<<(n + 255) / 256, 256, 0, s>>>(n, perm, st);
    const int dot_blocks = (n + 7) / 8 < 1216 ? (n + 7) / 8 : 1216;
    urv_norms<<<dot_blocks, 256, 0, s>>>(Fw, m, m, n, Jw, 0, h);
    // the hyperbolic QR: n step chains; a 2x2 pivot makes the last chains empty
    for (int it = 0; it < n; ++it) {
        const int cols = n - it - 1 > 0 ? n - it - 1 : 1;    // first trailing column >= it + 1
        const int gblocks = cols < 1216 ? cols : 1216;
        urv_select<<<1, NT1, 0, s>>>(Fw, m, m, n, perm, h, st);
        urv_dots<<<dot_blocks, 256, 0, s>>>(Fw, m, m, n, Jw, st, 1, mag);
        urv_bk1<<<1, NT1, 0, s>>>(h, mag, n, st);
        urv_dots<<<dot_blocks, 256, 0, s>>>(Fw, m, m, n, Jw, st, 2, mag2);
        urv_pivot<<<1, NT1, 0, s>>>(Fw, m, m, n, Jw, perm, h, mag2, sv, st);
        urv_apply<<<gblocks, NTA, 0, s>>>(Fw, m, m, n, Jw, sv, h, st, 1);
        urv_reflect2<<<1, NT1, 0, s>>>(Fw, m, m, n, Jw, sv, st);
        urv_apply<<<gblocks, NTA, 0, s>>>(Fw, m, m, n, Jw, sv, h, st, 2);
    }
    // the Householder QR of G~ P2
    qr_gather<<<n, 256, 0, s>>>(G, ldg, p, perm, Gw, p);
    qr_first<<<1, NTA, 0, s>>>(Gw, p, p, vb, qs);
    for (int k = 0; k + 1 < n; ++k) qr_step<<<n - k - 1, NTA, 0, s>>>(Gw, p, p, n, k, vb, p, qs);
    urv_extract<<<n, 256, 0, s>>>(Fw, m, n, Fs, ldfs);
    urv_extract<<<n, 256, 0, s>>>(Gw, p, n, Gs, ldgs);
    urv_finish<<<(n + 255) / 256, 256, 0, s>>>(Jw, perm, n, Js, perm_out, permi);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(d_flags, &st->err, 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(d_flags + 1, &st->n2x2, 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    return cudaMemcpyAsync(d_flags + 2, bad, 4, cudaMemcpyDeviceToDevice, s);
}

int urv_launches(int n) { return 3 + 8 * n + 2 + (n - 1) + 3; }

}  // namespace hz
