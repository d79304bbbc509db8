// hz_ozaki.cu -- the block update of Section 6.4.3 with FP64 accuracy on the
// bf16 tensor cores (an Ozaki-type splitting of the FP64 operands).
//
// For one block pair, C = A Z^ with A = [X_P X_Q] (Mt stacked rows of F', G',
// Z' x kk complex columns) and Z^ the kk x kk accumulated transformation.  In
// real form, with the real and imaginary parts interleaved,
//   A' = [Re a_1, Im a_1, Re a_2, ...]           (Mt x 2kk),
//   Z'[2k][2j] = Re z_kj, Z'[2k][2j+1] = Im z_kj,
//   Z'[2k+1][2j] = -Im z_kj, Z'[2k+1][2j+1] = Re z_kj,
// so that C' = A' Z' holds Re c_j, Im c_j in columns 2j, 2j+1.
//
// Scaling.  Column k of A' is scaled by 2^-e_k (e_k: exponent of the largest
// entry of column k of W) and row k of Z' by 2^e_k, which leaves the product
// unchanged and makes the entries of a row of A' comparable.  Then row r of
// A' is scaled by 2^-m_r and column j of Z' by 2^-c_j so that all entries are
// below 1 in magnitude, and each entry x is cut into 8 signed 7-bit integer
// slices, x = sum_s t_s 2^-7s + (|error| < 2^-56), by integer operations on
// its binary representation (no rounding).
//
// Products.  A slice product A_i Z_j (K = 2kk <= 128) of integers below 2^7 in
// magnitude is exact in FP32 accumulation (127^2 * 128 * 8 < 2^24 even when
// the up to 8 products of one level i + j are summed), so each level
// L = i + j (2..9) is an exact integer; the levels are combined exactly in
// 64-bit integers (two halves of four levels), converted to FP64 and scaled:
//   C'_rj = 2^(m_r + c_j) (hi 2^-35 + lo 2^-63)  (one rounding).
// The dropped products (i + j > 9) and the slicing remainders are below
// 2^-56 relative to the scaled operands.
//
// Kernels: oz_colexp (e_k of every column of W), oz_zslice (Z' scaled and
// sliced into the mma B-fragment layout, per pair and half of the outputs),
// oz_update (one CTA per (pair, output half, row group): the B slices of its
// half stay in shared memory while the CTA walks over 32-row tiles of A,
// slicing each tile into shared memory and running mma.sync m16n8k16 bf16).
// The update is out of place (W -> Wout): the two output halves of a pair
// are computed by different CTAs that both read all columns of the pair.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hz_launch.h"

namespace hz {
namespace {

constexpr int OZ_S = 8;           // slices per operand
constexpr int OZ_BITS = 7;        // bits per slice
constexpr int OZ_K = 2 * KKMAX;   // real contraction length (128)
constexpr int OZ_NH = 64;         // real output columns per CTA (half of 128)
constexpr int OZ_TR = 32;         // rows per tile
constexpr int OZ_THREADS = 256;
constexpr int OZ_EMPTY = -100000; // exponent of an all-zero column

// B fragments of one (pair, half): [slice 8][kstep 8][nblock 8][lane 32] x uint2
constexpr int OZ_BFRAGS = OZ_S * 8 * 8 * 32;
// A fragments of one tile: [slice 8][mblock 2][kstep 8][lane 32] x uint4
constexpr int OZ_AFRAGS = OZ_S * 2 * 8 * 32;
constexpr size_t OZ_SMEM = (size_t)OZ_BFRAGS * 8 + (size_t)OZ_AFRAGS * 16;   // 192 KB
constexpr size_t OZ_ZSMEM = (size_t)OZ_K * (OZ_NH + 1) * 8;                   // 66.5 KB

// frexp-style exponent: |x| < 2^E (E of 0 is OZ_EMPTY); denormals as 2^-1022.
__device__ __forceinline__ int oz_exp(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int eb = (int)((b >> 52) & 0x7FF);
    if ((b << 1) == 0) return OZ_EMPTY;
    return eb == 0 ? -1021 : eb - 1022;
}

// |x| 2^(56 - T) truncated to an integer (< 2^56 when |x| < 2^T), with the sign.
__device__ __forceinline__ unsigned long long oz_fixed(double x, int T, int *neg)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    *neg = (int)(b >> 63);
    const int eb = (int)((b >> 52) & 0x7FF);
    if ((b << 1) == 0) return 0ull;
    unsigned long long M = b & 0xFFFFFFFFFFFFFull;
    int e2;
    if (eb == 0) { e2 = -1074; }          // denormal: x = M 2^-1074
    else { M |= 1ull << 52; e2 = eb - 1075; }
    // |x| 2^(56 - T) = M 2^(e2 + 56 - T)
    const int sh = e2 + 56 - T;
    if (sh >= 0) return sh >= 11 ? 0ull : M << sh;   // |x| < 2^T keeps this below 2^56
    return -sh >= 64 ? 0ull : M >> (-sh);
}

__device__ __forceinline__ uint32_t oz_bf16(int t)
{
    // integers of magnitude below 128 are exact in bf16
    const float f = (float)t;
    return (uint32_t)(__float_as_uint(f) >> 16);
}

// slice s (1..8) of a fixed-point magnitude, with the sign
__device__ __forceinline__ int oz_slice(unsigned long long X, int neg, int s)
{
    const int t = (int)((X >> (56 - OZ_BITS * s)) & 0x7F);
    return neg ? -t : t;
}

__device__ __forceinline__ void mma_bf16(float *d, uint4 a, uint2 b)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
}

// e_k = largest oz_exp over the rows of column k of W (one CTA per column)
__global__ void __launch_bounds__(256)
oz_colexp(const double2 *__restrict__ W, long long ld, int rows, int *__restrict__ colexp)
{
    __shared__ int red[8];
    const double2 *col = W + ld * blockIdx.x;
    int e = OZ_EMPTY;
    for (int r = threadIdx.x; r < rows; r += 256) {
        const double2 v = col[r];
        e = max(e, max(oz_exp(v.x), oz_exp(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = red[0];
        for (int w = 1; w < 8; ++w) m = max(m, red[w]);
        colexp[blockIdx.x] = m;
    }
}

// Z' of one pair, scaled and sliced into B fragments for output half h.
// grid (npairs, 2), 256 threads.
__global__ void __launch_bounds__(256)
oz_zslice(const double2 *__restrict__ zhat, const int *__restrict__ slotcol, int kk,
          const int *__restrict__ pair_flag, const int *__restrict__ colexp, uint2 *__restrict__ zs,
          int *__restrict__ zexp)
{
    extern __shared__ double ztd[];          // [OZ_K][OZ_NH + 1]
    __shared__ int cexp[OZ_NH];
    __shared__ int rexp[KKMAX];
    const int pair = blockIdx.x, h = blockIdx.y;
    if (!pair_flag[pair]) return;
    const double2 *Z = zhat + (long long)pair * KKMAX * KKMAX;
    const int *slot = slotcol + pair * kk;
    const int tid = threadIdx.x;
    if (tid < KKMAX) {
        int e = 0;
        if (tid < kk && slot[tid] >= 0) {
            e = colexp[slot[tid]];
            if (e == OZ_EMPTY) e = 0;
        }
        rexp[tid] = e;
    }
    __syncthreads();
    // Z'[kp][n'] for the 64 outputs n' = 64 h + c of this half, times 2^e_k
    for (int idx = tid; idx < OZ_K * OZ_NH; idx += 256) {
        const int kp = idx % OZ_K, c = idx / OZ_K;
        const int np_ = OZ_NH * h + c;
        const int k = kp >> 1, j = np_ >> 1;
        double v = 0.0;
        if (k < kk && j < kk) {
            const double2 z = Z[k + KKMAX * j];
            const int ra = kp & 1, cb = np_ & 1;
            v = ra == 0 ? (cb == 0 ? z.x : z.y) : (cb == 0 ? -z.y : z.x);
            v = ldexp(v, rexp[k]);
        }
        ztd[kp * (OZ_NH + 1) + c] = v;
    }
    __syncthreads();
    if (tid < OZ_NH) {
        int e = OZ_EMPTY;
        for (int kp = 0; kp < OZ_K; ++kp) e = max(e, oz_exp(ztd[kp * (OZ_NH + 1) + tid]));
        cexp[tid] = e == OZ_EMPTY ? 0 : e;
        zexp[pair * (2 * OZ_NH) + OZ_NH * h + tid] = cexp[tid];
    }
    __syncthreads();
    // fragments: b0 = (k = 16 ks + 2 q + {0,1}, n = 8 nb + g), b1 = k + 8
    uint2 *out = zs + (long long)(pair * 2 + h) * OZ_BFRAGS;
    for (int f = tid; f < OZ_BFRAGS; f += 256) {
        const int lane = f & 31, nb = (f >> 5) & 7, ks = (f >> 8) & 7, s = f >> 11;
        const int g = lane >> 2, q = lane & 3;
        const int c = 8 * nb + g;
        uint32_t r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int kp = 16 * ks + 2 * q + (u & 1) + 8 * (u >> 1);
            int neg;
            const unsigned long long X = oz_fixed(ztd[kp * (OZ_NH + 1) + c], cexp[c], &neg);
            r[u] = oz_bf16(oz_slice(X, neg, s + 1));
        }
        out[f] = make_uint2(r[0] | (r[1] << 16), r[2] | (r[3] << 16));
    }
}

// grid = npairs * 2 * R; block 256; dynamic shared memory OZ_SMEM.
__global__ void __launch_bounds__(OZ_THREADS, 1)
oz_update(const double2 *__restrict__ Win, double2 *__restrict__ Wout, long long ld, int Mt,
          const int *__restrict__ slotcol, int kk, const int *__restrict__ pair_flag,
          const int *__restrict__ colexp, const uint2 *__restrict__ zs, const int *__restrict__ zexp,
          int R)
{
    extern __shared__ __align__(16) unsigned char oz_smem[];
    uint2 *Bs = reinterpret_cast<uint2 *>(oz_smem);
    uint4 *As = reinterpret_cast<uint4 *>(oz_smem + (size_t)OZ_BFRAGS * 8);
    uint32_t *As32 = reinterpret_cast<uint32_t *>(As);
    __shared__ int rmax[OZ_TR];
    __shared__ int ecol[KKMAX];
    __shared__ int scol[KKMAX];
    __shared__ int cexp[OZ_NH];

    const int pair = blockIdx.x / (2 * R);
    const int h = (blockIdx.x / R) & 1;
    const int rg = blockIdx.x % R;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int *slot = slotcol + pair * kk;
    const int rows_per = Mt / R;                  // a multiple of OZ_TR
    const int r_begin = rg * rows_per, r_end = r_begin + rows_per;
    if (tid < KKMAX) {
        const int sc = tid < kk ? slot[tid] : -1;
        scol[tid] = sc;
        int e = 0;
        if (sc >= 0) {
            e = colexp[sc];
            if (e == OZ_EMPTY) e = 0;
        }
        ecol[tid] = e;
    }
    if (!pair_flag[pair]) {
        // no transformation in this pair: copy this half of its columns
        __syncthreads();
        for (int c = 0; c < OZ_NH / 2; ++c) {
            const int j = (OZ_NH / 2) * h + c;
            const int sc = scol[j];
            if (sc < 0) continue;
            for (int r = r_begin + tid; r < r_end; r += OZ_THREADS) Wout[r + ld * sc] = Win[r + ld * sc];
        }
        return;
    }
    if (tid < OZ_NH) cexp[tid] = zexp[pair * (2 * OZ_NH) + OZ_NH * h + tid];
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(zs + (long long)(pair * 2 + h) * OZ_BFRAGS);
        uint4 *dst = reinterpret_cast<uint4 *>(Bs);
        for (int f = tid; f < OZ_BFRAGS / 2; f += OZ_THREADS) dst[f] = src[f];
    }
    __syncthreads();

    const int mb = warp & 1;                      // 16-row block of the tile
    const int nbp = warp >> 1;                    // 16-column block (n-blocks 2 nbp, 2 nbp + 1)
    const int g = lane >> 2, q = lane & 3;

    for (int r0 = r_begin; r0 < r_end; r0 += OZ_TR) {
        // ---- load the tile: thread = (row r0 + (tid & 31), columns (tid >> 5) + 8 u)
        const int tr = tid & 31;
        double2 a[8];
        int my = OZ_EMPTY;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = (tid >> 5) + 8 * u;
            const int sc = scol[k];
            a[u] = sc >= 0 ? Win[(r0 + tr) + ld * sc] : make_double2(0.0, 0.0);
            const int e = max(oz_exp(a[u].x), oz_exp(a[u].y));
            if (e != OZ_EMPTY) my = max(my, e - ecol[k]);
        }
        if (tid < OZ_TR) rmax[tid] = OZ_EMPTY;
        __syncthreads();
        atomicMax(&rmax[tr], my);
        __syncthreads();
        const int mr = rmax[tr] == OZ_EMPTY ? 0 : rmax[tr];
        // ---- slice into A fragments: element (row rr of m-block, k' = 2k + {re, im})
        // a0: rows 0-7, k 0-7; a1: rows 8-15, k 0-7; a2: rows 0-7, k 8-15; a3: rows 8-15, k 8-15
        {
            const int mbk = tr >> 4, rr = tr & 15;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = (tid >> 5) + 8 * u;
                const int kp = 2 * k;                       // re at kp, im at kp + 1
                const int ks = kp >> 4, kc = kp & 15;
                const int ln = (rr & 7) * 4 + ((kc & 7) >> 1);
                const int reg = (rr >> 3) + 2 * (kc >> 3);
                const int T = mr + ecol[k];
                int nre, nim;
                const unsigned long long Xr = oz_fixed(a[u].x, T, &nre);
                const unsigned long long Xi = oz_fixed(a[u].y, T, &nim);
#pragma unroll
                for (int s = 0; s < OZ_S; ++s) {
                    const uint32_t w = oz_bf16(oz_slice(Xr, nre, s + 1)) |
                                       (oz_bf16(oz_slice(Xi, nim, s + 1)) << 16);
                    As32[(((s * 2 + mbk) * 8 + ks) * 32 + ln) * 4 + reg] = w;
                }
            }
        }
        __syncthreads();
        // ---- products: levels L = i + j (slices i, j = 1..8, L <= 9)
        float acc[8][2][4];
#pragma unroll
        for (int L = 0; L < 8; ++L)
#pragma unroll
            for (int nb = 0; nb < 2; ++nb)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[L][nb][c] = 0.f;
#pragma unroll 1
        for (int ks = 0; ks < 8; ++ks) {
            uint4 af[OZ_S];
            uint2 bf[OZ_S][2];
#pragma unroll
            for (int s = 0; s < OZ_S; ++s) {
                af[s] = As[((s * 2 + mb) * 8 + ks) * 32 + lane];
#pragma unroll
                for (int nb = 0; nb < 2; ++nb) bf[s][nb] = Bs[((s * 8 + ks) * 8 + 2 * nbp + nb) * 32 + lane];
            }
#pragma unroll
            for (int i = 0; i < OZ_S; ++i)
#pragma unroll
                for (int j = 0; j < OZ_S - i; ++j)
#pragma unroll
                    for (int nb = 0; nb < 2; ++nb) mma_bf16(acc[i + j][nb], af[i], bf[j][nb]);
        }
        // ---- exact combination and FP64 output
#pragma unroll
        for (int nb = 0; nb < 2; ++nb) {
            const int cl = 16 * nbp + 8 * nb + 2 * q;      // real output columns cl (re), cl + 1 (im)
            const int j = (OZ_NH / 2) * h + (cl >> 1);     // complex column of the pair
            const int sc = scol[j];
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) {               // rows g and g + 8
                const int rr = 16 * mb + g + 8 * hr;
                const int T = rmax[rr] == OZ_EMPTY ? 0 : rmax[rr];
                double out[2];
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                    const int ci = 2 * hr + part;
                    long long hi = 0, lo = 0;
#pragma unroll
                    for (int L = 0; L < 4; ++L) hi += (long long)__float2ll_rz(acc[L][nb][ci]) << (OZ_BITS * (3 - L));
#pragma unroll
                    for (int L = 4; L < 8; ++L) lo += (long long)__float2ll_rz(acc[L][nb][ci]) << (OZ_BITS * (7 - L));
                    // value = 2^(T + c) (hi 2^-35 + lo 2^-63) = 2^(T + c - 63) (hi 2^28 + lo)
                    const double v = __fma_rn((double)hi, 268435456.0, (double)lo);
                    out[part] = ldexp(v, T + cexp[cl + part] - 63);
                }
                if (sc >= 0) Wout[(r0 + rr) + ld * sc] = make_double2(out[0], out[1]);
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t oz_workspace_bytes(int n, int npairs)
{
    auto a = [](size_t b) { return (b + 255) / 256 * 256; };
    return a(4ull * n) + a((size_t)npairs * 2 * OZ_BFRAGS * 8) + a(4ull * npairs * 2 * OZ_NH);
}

cudaError_t setup_ozaki()
{
    cudaError_t e = cudaFuncSetAttribute(oz_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(oz_zslice, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_ZSMEM);
    return e;
}

int oz_row_groups(long long Mt, int npairs, int sms)
{
    int R = sms / (2 * (npairs > 0 ? npairs : 1));
    if (R < 1) R = 1;
    while (R > 1 && (Mt % ((long long)R * OZ_TR) != 0)) --R;
    return R;
}

// W (in) -> Wout for the pairs of one step; ws: oz_workspace_bytes(n, npairs)
cudaError_t launch_oz_update(const double2 *W, double2 *Wout, const StepArgs &a, int n, const double2 *zhat,
                             const int *pair_flag, void *ws, int R, cudaStream_t s)
{
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    char *base = (char *)ws;
    int *colexp = (int *)base; base += al(4ull * n);
    uint2 *zs = (uint2 *)base; base += al((size_t)a.npairs * 2 * OZ_BFRAGS * 8);
    int *zexp = (int *)base;
    const long long Mt = (long long)a.m_pad + a.p_pad + a.n_pad;
    oz_colexp<<<n, 256, 0, s>>>(W, a.ld, (int)Mt, colexp);
    oz_zslice<<<dim3(a.npairs, 2), 256, OZ_ZSMEM, s>>>(zhat, a.slotcol, a.kk, pair_flag, colexp, zs, zexp);
    oz_update<<<a.npairs * 2 * R, OZ_THREADS, OZ_SMEM, s>>>(W, Wout, a.ld, (int)Mt, a.slotcol, a.kk, pair_flag,
                                                          colexp, zs, zexp, R);
    return cudaGetLastError();
}

}  // namespace hz
