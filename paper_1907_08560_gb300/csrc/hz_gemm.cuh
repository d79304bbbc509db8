// hz_gemm.cuh -- the FP64 product tile of the transformations applied to the
// stacked factors (warm start, the complex64 rounds of the mixed schedule).
#pragma once
#include <cuda_runtime.h>

namespace hz {

// ----------------------------------------------------------------------------
// C = A B for a column-major A (rows x n, rows a multiple of 64) and a square
// B (n x n, complex128 or complex64 promoted to FP64), FP64 accumulation.
// One 64 x 64 output tile (rows row0.., columns col0..) computed by the 256
// threads of a CTA, 16-deep K slices staged in shared memory.
// The complex products take the three-multiplication form
//   a b = (ar br - ai bi) + i ((ar + ai)(br + bi) - ar br - ai bi)
// (three real FMA chains per output; the FP64 pipe bounds this kernel), whose
// error is bounded entrywise by a small multiple of |A||B| as the usual form's.
// ----------------------------------------------------------------------------
template <typename TB>
__device__ __forceinline__ void gemm_tile_3m(const double2 *__restrict__ A, long long lda,
                                             const TB *__restrict__ B, long long ldb,
                                             double2 *__restrict__ C, long long ldc, int n,
                                             long long row0, int col0)
{
    __shared__ double2 as[64][17];
    __shared__ double2 bs[16][64];
    __shared__ double bq[16][64];     // br + bi
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double t1[4][4], t2[4][4], t3[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { t1[i][j] = 0; t2[i][j] = 0; t3[i][j] = 0; }
    for (int k0 = 0; k0 < n; k0 += 16) {
        __syncthreads();
        for (int e = tid; e < 64 * 16; e += 256) {
            const int r = e % 64, k = e / 64;
            as[r][k] = (k0 + k < n) ? A[row0 + r + lda * (k0 + k)] : make_double2(0.0, 0.0);
        }
        for (int e = tid; e < 16 * 64; e += 256) {
            const int k = e % 16, c = e / 16;
            double2 v = make_double2(0.0, 0.0);
            if (k0 + k < n && col0 + c < n) {
                const TB b = B[(k0 + k) + ldb * (col0 + c)];
                v = make_double2((double)b.x, (double)b.y);
            }
            bs[k][c] = v;
            bq[k][c] = v.x + v.y;
        }
        __syncthreads();
#pragma unroll 2
        for (int k = 0; k < 16; ++k) {
            double2 x[4], z[4];
            double xp[4], zq[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                x[i] = as[ty + 16 * i][k];
                xp[i] = x[i].x + x[i].y;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                z[j] = bs[k][tx + 16 * j];
                zq[j] = bq[k][tx + 16 * j];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    t1[i][j] = fma(x[i].x, z[j].x, t1[i][j]);
                    t2[i][j] = fma(x[i].y, z[j].y, t2[i][j]);
                    t3[i][j] = fma(xp[i], zq[j], t3[i][j]);
                }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = col0 + tx + 16 * j;
            if (c < n)
                C[row0 + ty + 16 * i + ldc * c] =
                    make_double2(t1[i][j] - t2[i][j], (t3[i][j] - t1[i][j]) - t2[i][j]);
        }
}

}  // namespace hz
