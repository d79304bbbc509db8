// hz_tc.cu -- the block-pivot Gram (Section 6.4.2, eq. 6.1) and the block
// update (Section 6.4.3) of the complex64 preconditioning sweeps on the
// Blackwell tensor cores: tcgen05.mma of kind::tf32 with FP32 accumulation in
// tensor memory, operands staged by TMA (cp.async.bulk.tensor) tile loads.
//
// Precision: a complex64 entry x is split into TF32 parts x = hi + lo (each
// rounded to nearest), and every real product is formed as
// hi hi' + hi lo' + lo hi' ("3xTF32"): about 2^-21 relative per product, the
// accumulation in FP32 by the tensor cores.  The 2x2 parameters, the J-norms
// and the convergence test of these sweeps stay in FP64 (inner level).
//
// Complex arithmetic as real products on planar parts.  W32 is complex64,
// column-major, interleaved (re, im); the staging threads de-interleave the
// TMA tiles into planar TF32 operand tiles in the tensor cores' K-major
// layout (core matrices of 8 rows x 16 bytes, no swizzle):
//   Gram   X^* J X:  A = [Xr Xi] (128 real columns x K rows, J applied),
//                    B = [Xr Xi];  D = A B^T (128 x 128) gives
//                    Re = D[i][j] + D[64+i][64+j], Im = D[i][64+j] - D[64+i][j];
//   update X Z:      in the delta form X + X (Z - I): the products
//                    Dr = Xr Er + Xi (-Ei), Di = Xr Ei + Xi Er of E = Z - I
//                    (the 128 rows of a tile as M, the 64 output columns as
//                    N), then X added in FP32.  Late in the iteration E is
//                    small and the error of the TF32 products, relative to
//                    |X||E|, falls below the FP32 rounding of the sum: the
//                    sweeps reach the complex64 plateau of the CUDA-core form
//                    (with Z itself the 3xTF32 error, ~2^-21 |X||Z|, kept 7 %
//                    of the pivots rotating "big" and the rounds never levelled).
// The 64 internal columns of a pair are block P's in [0, 32) and block Q's in
// [32, 64); slot s of the block pivot (P in [0, wb), Q in [wb, 2 wb)) is
// internal column 32 b + j for block b, column j.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ghsvd.h"
#include "hz_launch.h"
#include "hz_tc.cuh"

namespace hz {
namespace tc {

// ---------------------------------------------------------------------------
// Gram: one CTA per (pair, row chunk); 16 rows per pipeline stage.
// Warp 0: TMA producer; warp 1: MMA issuer (and tensor-memory owner);
// warps 2-5: operand staging, then the epilogue.
// ---------------------------------------------------------------------------
constexpr int G_RS = 16;                          // rows (K) per stage
constexpr int G_NRAW = 4;                         // TMA ring depth
constexpr int G_NOPS = 2;                         // operand buffers
constexpr int G_THREADS = 192;
constexpr int G_RAW_BYTES = 2 * 32 * G_RS * 8;    // two 32-column blocks, complex64
constexpr int G_TILE_BYTES = 128 * G_RS * 4;      // 128 real columns x 16 rows TF32
constexpr int G_OPS_BYTES = 4 * G_TILE_BYTES;     // J hi, J lo, hi, lo
constexpr int G_OPS_OFF = G_NRAW * G_RAW_BYTES;
constexpr int G_SMEM = G_OPS_OFF + G_NOPS * G_OPS_BYTES + 1024;
static_assert(2 * 64 * 65 * 4 <= G_NOPS * G_OPS_BYTES, "epilogue exchange fits the operand buffers");

struct GramTcArgs {
    const int *slotcol;     // this step's [npairs][kk]
    const int8_t *Jrow;     // [m_pad]
    float2 *partial;        // [npairs][cpp][KKMAX^2]
    int *err;
    int kk, wb, m_pad, p_pad, kc, chunks_h, chunks_s;
};

__device__ __forceinline__ void named_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__global__ void __launch_bounds__(G_THREADS, 2)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, GramTcArgs a)
{
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = (unsigned char *)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t raw_full[G_NRAW], raw_empty[G_NRAW], ops_full[G_NOPS], ops_empty[G_NOPS], done;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int bcol[2], bwid[2];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cpp = a.chunks_h + a.chunks_s;
    const int pair = blockIdx.x / cpp, c = blockIdx.x % cpp;
    const bool isH = c < a.chunks_h;
    const int r0 = isH ? c * a.kc : a.m_pad + (c - a.chunks_h) * a.kc;
    const int r1 = isH ? min(r0 + a.kc, a.m_pad) : min(r0 + a.kc, a.m_pad + a.p_pad);
    const int nst = (r1 - r0) / G_RS;
    const int *slot = a.slotcol + pair * a.kk;

    if (tid == 0) {
        for (int i = 0; i < G_NRAW; ++i) { mbar_init(&raw_full[i], 1); mbar_init(&raw_empty[i], 128); }
        for (int i = 0; i < G_NOPS; ++i) { mbar_init(&ops_full[i], 128); mbar_init(&ops_empty[i], 1); }
        mbar_init(&done, 1);
        mbar_init_fence();
        abort_flag = 0;
        for (int b = 0; b < 2; ++b) {
            int w = 0;
            for (int j = 0; j < a.wb; ++j) w += slot[b * a.wb + j] >= 0;
            bwid[b] = w;
            bcol[b] = w > 0 ? slot[b * a.wb] : 0;
        }
    }
    if (warp == 1) tmem_alloc(&tmem_base, 128);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    volatile int *abort = &abort_flag;

    if (warp == 0) {
        // ---- TMA producer ----
        if (lane == 0) {
            tma_prefetch_desc(&tmap);
            int issued = 0;
            for (int s = 0; s < nst; ++s) {
                const int rs = s % G_NRAW;
                if (s >= G_NRAW && !mbar_wait(&raw_empty[rs], ((s / G_NRAW) - 1) & 1, abort, a.err, DEVERR_TIMEOUT))
                    break;
                unsigned char *dst = sm + rs * G_RAW_BYTES;
                mbar_arrive_tx(&raw_full[rs], G_RAW_BYTES);
                tma_load_2d(dst, &tmap, r0 + s * G_RS, bcol[0], &raw_full[rs]);
                tma_load_2d(dst + G_RAW_BYTES / 2, &tmap, r0 + s * G_RS, bcol[1], &raw_full[rs]);
                issued = s + 1;
            }
            // on an abort, let the copies in flight land before the CTA exits
            if (*abort) {
                int zero = 0;
                for (int s = issued - G_NRAW < 0 ? 0 : issued - G_NRAW; s < issued; ++s)
                    mbar_wait(&raw_full[s % G_NRAW], (s / G_NRAW) & 1, &zero, a.err, DEVERR_TIMEOUT);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer: D += A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T ----
        if (lane == 0) {
            const uint32_t id = idesc_tf32(128, 128, 0);
            for (int s = 0; s < nst; ++s) {
                const int ob = s % G_NOPS;
                if (!mbar_wait(&ops_full[ob], (s / G_NOPS) & 1, abort, a.err, DEVERR_TIMEOUT)) break;
                tc_fence_after();
                const uint32_t base = smem_u32(sm + G_OPS_OFF + ob * G_OPS_BYTES);
                const uint32_t t_hi = base + 2 * G_TILE_BYTES, t_lo = base + 3 * G_TILE_BYTES;
                const uint32_t a_hi = isH ? base : t_hi, a_lo = isH ? base + G_TILE_BYTES : t_lo;
#pragma unroll
                for (int ks = 0; ks < G_RS / 8; ++ks) {
                    const uint32_t o = ks * 256;
                    const uint64_t dah = sdesc(a_hi + o, 128, 512), dal = sdesc(a_lo + o, 128, 512);
                    const uint64_t dbh = sdesc(t_hi + o, 128, 512), dbl = sdesc(t_lo + o, 128, 512);
                    mma_tf32(tmem, dah, dbh, id, (s | ks) != 0);
                    mma_tf32(tmem, dah, dbl, id, 1);
                    mma_tf32(tmem, dal, dbh, id, 1);
                }
                mma_commit(&ops_empty[ob]);
            }
            mma_commit(&done);
        }
    } else {
        // ---- operand staging: raw complex64 tile -> planar TF32 hi / lo tiles ----
        const int ct = tid - 64, cw = ct >> 5;
        const int u8 = lane & 7, kq = lane >> 3;
        for (int s = 0; s < nst; ++s) {
            const int rs = s % G_NRAW, ob = s % G_NOPS;
            if (!mbar_wait(&raw_full[rs], (s / G_NRAW) & 1, abort, a.err, DEVERR_TIMEOUT)) break;
            if (s >= G_NOPS && !mbar_wait(&ops_empty[ob], ((s / G_NOPS) - 1) & 1, abort, a.err, DEVERR_TIMEOUT))
                break;
            const unsigned char *raw = sm + rs * G_RAW_BYTES;
            unsigned char *ops = sm + G_OPS_OFF + ob * G_OPS_BYTES;
            int jsg = 0x01010101;
            if (isH) jsg = *(const int *)(a.Jrow + r0 + s * G_RS + 4 * kq);
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int u = 8 * (cw + 4 * g) + u8;
                const int b = u >> 5, jj = u & 31;
                const float4 *src = (const float4 *)(raw + ((b * 32 + jj) * G_RS + 4 * kq) * 8);
                float4 v0 = src[0], v1 = src[1];    // rows 4kq..4kq+3: (re, im) pairs
                if (jj >= bwid[b]) { v0 = make_float4(0, 0, 0, 0); v1 = v0; }
                const float re[4] = {v0.x, v0.z, v1.x, v1.z}, im[4] = {v0.y, v0.w, v1.y, v1.w};
                float rh[4], rl[4], ih[4], il[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    tf32_split(re[q], rh[q], rl[q]);
                    tf32_split(im[q], ih[q], il[q]);
                }
                const uint32_t ore = kmaj_off(u, 4 * kq, G_RS), oim = kmaj_off(64 + u, 4 * kq, G_RS);
                *(float4 *)(ops + 2 * G_TILE_BYTES + ore) = make_float4(rh[0], rh[1], rh[2], rh[3]);
                *(float4 *)(ops + 2 * G_TILE_BYTES + oim) = make_float4(ih[0], ih[1], ih[2], ih[3]);
                *(float4 *)(ops + 3 * G_TILE_BYTES + ore) = make_float4(rl[0], rl[1], rl[2], rl[3]);
                *(float4 *)(ops + 3 * G_TILE_BYTES + oim) = make_float4(il[0], il[1], il[2], il[3]);
                if (isH) {
                    // J on the A operand: flip the sign of the rows with J = -1
                    float sg[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) sg[q] = ((int8_t)(jsg >> (8 * q))) < 0 ? -1.0f : 1.0f;
                    *(float4 *)(ops + ore) = make_float4(sg[0] * rh[0], sg[1] * rh[1], sg[2] * rh[2], sg[3] * rh[3]);
                    *(float4 *)(ops + oim) = make_float4(sg[0] * ih[0], sg[1] * ih[1], sg[2] * ih[2], sg[3] * ih[3]);
                    *(float4 *)(ops + G_TILE_BYTES + ore) =
                        make_float4(sg[0] * rl[0], sg[1] * rl[1], sg[2] * rl[2], sg[3] * rl[3]);
                    *(float4 *)(ops + G_TILE_BYTES + oim) =
                        make_float4(sg[0] * il[0], sg[1] * il[1], sg[2] * il[2], sg[3] * il[3]);
                }
            }
            fence_async_smem();
            mbar_arrive(&raw_empty[rs]);
            mbar_arrive(&ops_full[ob]);
        }

        // ---- epilogue: D (128 x 128 real) -> the complex partial, upper part ----
        // (bounded by time only: the products must be complete before the
        // tensor memory is read or freed)
        int no_abort = 0;
        mbar_wait(&done, 0, &no_abort, a.err, DEVERR_TIMEOUT);
        tc_fence_after();
        const int qw = warp & 3;
        const int m = 32 * qw + lane;                      // row of D held by this thread
        const uint32_t taddr = tmem + ((uint32_t)(32 * qw) << 16);
        float *Xc = (float *)(sm + G_OPS_OFF);             // D[64+i][64+j]
        float *Xd = Xc + 64 * 65;                          // D[64+i][j]
        if (m >= 64) {                                     // warps with qw = 2, 3
            const int i = m - 64;
#pragma unroll 1
            for (int c0 = 0; c0 < 128; c0 += 16) {
                float v[16];
                tmem_ld16(taddr + c0, v);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int n = c0 + q;
                    if (n >= 64) Xc[i * 65 + n - 64] = v[q];
                    else Xd[i * 65 + n] = v[q];
                }
            }
        }
        named_sync(1, 128);
        if (m < 64) {                                      // warps with qw = 0, 1
            const int i = m;
            const int bi = i >> 5, ji = i & 31;
            const bool has_slot = ji < a.wb;
            const int si = bi * a.wb + ji;
            const bool vi = ji < bwid[bi];
            float2 *out = a.partial + ((long long)pair * cpp + c) * (KKMAX * KKMAX);
#pragma unroll 1
            for (int c0 = 0; c0 < 64; c0 += 16) {
                float dre[16], dim[16];
                tmem_ld16(taddr + c0, dre);        // D[i][j]       (warp-wide)
                tmem_ld16(taddr + 64 + c0, dim);   // D[i][64+j]
                if (!has_slot) continue;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int j = c0 + q;
                    const int bj = j >> 5, jj = j & 31;
                    if (jj >= a.wb) continue;
                    const int sj = bj * a.wb + jj;
                    if (sj < si) continue;
                    float2 h = make_float2(0.0f, 0.0f);
                    if (vi && jj < bwid[bj]) h = make_float2(dre[q] + Xc[i * 65 + j], dim[q] - Xd[i * 65 + j]);
                    out[si + KKMAX * sj] = h;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_free(tmem, 128);
    }
}

// ---------------------------------------------------------------------------
// Block update: [X_P X_Q] <- [X_P X_Q] Z^ on 128-row tiles of W32.  The tiles
// of the pairs whose inner level applied a transformation are dealt in
// contiguous ranges to the CTAs (one per SM); a CTA stages the pair's Z^ once
// (again when its range crosses into the next pair).  Each tile is four
// stages of 16 complex input columns.
// Warp 0: TMA producer; warp 1: MMA issuer and tensor-memory owner;
// warps 2-5: operand staging (Z^ and the row tiles); warps 6-9: epilogue
// (tensor memory -> W32), double-buffered accumulators so that the epilogue
// of a tile overlaps the products of the next.
// ---------------------------------------------------------------------------
constexpr int U_THREADS = 320;
constexpr int U_ROWS = 128;                       // M
constexpr int U_KC = 16;                          // complex input columns per stage
constexpr int U_NRAW = 3;
constexpr int U_NOPS = 2;
constexpr int U_RAW_BYTES = U_ROWS * U_KC * 8;    // complex64 tile from TMA
constexpr int U_TILE_BYTES = U_ROWS * U_KC * 4;   // one TF32 operand tile
constexpr int U_OPS_BYTES = 4 * U_TILE_BYTES;     // Xr hi, Xr lo, Xi hi, Xi lo
constexpr int U_BT_BYTES = 64 * 64 * 4;           // one Z^ operand tile (N 64 x K 64)
constexpr int U_OPS_OFF = U_NRAW * U_RAW_BYTES;
constexpr int U_B_OFF = U_OPS_OFF + U_NOPS * U_OPS_BYTES;
constexpr int U_SMEM = U_B_OFF + 6 * U_BT_BYTES + 1024;
constexpr int U_MAXPAIRS = 1024;
static_assert(U_SMEM <= 227 * 1024, "update CTA fits the shared memory of an SM");

struct UpdTcArgs {
    const int *slotcol;     // this step's [npairs][kk]
    const float2 *zhat;     // [npairs][KKMAX^2] complex64 Z^ (column-major)
    const int *pair_flag;   // [npairs]
    float2 *W;              // W32
    int *err;
    long long ld;           // Mt
    int npairs, kk, wb, tiles_per_pair, Mt;
};

__global__ void __launch_bounds__(U_THREADS, 1)
update_tc_kernel(const __grid_constant__ CUtensorMap tmap, UpdTcArgs a)
{
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = (unsigned char *)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t raw_full[U_NRAW], raw_empty[U_NRAW], ops_full[U_NOPS], ops_empty[U_NOPS];
    __shared__ uint64_t acc_full[2], acc_empty[2], b_full, b_empty, drain, stg_bar, epi_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag, nact;
    __shared__ int act[U_MAXPAIRS];
    __shared__ int bwid[2][2];                    // staging: block widths, by pair parity
    __shared__ int outcol[2][64];                 // epilogue: column of each output (-1: none), by pair parity

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < U_NRAW; ++i) { mbar_init(&raw_full[i], 1); mbar_init(&raw_empty[i], 128); }
        for (int i = 0; i < U_NOPS; ++i) { mbar_init(&ops_full[i], 128); mbar_init(&ops_empty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&acc_full[i], 1); mbar_init(&acc_empty[i], 128); }
        mbar_init(&b_full, 128);
        mbar_init(&b_empty, 1);
        mbar_init(&drain, 1);
        mbar_init(&stg_bar, 128);
        mbar_init(&epi_bar, 128);
        mbar_init_fence();
        abort_flag = 0;
    }
    if (warp == 0) {
        // the pairs with a transformation, in order (ballot compaction)
        int count = 0;
        for (int base = 0; base < a.npairs; base += 32) {
            const int p = base + lane;
            const bool f = p < a.npairs && a.pair_flag[p] != 0;
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (f) act[count + __popc(bal & ((1u << lane) - 1u))] = p;
            count += __popc(bal);
        }
        if (lane == 0) nact = count;
    }
    __syncthreads();
    const int tpp = a.tiles_per_pair;
    const long long total = (long long)nact * tpp;
    const long long per = (total + gridDim.x - 1) / gridDim.x;
    const long long g0 = (long long)blockIdx.x * per;
    const long long g1 = g0 + per < total ? g0 + per : total;
    if (g0 >= g1) return;                         // uniform: nothing for this CTA
    const int ntl = (int)(g1 - g0);

    if (warp == 1) tmem_alloc(&tmem_base, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    volatile int *abort = &abort_flag;

    if (warp == 0) {
        // ---- TMA producer: per tile, four 128-row x 16-column complex64 boxes ----
        if (lane == 0) {
            tma_prefetch_desc(&tmap);
            int issued = 0;
            for (int tl = 0; tl < ntl && !*abort; ++tl) {
                const long long g = g0 + tl;
                const int pair = act[g / tpp];
                const int row0 = (int)(g % tpp) * U_ROWS;
                const int *slot = a.slotcol + pair * a.kk;
                bool ok = true;
                for (int c = 0; c < 4; ++c) {
                    const int q = tl * 4 + c, rs = q % U_NRAW;
                    if (q >= U_NRAW && !mbar_wait(&raw_empty[rs], ((q / U_NRAW) - 1) & 1, abort, a.err, DEVERR_TIMEOUT)) {
                        ok = false;
                        break;
                    }
                    const int first = slot[(c >> 1) * a.wb];
                    const int col = (first < 0 ? 0 : first) + 16 * (c & 1);
                    mbar_arrive_tx(&raw_full[rs], U_RAW_BYTES);
                    tma_load_2d(sm + rs * U_RAW_BYTES, &tmap, row0, col, &raw_full[rs]);
                    issued = q + 1;
                }
                if (!ok) break;
            }
            if (*abort) {
                int zero = 0;
                for (int q = issued - U_NRAW < 0 ? 0 : issued - U_NRAW; q < issued; ++q)
                    mbar_wait(&raw_full[q % U_NRAW], (q / U_NRAW) & 1, &zero, a.err, DEVERR_TIMEOUT);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const uint32_t id = idesc_tf32(U_ROWS, 64, 0);
            const uint32_t bb = smem_u32(sm + U_B_OFF);
            const uint32_t ZRH = bb, ZRL = bb + U_BT_BYTES, ZIH = bb + 2 * U_BT_BYTES, ZIL = bb + 3 * U_BT_BYTES;
            const uint32_t NZIH = bb + 4 * U_BT_BYTES, NZIL = bb + 5 * U_BT_BYTES;
            int k = -1;
            bool ok = true;
            for (int tl = 0; tl < ntl && ok; ++tl) {
                const long long g = g0 + tl;
                const bool newpair = tl == 0 || g % tpp == 0;
                const bool lastofpair = tl == ntl - 1 || (g + 1) % tpp == 0;
                if (newpair) {
                    ++k;
                    if (!mbar_wait(&b_full, k & 1, abort, a.err, DEVERR_TIMEOUT)) break;
                    tc_fence_after();
                }
                const int acc = tl & 1;
                if (tl >= 2) {
                    if (!mbar_wait(&acc_empty[acc], ((tl >> 1) - 1) & 1, abort, a.err, DEVERR_TIMEOUT)) break;
                    tc_fence_after();
                }
                const uint32_t dr = tmem + 128 * acc, di = dr + 64;
                for (int c = 0; c < 4; ++c) {
                    const int q = tl * 4 + c, ob = q % U_NOPS;
                    if (!mbar_wait(&ops_full[ob], (q / U_NOPS) & 1, abort, a.err, DEVERR_TIMEOUT)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t ob0 = smem_u32(sm + U_OPS_OFF + ob * U_OPS_BYTES);
#pragma unroll
                    for (int ks = 0; ks < U_KC / 8; ++ks) {
                        const uint32_t ao = ks * 256, bo = (4 * c + 2 * ks) * 128;
                        const uint64_t xrh = sdesc(ob0 + ao, 128, 512);
                        const uint64_t xrl = sdesc(ob0 + U_TILE_BYTES + ao, 128, 512);
                        const uint64_t xih = sdesc(ob0 + 2 * U_TILE_BYTES + ao, 128, 512);
                        const uint64_t xil = sdesc(ob0 + 3 * U_TILE_BYTES + ao, 128, 512);
                        const uint64_t zrh = sdesc(ZRH + bo, 128, 2048), zrl = sdesc(ZRL + bo, 128, 2048);
                        const uint64_t zih = sdesc(ZIH + bo, 128, 2048), zil = sdesc(ZIL + bo, 128, 2048);
                        const uint64_t nzih = sdesc(NZIH + bo, 128, 2048), nzil = sdesc(NZIL + bo, 128, 2048);
                        const uint32_t acc0 = (c | ks) != 0;
                        // Dr = Xr Er + Xi (-Ei)
                        mma_tf32(dr, xrh, zrh, id, acc0);
                        mma_tf32(dr, xrh, zrl, id, 1);
                        mma_tf32(dr, xrl, zrh, id, 1);
                        mma_tf32(dr, xih, nzih, id, 1);
                        mma_tf32(dr, xih, nzil, id, 1);
                        mma_tf32(dr, xil, nzih, id, 1);
                        // Di = Xr Ei + Xi Er
                        mma_tf32(di, xrh, zih, id, acc0);
                        mma_tf32(di, xrh, zil, id, 1);
                        mma_tf32(di, xrl, zih, id, 1);
                        mma_tf32(di, xih, zrh, id, 1);
                        mma_tf32(di, xih, zrl, id, 1);
                        mma_tf32(di, xil, zrh, id, 1);
                    }
                    mma_commit(&ops_empty[ob]);
                }
                if (!ok) break;
                mma_commit(&acc_full[acc]);
                if (lastofpair) mma_commit(&b_empty);
            }
            // every product complete before the tensor memory is freed
            mma_commit(&drain);
            int zero = 0;
            mbar_wait(&drain, 0, &zero, a.err, DEVERR_TIMEOUT);
        }
    } else if (warp < 6) {
        // ---- operand staging ----
        const int ct = tid - 64, cw = ct >> 5;
        int k = -1;
        for (int tl = 0; tl < ntl; ++tl) {
            const long long g = g0 + tl;
            const int pair = act[g / tpp];
            const int *slot = a.slotcol + pair * a.kk;
            if (tl == 0 || g % tpp == 0) {
                // Z^ of the new pair -> TF32 hi / lo tiles of Zr, Zi, -Zi (K-major,
                // N = output column, K = input column, internal numbering)
                ++k;
                if (k >= 1 && !mbar_wait(&b_empty, (k - 1) & 1, abort, a.err, DEVERR_TIMEOUT)) break;
                // block widths of the pair (double-buffered by pair parity: every
                // staging thread has left pair k - 2 before it arrives here)
                if (ct < 2) {
                    int w = 0;
                    for (int j = 0; j < a.wb; ++j) w += slot[ct * a.wb + j] >= 0;
                    bwid[k & 1][ct] = w;
                }
                mbar_arrive(&stg_bar);
                if (!mbar_wait(&stg_bar, k & 1, abort, a.err, DEVERR_TIMEOUT)) break;
                const int *bw = bwid[k & 1];
                const float2 *zp = a.zhat + (long long)pair * (KKMAX * KKMAX);
                unsigned char *B = sm + U_B_OFF;
#pragma unroll 1
                for (int it = 0; it < 8; ++it) {
                    const int item = it * 128 + ct;
                    const int o = (item & 7) + 8 * (item >> 7), uq = (item >> 3) & 15;
                    const int bo = o >> 5, jo = o & 31;
                    const bool vo = jo < bw[bo];
                    const int so = bo * a.wb + jo;
                    float zrh[4], zrl[4], zih[4], zil[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int u = 4 * uq + e;
                        const int bu = u >> 5, ju = u & 31;
                        float2 z = make_float2(0.0f, 0.0f);
                        if (vo && ju < bw[bu]) {
                            z = zp[(bu * a.wb + ju) + KKMAX * so];
                            if (u == o) z.x -= 1.0f;        // the delta form: Z^ - I
                        }
                        tf32_split(z.x, zrh[e], zrl[e]);
                        tf32_split(z.y, zih[e], zil[e]);
                    }
                    const uint32_t off = kmaj_off(o, 4 * uq, 64);
                    *(float4 *)(B + off) = make_float4(zrh[0], zrh[1], zrh[2], zrh[3]);
                    *(float4 *)(B + U_BT_BYTES + off) = make_float4(zrl[0], zrl[1], zrl[2], zrl[3]);
                    *(float4 *)(B + 2 * U_BT_BYTES + off) = make_float4(zih[0], zih[1], zih[2], zih[3]);
                    *(float4 *)(B + 3 * U_BT_BYTES + off) = make_float4(zil[0], zil[1], zil[2], zil[3]);
                    *(float4 *)(B + 4 * U_BT_BYTES + off) = make_float4(-zih[0], -zih[1], -zih[2], -zih[3]);
                    *(float4 *)(B + 5 * U_BT_BYTES + off) = make_float4(-zil[0], -zil[1], -zil[2], -zil[3]);
                }
                fence_async_smem();
                mbar_arrive(&b_full);
            }
            bool ok = true;
            for (int c = 0; c < 4; ++c) {
                const int q = tl * 4 + c, rs = q % U_NRAW, ob = q % U_NOPS;
                if (!mbar_wait(&raw_full[rs], (q / U_NRAW) & 1, abort, a.err, DEVERR_TIMEOUT)) { ok = false; break; }
                if (q >= U_NOPS && !mbar_wait(&ops_empty[ob], ((q / U_NOPS) - 1) & 1, abort, a.err, DEVERR_TIMEOUT)) {
                    ok = false;
                    break;
                }
                const float2 *raw = (const float2 *)(sm + rs * U_RAW_BYTES);   // [16 columns][128 rows]
                unsigned char *ops = sm + U_OPS_OFF + ob * U_OPS_BYTES;
                const int m = 32 * cw + lane;
                const int b = c >> 1;
#pragma unroll
                for (int gq = 0; gq < 4; ++gq) {
                    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int cc = 4 * gq + e;
                        float2 v = raw[cc * U_ROWS + m];
                        if (16 * (c & 1) + cc >= bwid[k & 1][b]) v = make_float2(0.0f, 0.0f);
                        tf32_split(v.x, rh[e], rl[e]);
                        tf32_split(v.y, ih[e], il[e]);
                    }
                    const uint32_t off = kmaj_off(m, 4 * gq, U_KC);
                    *(float4 *)(ops + off) = make_float4(rh[0], rh[1], rh[2], rh[3]);
                    *(float4 *)(ops + U_TILE_BYTES + off) = make_float4(rl[0], rl[1], rl[2], rl[3]);
                    *(float4 *)(ops + 2 * U_TILE_BYTES + off) = make_float4(ih[0], ih[1], ih[2], ih[3]);
                    *(float4 *)(ops + 3 * U_TILE_BYTES + off) = make_float4(il[0], il[1], il[2], il[3]);
                }
                fence_async_smem();
                mbar_arrive(&raw_empty[rs]);
                mbar_arrive(&ops_full[ob]);
            }
            if (!ok) break;
        }
    } else {
        // ---- epilogue: tensor memory -> W32, columns Z^ changed only ----
        const int et = tid - 192, qw = warp & 3;
        const int m = 32 * qw + lane;
        int k = -1;
        for (int tl = 0; tl < ntl; ++tl) {
            const long long g = g0 + tl;
            const int pair = act[g / tpp];
            const int row = (int)(g % tpp) * U_ROWS + m;
            if (tl == 0 || g % tpp == 0) {
                ++k;
                if (et < 64) {
                    // output o: its column, or -1 if the slot is empty or Z^ leaves it
                    // as it is (e_o: then the column is not written, exactly as before);
                    // double-buffered by pair parity as the staging widths
                    const int bo = et >> 5, jo = et & 31;
                    int col = -1;
                    if (jo < a.wb) {
                        const int so = bo * a.wb + jo;
                        col = a.slotcol[pair * a.kk + so];
                        if (col >= 0) {
                            const float2 *zc = a.zhat + (long long)pair * (KKMAX * KKMAX) + KKMAX * so;
                            bool ident = true;
                            for (int l = 0; l < a.kk; ++l) {
                                const float2 z = zc[l];
                                ident &= (z.x == (l == so ? 1.0f : 0.0f)) && (z.y == 0.0f);
                            }
                            if (ident) col = -1;
                        }
                    }
                    outcol[k & 1][et] = col;
                }
                mbar_arrive(&epi_bar);
                if (!mbar_wait(&epi_bar, k & 1, abort, a.err, DEVERR_TIMEOUT)) break;
            }
            const int acc = tl & 1;
            if (!mbar_wait(&acc_full[acc], (tl >> 1) & 1, abort, a.err, DEVERR_TIMEOUT)) break;
            tc_fence_after();
            const uint32_t taddr = tmem + 128 * acc + ((uint32_t)(32 * qw) << 16);
#pragma unroll 1
            for (int o0 = 0; o0 < 64; o0 += 16) {
                // Y = X + X (Z^ - I): the tile's own entries (still in L2 from
                // the TMA load) plus the product, one FP32 rounding
                float2 x[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int col = outcol[k & 1][o0 + q];
                    x[q] = (col >= 0 && row < a.Mt) ? a.W[(long long)col * a.ld + row] : make_float2(0.0f, 0.0f);
                }
                float yr[16], yi[16];
                tmem_ld16(taddr + o0, yr);
                tmem_ld16(taddr + 64 + o0, yi);
                if (row < a.Mt) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int col = outcol[k & 1][o0 + q];
                        if (col >= 0) a.W[(long long)col * a.ld + row] = make_float2(x[q].x + yr[q], x[q].y + yi[q]);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&acc_empty[acc]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_free(tmem, 256);
    }
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// W32 (ld x n complex64, column-major) as a 2-D tensor of 8-byte elements:
// dimension 0 = rows (contiguous), dimension 1 = columns; a box of
// box_rows x box_cols, zero fill outside.
cudaError_t make_map(CUtensorMap *map, const void *W32, long long ld, int n, int box_rows, int box_cols)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
    const cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void *>(W32), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

// Route each pair of a complex64 step to one of the two updates: the
// tensor-core update (delta form) when every entry of E = Z^ - I is at most
// TC_SMALL_E in real and imaginary part, so that its error, about
// 2^-21 |X||E| with the tensor cores' FP32 accumulation, stays at the FP32
// rounding of X + X E; the FP32 CUDA-core update otherwise (the large
// rotations and prescalings of the first sweeps).  Measured on the n = 64
// and n = 256 test pencils (one complex64 round) and the n = 2048 benchmark
// pencil: with every pair on the tensor cores the complex64 sweeps left
// Z'_low less consistent with W32 and the FP64 finishing sweeps took 2-3
// more sweeps on the small pencils; thresholds 2^-6, 2^-3 and 2^-1 all kept
// their sweep counts, 2^-1 routing most pairs of the n = 2048 solve to the
// tensor cores.  tc_flag[p], cc_flag[p] in {0, 1}.
constexpr float TC_SMALL_E = 0.5f;

__global__ void route_kernel(const float2 *__restrict__ zhat, const int *__restrict__ pair_flag, int kk,
                             float small_e, int *__restrict__ tc_flag, int *__restrict__ cc_flag)
{
    __shared__ int large;
    const int pair = blockIdx.x;
    if (threadIdx.x == 0) large = 0;
    __syncthreads();
    const bool active = pair_flag[pair] != 0;
    if (active) {
        const float2 *zp = zhat + (long long)pair * (KKMAX * KKMAX);
        bool big = false;
        for (int e = threadIdx.x; e < kk * kk; e += blockDim.x) {
            const int l = e % kk, j = e / kk;
            const float2 z = zp[l + KKMAX * j];
            const float ex = z.x - (l == j ? 1.0f : 0.0f);
            big |= fabsf(ex) > small_e || fabsf(z.y) > small_e || !(ex == ex) || !(z.y == z.y);
        }
        if (big) large = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_flag[pair] = active && !large;
        cc_flag[pair] = active && large;
    }
}

bool tc_supported(int kk, int npairs, long long ld)
{
    // W32's base and column stride must be 16-byte aligned (cudaMalloc'd; ld a
    // multiple of ROWPAD); two blocks of at most 32 columns; the active-pair
    // list of the update fits its shared table.
    return kk <= KKMAX && npairs <= tc::U_MAXPAIRS && ld % 2 == 0 && encode_fn() != nullptr;
}

int tc_gram_chunk_rows(int m_pad, int p_pad, int npairs, int sms)
{
    // two Gram CTAs per SM: the chunk (a multiple of 16 rows, at least 64)
    // whose CTA count fills whole waves of 2 x sms best
    const long long slots = 2LL * sms;
    int best = 256;
    double best_eff = -1.0;
    for (int kc = 64; kc <= 2048; kc += 16) {
        const long long ch = (m_pad + kc - 1) / kc + (p_pad + kc - 1) / kc;
        const long long ctas = ch * npairs;
        const long long waves = (ctas + slots - 1) / slots;
        // time ~ waves x rows per CTA, plus a fixed cost per CTA (tensor-memory
        // allocation, pipeline fill, epilogue) of about 48 rows
        const double cost = (double)waves * (kc + 48);
        const double eff = 1.0 / cost;
        if (eff > best_eff * (1.0 + 1e-9)) {
            best_eff = eff;
            best = kc;
        }
    }
    return best;
}

cudaError_t tc_setup()
{
    cudaError_t e = cudaFuncSetAttribute(tc::gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::G_SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(tc::update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::U_SMEM);
}

cudaError_t launch_gram_tc(const void *W32, const int8_t *Jrow, const StepArgs &s, int n, void *partial, int *err,
                           cudaStream_t st)
{
    CUtensorMap map;
    cudaError_t e = make_map(&map, W32, s.ld, n, tc::G_RS, 32);
    if (e != cudaSuccess) return e;
    tc::GramTcArgs a;
    a.slotcol = s.slotcol;
    a.Jrow = Jrow;
    a.partial = (float2 *)partial;
    a.err = err;
    a.kk = s.kk;
    a.wb = s.kk / 2;
    a.m_pad = s.m_pad;
    a.p_pad = s.p_pad;
    a.kc = s.kc;
    a.chunks_h = s.chunks_h;
    a.chunks_s = s.chunks_s;
    const int grid = s.npairs * (s.chunks_h + s.chunks_s);
    tc::gram_tc_kernel<<<grid, tc::G_THREADS, tc::G_SMEM, st>>>(map, a);
    return cudaGetLastError();
}

cudaError_t launch_route(const double2 *zhat, const int *pair_flag, int kk, int npairs, int *tc_flag, int *cc_flag,
                         cudaStream_t st)
{
    route_kernel<<<npairs, 256, 0, st>>>((const float2 *)zhat, pair_flag, kk, TC_SMALL_E, tc_flag, cc_flag);
    return cudaGetLastError();
}

cudaError_t launch_update_tc(void *W32, const StepArgs &s, int n, const double2 *zhat, const int *pair_flag,
                             int *err, int sms, cudaStream_t st)
{
    CUtensorMap map;
    cudaError_t e = make_map(&map, W32, s.ld, n, tc::U_ROWS, tc::U_KC);
    if (e != cudaSuccess) return e;
    tc::UpdTcArgs a;
    a.slotcol = s.slotcol;
    a.zhat = (const float2 *)zhat;
    a.pair_flag = pair_flag;
    a.W = (float2 *)W32;
    a.err = err;
    a.ld = s.ld;
    a.npairs = s.npairs;
    a.kk = s.kk;
    a.wb = s.kk / 2;
    a.tiles_per_pair = (int)((s.ld + tc::U_ROWS - 1) / tc::U_ROWS);
    a.Mt = (int)s.ld;
    tc::update_tc_kernel<<<sms, tc::U_THREADS, tc::U_SMEM, st>>>(map, a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ghsvd_tc_block_ops: the two tensor-core kernels on one block pair, for
// verification against an FP64 reference (include/ghsvd.h).
// ---------------------------------------------------------------------------
namespace {

__global__ void tc_check_setup(int *slotcol, int *pair_flag, int8_t *Jrow, const int8_t *J, int rows)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 64) slotcol[t] = t;
    if (t == 0) pair_flag[0] = 1;
    if (t < rows) Jrow[t] = J ? J[t] : (int8_t)1;
}

// sum the complex64 partials of one pair in chunk order (FP64), mirror the
// upper part into the lower (conjugate), round to complex64
__global__ void tc_check_sum(const float2 *partial, int chunks, float2 *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 64 * 64) return;
    const int i = t % 64, j = t / 64;
    const bool mirror = i > j;
    const int e = mirror ? j + 64 * i : i + 64 * j;
    double re = 0.0, im = 0.0;
    for (int c = 0; c < chunks; ++c) {
        re += (double)partial[(long long)c * 64 * 64 + e].x;
        im += (double)partial[(long long)c * 64 * 64 + e].y;
    }
    out[t] = make_float2((float)re, (float)(mirror ? -im : im));
}

}  // namespace
}  // namespace hz

namespace {

// p is device (or managed) memory of the current device
bool on_current_device(const void *p)
{
    int dev = 0;
    cudaPointerAttributes a{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" ghsvd_status ghsvd_tc_block_ops(int64_t rows, void *X, int64_t ldx, const int8_t *J, const void *Z,
                                           void *gram, void *stream)
{
    if (rows < 64 || rows % 64 != 0 || rows > (1 << 24) || !X || !Z || !gram || ldx != rows)
        return GHSVD_ERR_INVALID_ARG;
    if (!on_current_device(X) || !on_current_device(Z) || !on_current_device(gram) ||
        (J && !on_current_device(J)))
        return GHSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (hz::tc_setup() != cudaSuccess || !hz::tc_supported(64, 1, ldx)) return GHSVD_ERR_CUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GHSVD_ERR_CUDA;
    const int r = (int)rows;
    // J given: X is the F range of a pencil (J applied); else the G range
    const int m_pad = J ? r : 0, p_pad = J ? 0 : r;
    const int kc = hz::tc_gram_chunk_rows(m_pad, p_pad, 1, sms);
    const int ch = (r + kc - 1) / kc;
    int *slotcol = nullptr, *flag = nullptr, *err = nullptr;
    int8_t *Jrow = nullptr;
    void *partial = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&slotcol, 64 * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&flag, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&err, 2 * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&Jrow, (size_t)r, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&partial, (size_t)ch * 64 * 64 * sizeof(float2), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) {
        hz::tc_check_setup<<<(r + 255) / 256, 256, 0, st>>>(slotcol, flag, Jrow, J, r);
        e = cudaGetLastError();
    }
    hz::StepArgs sa{};
    sa.slotcol = slotcol;
    sa.npairs = 1;
    sa.kk = 64;
    sa.m_pad = m_pad;
    sa.p_pad = p_pad;
    sa.n_pad = 0;
    sa.ld = ldx;
    sa.kc = kc;
    sa.chunks_h = J ? ch : 0;
    sa.chunks_s = J ? 0 : ch;
    if (e == cudaSuccess) e = hz::launch_gram_tc(X, Jrow, sa, 64, partial, err, st);
    if (e == cudaSuccess) {
        hz::tc_check_sum<<<16, 256, 0, st>>>((const float2 *)partial, ch, (float2 *)gram);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = hz::launch_update_tc(X, sa, 64, (const double2 *)Z, flag, err, sms, st);
    int herr[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(slotcol, st);
    cudaFreeAsync(flag, st);
    cudaFreeAsync(err, st);
    cudaFreeAsync(Jrow, st);
    cudaFreeAsync(partial, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return GHSVD_ERR_CUDA;
    if (herr[0] & hz::DEVERR_TIMEOUT) return GHSVD_ERR_CUDA;
    return GHSVD_OK;
}
