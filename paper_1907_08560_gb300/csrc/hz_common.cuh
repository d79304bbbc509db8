// hz_common.cuh -- shared device types of the step kernels of one outer step
// of the Level-2 block HZ method (arXiv 1907.08560, Section 6.4): the Gram
// (hz_gram.cuh), the inner level (hz_inner.cuh) and the update (hz_update.cuh).
//
// Data layout in HBM (one working buffer W per precision):
//   W is column-major with leading dimension ld = Mt = m_pad + p_pad + n_pad;
//   rows [0, m_pad) hold F, rows [m_pad, m_pad + p_pad) hold G and rows
//   [m_pad + p_pad, Mt) hold Z'.  Each row range is padded with zero rows to a
//   multiple of 64, so no kernel has a ragged row tail: zero rows add nothing
//   to a Gram and stay zero under a column update.  Stacking F, G, Z' makes
//   the block update of Section 6.4.3 (three ZGEMMs in the paper) one
//   contraction over all Mt rows.
//
// A block column pair (P, Q) of an outer step occupies the kk = 2 wb slots of
// its block pivot: P's columns in slots [0, |P|), Q's in [wb, wb + |Q|), wb
// the widest block; slotcol[pair][s] is the column of slot s or -1 (an empty
// slot, i.e. a bordered one, Section 6.3.2).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "hz_launch.h"
#include "hz_pivot.cuh"

namespace hz {

template <typename T> struct cplx;
template <> struct cplx<double> { using t = double2; };
template <> struct cplx<float> { using t = float2; };

// Asynchronous copy of one B-byte element (B = 4, 8 or 16) from global to
// shared memory through L1 (cp.async), the commit of the copies issued so far
// as a group, and the wait until at most N groups are still in flight.
template <int B>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

}  // namespace hz
