// hz_kernels.cuh -- kernels of one outer step of the Level-2 block HZ method
// (arXiv 1907.08560, Section 6.4), and the set-up / finalization kernels.
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
#include "hz_gram.cuh"
#include "hz_inner.cuh"
#include "hz_update.cuh"
