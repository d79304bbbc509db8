"""Host-side rules of the CUDA library (hz_launch.h, hz_pivot.cuh), compiled
for the CPU with nvcc and checked without a GPU: the Gram row chunk, the
thread counts of the Gram CTAs, the shared-memory budgets of the step kernels
and the round-robin table (Section 6.3)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SMEM_MAX = 227 * 1024          # dynamic shared memory of one CTA on sm_103a


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("host") / "host_logic")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode",
                        "arch=compute_103a,code=sm_103a", os.path.join(HERE, "host_logic.cu"),
                        "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def run(prog, *args):
    return subprocess.run([prog, *map(str, args)], capture_output=True, text=True,
                          check=True).stdout.split("\n")


def chunk(prog, m_pad, p_pad, npairs, sms):
    return int(run(prog, "chunk", m_pad, p_pad, npairs, sms)[0])


def test_gram_chunk_of_the_benchmark_pencils(prog):
    # tall n = 2048 pencil (3072 + 4096 rows): 14 chunks x 32 pairs = 448 CTAs;
    # shortened (2048 + 2048 rows): 320-row chunks, again 448 CTAs, not the
    # 1024-row chunks (128 CTAs, one per SM) of the plain wave count
    assert chunk(prog, 3072, 4096, 32, 152) == 512
    assert chunk(prog, 2048, 2048, 32, 152) == 320


@pytest.mark.parametrize("m_pad,p_pad,npairs", [(3072, 4096, 32), (2048, 2048, 32), (576, 768, 12),
                                                (64, 128, 1), (1536, 2048, 24), (8192, 8192, 64)])
def test_gram_chunk_rule(prog, m_pad, p_pad, npairs):
    sms = 152
    kc = chunk(prog, m_pad, p_pad, npairs, sms)
    assert kc % 16 == 0 and 128 <= kc <= 4096

    def ctas(c):
        return npairs * (-(-m_pad // c) - (-p_pad // c))
    candidates = range(128, 4097, 64)
    if any(ctas(c) >= 2 * sms for c in candidates):
        assert ctas(kc) >= 2 * sms      # at least two CTAs per SM when any chunk gives that


def test_shared_memory_budgets_and_gram_threads(prog):
    lines = [l.split() for l in run(prog, "sizes") if l]
    smem = dict(zip(lines[0][1::2], map(int, lines[0][2::2])))
    assert all(v <= SMEM_MAX for v in smem.values())
    # complex128 update: Z^ and the row tile plus their real sums (24 bytes an entry)
    assert smem["update16"] == 24 * 128 * 65
    for _, kk, t64, t128 in lines[1:]:
        kk, t64, t128 = int(kk), int(t64), int(t128)
        nt = (kk + 15) // 16
        # complex64: 16 threads per upper 16 x 16 tile; complex128: whole warps
        # for the off-diagonal tiles, one warp for the diagonal ones, and at
        # least two threads per diagonal entry
        assert t64 == max(32, 16 * nt * (nt + 1) // 2)
        assert t128 % 32 == 0 and t128 - 32 >= 16 * nt * (nt - 1) // 2 and t128 >= 32 * nt
        assert t128 <= 128


@pytest.mark.parametrize("N", [2, 4, 10, 64, 66])
def test_round_robin_table(prog, N):
    rows = [tuple(map(int, l.split())) for l in run(prog, "rr", N) if l]
    seen = set()
    for r in range(N - 1):
        step = [(a, b) for (rr, _, a, b) in rows if rr == r]
        cols = [c for p in step for c in p]
        assert len(step) == N // 2 and sorted(cols) == list(range(N))   # disjoint, all slots
        assert all(a < b for a, b in step)
        seen.update(step)
    assert len(seen) == N * (N - 1) // 2                              # every pair once a sweep


def test_delta_update_tiles_fit(prog):
    # the delta-form tiles of the FP64 sweeps: the double-float tile runs two
    # CTAs per SM; the batched FP64 update runs either delta tile (and the
    # double-float tile twice, on the two halves of a 64-row tile) inside the
    # shared memory it is launched with for the FP64 product
    d64, df, upd16, upd_r, df_r, delta_e, df_e = run(prog, "delta")[0].split()
    d64, df, upd16, upd_r, df_r = map(int, (d64, df, upd16, upd_r, df_r))
    assert upd_r == 2 * df_r
    assert d64 <= upd16 and df <= upd16 <= SMEM_MAX
    assert 2 * (df + 1024) <= 228 * 1024
    assert float(delta_e) == 2.0 ** -29 and float(df_e) == 2.0 ** -11
