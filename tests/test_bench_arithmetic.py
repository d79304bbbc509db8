"""The roofline arithmetic of bench.py, on the CPU: the algorithmic flops of a
sweep and of one Gram / update launch (complex MAC = 8 real flops; Hermitian
block Grams; the update of the stacked rows of F, G and Z'), counted here
pair by pair over the round-robin of one sweep, and the DRAM-traffic record
of the update kernel, reported only while it belongs to the kernel source."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def count_sweep(n, m, p, w):
    # one sweep of the block round-robin (circle method over nb blocks):
    # every pair of block columns once, each pair a Hermitian 2w x 2w Gram
    # over the m + p rows of F and G and a 2w x 2w update of m + p + n rows
    nb = n // w
    k = 2 * w
    pairs = set()
    for r in range(nb - 1):
        for j in range(nb // 2):
            if j == 0:
                a, b = nb - 1, r
            else:
                a, b = (r + j) % (nb - 1), (r - j) % (nb - 1)
            pairs.add((min(a, b), max(a, b)))
    assert len(pairs) == nb * (nb - 1) // 2
    gram = sum(k * (k + 1) // 2 * (m + p) for _ in pairs)
    update = sum(k * k * (m + p + n) for _ in pairs)
    return 8 * gram, 8 * update, nb


def test_flops_of_the_n2048_sweep():
    gram, update, nb = count_sweep(2048, 3072, 4096, 32)
    assert bench.flops_per_sweep() == gram + update
    assert abs((gram + update) / 1e12 - 0.849) < 0.001          # 0.849 TFLOP per sweep
    # a step launches each kernel once over nb / 2 pairs; nb - 1 steps a sweep
    assert bench.update_flops_per_launch() * (nb - 1) == update
    assert bench.gram_flops_per_launch() * (nb - 1) == gram
    assert bench.update_flops_per_launch() == 32 * 9216 * 64 * 64 * 8
    assert bench.gram_flops_per_launch() == 32 * 2080 * 7168 * 8


def test_traffic_record_is_used_only_for_the_kernel_it_was_taken_on():
    rec = json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))
    src = os.path.join(ROOT, "paper_1907_08560_gb300", "csrc", rec["source"])
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["sha256"]:
        assert bench.traffic_per_launch() is None     # the kernel changed since: null
        return
    assert rec["bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    assert bench.traffic_per_launch() == rec["bytes_per_launch"]
    # at the algorithmic bytes of a launch (302 MB read, 302 MB written; part
    # of the writes still in L2 when the kernel ends), no re-reads
    algo = 2 * 9216 * 2048 * 16
    assert 0.8 * algo < rec["bytes_per_launch"] <= 1.05 * algo
