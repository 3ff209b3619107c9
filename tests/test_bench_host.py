"""Host-side bookkeeping of bench.py (CPU only): compulsory bytes, whole-job
rates, the arithmetic ceiling, and the rule that ncu traffic is reported only
for the kernel source it was captured from."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_compulsory_bytes():
    dim = 6435 * 6435
    assert bench.alg_bytes("df64", dim) == 2 * dim * 8 == 662547600
    assert bench.alg_bytes("fp64", dim) == 662547600
    assert bench.alg_bytes("fp32", dim) == 2 * dim * 4


def test_whole_job_rate_counts_every_rank():
    # 662.5 MB per rank in 0.6 ms: 1104 GB/s on one rank, four times that on four
    one = bench.whole_job_gbs(1, 662547600, 0.6)
    assert one == pytest.approx(662547600 / 0.6e-3 / 1e9)
    assert bench.whole_job_gbs(4, 662547600, 0.6) == pytest.approx(4 * one)


def test_alu_ceiling_arithmetic():
    dim, nnz = 41409225, 14.653
    r = bench.alu_roofline("df64", dim, nnz, 0.6)
    ops = dim * (nnz + 1.0) * 12
    assert r["ops_per_launch"] == pytest.approx(ops)
    assert r["peak"] == pytest.approx(152 * 128 * 2.07e9 / 1e12, abs=1e-3)
    assert r["frac"] == pytest.approx(ops / 0.6e-3 / (152 * 128 * 2.07e9), abs=1e-4)
    f = bench.alu_roofline("fp64", dim, nnz, 1.3)
    assert f["unit"] == "T DFMA/s" and f["ops_per_launch"] == pytest.approx(dim * (nnz + 1.0))
    assert f["peak"] == pytest.approx(0.50, abs=1e-3)      # measured DFMA rate, T/s
    # FP32 vectors: one FP32 FMA per multiply-add (natural-order kernel, float sums)
    assert bench.alu_roofline("fp32", dim, nnz, 0.5)["ops_per_launch"] == pytest.approx(dim * (nnz + 1.0))


@pytest.mark.parametrize("prec,kernel", [("df64", "k_apply_win"), ("fp32", "k_apply_pair"), ("fp64", "k_apply_win")])
def test_traffic_only_for_the_captured_source(prec, kernel):
    p = os.path.join(ROOT, "profiles", f"{kernel}_{prec}_n15_traffic.txt")
    kv = dict(line.split(":", 1) for line in open(p) if ":" in line)
    sha = kv["apply_src_sha"].strip()
    assert bench.traffic_for(sha, prec, kernel) == float(kv["dram_bytes_per_launch"])
    assert bench.traffic_for("0" * 16, prec, kernel) is None          # another kernel source
    assert bench.traffic_for(sha, prec, "no_such_kernel") is None      # no capture at all


def test_row_kernel_names():
    assert bench.row_kernel("fp32") == "k_apply_nat" and bench.row_kernel("df64") == "k_apply_win"
    assert bench.row_kernel_of(2) == "k_apply_win" and bench.row_kernel_of(3) == "k_apply_pair"
    assert bench.row_kernel_of(4) == "k_apply_nat"
