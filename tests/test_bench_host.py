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


@pytest.mark.parametrize("prec,kernel", [("df64", "k_apply_win"), ("fp32", "k_apply_nat"), ("fp64", "k_apply_win")])
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


def test_serve_oracle_errors_match_requests_by_model():
    """Served energies are compared with the oracle golden only for requests
    whose model seed, N_s and sector match the golden entry (streams of other
    lengths draw other N_s for the same request index)."""
    stream = [{"n_s": 10, "model_seed": 1000, "n_up": 5, "n_dn": 5},
              {"n_s": 11, "model_seed": 1001, "n_up": 6, "n_dn": 5}]
    golden = {0: {"n_s": 10, "model_seed": 1000, "sector": [5, 5], "E": [-2.0, -1.0], "G_re": [0.5], "G_im": [-0.5]},
              1: {"n_s": 12, "model_seed": 1001, "sector": [6, 6], "E": [-9.0, -8.0], "G_re": [0.0], "G_im": [0.0]}}
    import numpy as np
    res = {0: {"E": [-2.0 * (1 + 1e-9), -1.0], "G": np.array([0.5 - 0.5j + 1e-7])},
           1: {"E": [-1.0, 0.0], "G": np.array([1.0 + 0j])}}
    r = bench.oracle_errors(res, golden, [0], 2, stream)
    assert r["requests_checked"] == 1                      # request 1 is another model
    assert r["max_rel_E_err_vs_oracle"] == pytest.approx(1e-9, rel=1e-6)
    assert r["max_abs_G_err_vs_oracle"] == pytest.approx(1e-7, rel=1e-6)
    assert bench.oracle_errors(res, {}, [], 2, stream)["requests_checked"] == 0


def test_serve_fifo_latencies():
    """The plain path's latencies: a first-come-first-served queue over the
    measured service times."""
    # all at t = 0: each waits for the ones before it
    assert bench.fifo_latencies_ms([1.0, 2.0, 0.5], [0.0, 0.0, 0.0]) == pytest.approx([1000, 3000, 3500])
    # sparse arrivals: no queueing; a burst: the second waits
    assert bench.fifo_latencies_ms([1.0, 1.0], [0.0, 5.0]) == pytest.approx([1000, 1000])
    assert bench.fifo_latencies_ms([1.0, 1.0, 1.0], [0.0, 0.5, 10.0]) == pytest.approx([1000, 1500, 1000])
    assert bench.tr_basis(4) == 24 and bench.tr_basis(1) == 20 and bench.tr_basis(16) == 64
