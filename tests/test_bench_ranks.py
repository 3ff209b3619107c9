"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks.

The path does not shard (replicas only): ranks share nothing but the
max-over-ranks timing and a barrier.  Checks that the reduction takes each
timing's maximum, that the whole-job rate counts every rank's bytes against the
slowest rank, and that the reference arm runs on rank 0 only.
"""
import contextlib
import io
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.ranks_max([1.0 + rank, 5.0 - rank, 0.25], dist, "cpu")
        dist.barrier()
        q.put((rank, ms, bench.whole_job_gbs(world, 2e9, ms[0])))
    finally:
        dist.destroy_process_group()


def test_ranks_max_and_whole_job_rate_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, gbs in got:
        assert ms == [2.0, 5.0, 0.25]
        # both ranks' 2 GB against the slower rank's 2 ms
        assert gbs == pytest.approx(2 * 2e9 / 2e-3 / 1e9)


def test_single_rank_identity():
    assert bench.ranks_max([3.5, 1], None, "cpu") == [3.5, 1.0]
    assert bench.whole_job_gbs(1, 1e9, 1.0) == pytest.approx(1000.0)


def test_reference_arm_other_ranks_do_nothing(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(bench.args_parse([]))
    assert out.getvalue() == ""


def test_reference_arm_json_line(monkeypatch):
    """bench.py --impl reference on rank 0: one JSON line with the base
    contract's keys, the oracle as the CPU baseline, and an e2e with no copies."""
    import json
    monkeypatch.setenv("RANK", "0")
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(bench.args_parse(["--impl", "reference", "--steps", "1", "--warmup", "0"]))
    lines = [l for l in out.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GB/s"
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("three-orbital Kanamori impurity, N_s=15")
