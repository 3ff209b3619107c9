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
