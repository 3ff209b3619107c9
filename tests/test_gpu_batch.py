"""Batched Lanczos over many sectors (one graph replay per step, one launch per
kernel over all sectors) vs the oracle's exact spectra, sector by sector."""
import numpy as np
import pytest

import workloads as W
from oracle import sector as osec, spectrum
from tests._gpu import ensure_built, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    ed = ensure_built()
    ctx = ed.ed_ctx_create(0)
    yield ed, ctx, torch
    ed.ed_ctx_destroy(ctx)


def oracle_lowest(m, nu, nd, k):
    H = osec.build_csr(m, nu, nd)
    return spectrum.lowest(H, min(k, H.shape[0]))


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_all_sectors_small_model(env, prec):
    """Every (N_up, N_dn) sector of a 7-site two-orbital Kanamori impurity."""
    ed, ctx, torch = env
    m = W.kanamori(7, seed=2, n_orb=2)
    secs = [(a, b) for a in range(8) for b in range(8)]
    k = 4
    b = ed.ed_batch_create(ctx, m, secs, prec)
    try:
        ev, it, info, st = ed.ed_batch_lanczos(b, len(secs), k=k, tol=1e-11, max_iter=200, check_every=5)
        assert info.n_sectors == len(secs) and info.graph_replays == info.steps
        for q, (a, bb) in enumerate(secs):
            ref = oracle_lowest(m, a, bb, k)
            got = ev[q, :len(ref)]
            assert np.all(np.isnan(ev[q, len(ref):]))
            assert np.max(np.abs(got - ref) / np.maximum(1, np.abs(ref))) <= 1e-10, (a, bb, got, ref)
    finally:
        ed.ed_batch_destroy(b)


def test_n12_mixed_sizes(env):
    """Sectors of the N_s=12 three-orbital model from dim 1 to 853,776 in one batch."""
    ed, ctx, torch = env
    m = W.kanamori(12, seed=0)
    secs = [(6, 6), (0, 0), (12, 12), (1, 0), (11, 3), (5, 6), (2, 9)]
    k = 8
    b = ed.ed_batch_create(ctx, m, secs, "fp64")
    try:
        ev, it, info, st = ed.ed_batch_lanczos(b, len(secs), k=k, tol=1e-10, max_iter=400)
        for q, (a, bb) in enumerate(secs):
            ref = oracle_lowest(m, a, bb, k)
            got = ev[q, :len(ref)]
            assert np.max(np.abs(got - ref) / np.maximum(1, np.abs(ref))) <= 1e-10, (a, bb, got, ref)
    finally:
        ed.ed_batch_destroy(b)


def test_fp32_vectors_batch(env):
    ed, ctx, torch = env
    m = W.kanamori(10, seed=4)
    secs = [(5, 5), (4, 5), (5, 4), (3, 3)]
    b = ed.ed_batch_create(ctx, m, secs, "fp32")
    try:
        ev, it, info, st = ed.ed_batch_lanczos(b, len(secs), k=1, tol=1e-6, max_iter=300, allow_not_converged=True)
        for q, (a, bb) in enumerate(secs):
            ref = oracle_lowest(m, a, bb, 1)
            assert abs(ev[q, 0] - ref[0]) <= 1e-6 * abs(ref[0]), (a, bb, ev[q, 0], ref[0])
    finally:
        ed.ed_batch_destroy(b)


def test_sector_packing_chunks_and_tuner(env):
    """Eigenvalues do not depend on how sectors are cut into work items (beyond
    the order of sums); the packing tuner reports every candidate and keeps the
    fastest; bad chunk sizes are rejected."""
    ed, ctx, torch = env
    m = W.kanamori(8, seed=1)
    secs = [(a, b) for a in range(2, 7) for b in range(2, 7)]
    b = ed.ed_batch_create(ctx, m, secs, "fp64")
    try:
        res = {}
        for c in (64, 1024, 8192):
            ed.ed_batch_set_chunk(b, c)
            ev, it, info, st = ed.ed_batch_lanczos(b, len(secs), k=3, tol=1e-11, max_iter=200, check_every=5)
            res[c] = ev
        for c in (64, 8192):
            assert np.nanmax(np.abs(res[c] - res[1024])) <= 1e-10
        for q, (a, bb) in enumerate(secs[:6]):
            ref = oracle_lowest(m, a, bb, 3)
            assert np.max(np.abs(res[1024][q, :len(ref)] - ref)) <= 1e-10 * max(1, np.max(np.abs(ref)))
        r = ed.ed_batch_autotune(b, steps=8)
        ms = np.array(r.ms_per_step[:r.n_candidates])
        assert r.n_candidates == 8 and np.all(ms > 0)
        assert r.chosen == int(np.argmin(ms))
        assert list(r.chunk[:8]) == [256, 512, 1024, 2048, 4096, 8192, 16384, 32768]
        ev, it, info, st = ed.ed_batch_lanczos(b, len(secs), k=3, tol=1e-11, max_iter=200, check_every=5)
        assert np.nanmax(np.abs(ev - res[1024])) <= 1e-10
        for bad in (0, 100, 32, 131072):
            with pytest.raises(ed.EdError):
                ed.ed_batch_set_chunk(b, bad)
    finally:
        ed.ed_batch_destroy(b)
