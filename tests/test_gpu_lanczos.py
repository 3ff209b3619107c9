"""Lanczos on the GPU (through the C ABI) vs the oracle's exact spectra.

Eigenvalues: |theta - lambda| <= 1e-10 max(1, |lambda|) for FP64 and DF64
vectors; FP32 vectors: ground energy within 1e-6 relative.
"""
import numpy as np
import pytest

import workloads as W
from oracle import sector as osec, spectrum
from tests._gpu import ensure_built, torch_cuda, empty_vec, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    ed = ensure_built()
    ctx = ed.ed_ctx_create(0)
    yield ed, ctx, torch
    ed.ed_ctx_destroy(ctx)


def ev_err(a, b):
    return np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)))


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_c0_ground_energy(env, prec):
    """AIM N_s=6, (3,3), dim 400: lowest eigenvalue to tol 1e-12."""
    ed, ctx, torch = env
    m = W.aim(6, seed=0)
    ref = spectrum.lowest(osec.build_csr(m, 3, 3), 1)
    sec = ed.ed_sector_create(ctx, m, 3, 3, prec)
    try:
        ev, info, st = ed.ed_lanczos(sec, k=1, tol=1e-12, max_iter=400)
        assert ev_err(ev, ref) <= 1e-10, (ev, ref)
        assert info.n_converged == 1 and info.residual[0] <= 1e-12 * max(1, abs(ev[0]))
    finally:
        ed.ed_sector_destroy(sec)


def test_c0_fp32_vectors(env):
    ed, ctx, torch = env
    m = W.aim(6, seed=0)
    ref = spectrum.lowest(osec.build_csr(m, 3, 3), 1)
    sec = ed.ed_sector_create(ctx, m, 3, 3, "fp32")
    try:
        ev, info, st = ed.ed_lanczos(sec, k=1, tol=1e-7, max_iter=400, allow_not_converged=True)
        assert abs(ev[0] - ref[0]) <= 1e-6 * abs(ref[0])
    finally:
        ed.ed_sector_destroy(sec)


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_eight_lowest_small(env, prec):
    ed, ctx, torch = env
    m = W.kanamori(8, seed=1)
    H = osec.build_csr(m, 4, 3)
    ref = spectrum.lowest(H, 8)
    sec = ed.ed_sector_create(ctx, m, 4, 3, prec)
    try:
        n = H.shape[0]
        vecs = empty_vec(n, prec, ed, torch, count=8)
        ev, info, st = ed.ed_lanczos(sec, k=8, tol=1e-11, max_iter=600, evecs=vecs)
        assert ev_err(ev, ref) <= 1e-10, (ev, ref)
        V = to_host(vecs, prec, 8 * n, ed, torch).reshape(8, n)
        for i in range(8):
            r = H @ V[i] - ev[i] * V[i]
            assert np.linalg.norm(r) <= 1e-8 * max(1, abs(ev[i])), (i, np.linalg.norm(r))
            assert abs(np.linalg.norm(V[i]) - 1.0) < 1e-10
    finally:
        ed.ed_sector_destroy(sec)


def test_c1_eight_lowest(env):
    """Three-orbital Kanamori, N_s=12, (6,6), dim 853,776, 8 lowest, FP64 vectors."""
    ed, ctx, torch = env
    m = W.kanamori(12, seed=0)
    H = osec.build_csr(m, 6, 6)
    ref = spectrum.lowest(H, 8)
    sec = ed.ed_sector_create(ctx, m, 6, 6, "fp64")
    try:
        ev, info, st = ed.ed_lanczos(sec, k=8, tol=1e-10, max_iter=500)
        assert ev_err(ev, ref) <= 1e-10, (ev, ref)
    finally:
        ed.ed_sector_destroy(sec)


def test_small_dimensions_and_restart(env):
    ed, ctx, torch = env
    m = W.kanamori(8, seed=2)
    # dim 1 sectors
    for nu, nd in ((0, 0), (8, 8)):
        H = osec.build_csr(m, nu, nd)
        sec = ed.ed_sector_create(ctx, m, nu, nd, "fp64")
        try:
            ev, info, st = ed.ed_lanczos(sec, k=1, tol=1e-12, max_iter=10)
            assert abs(ev[0] - H.toarray()[0, 0]) <= 1e-12 * max(1, abs(ev[0]))
        finally:
            ed.ed_sector_destroy(sec)
    # dim 8 < k = 12: every eigenvalue, rest NaN; restarts after the Krylov space closes
    H = osec.build_csr(m, 1, 8)
    ref = np.linalg.eigvalsh(H.toarray())
    sec = ed.ed_sector_create(ctx, m, 1, 8, "fp64")
    try:
        ev, info, st = ed.ed_lanczos(sec, k=12, tol=1e-12, max_iter=50)
        assert np.all(np.isnan(ev[8:]))
        assert ev_err(ev[:8], ref) <= 1e-10
    finally:
        ed.ed_sector_destroy(sec)
    # atomic limit: degenerate multiplets inside one sector need restarts
    a = W.atom(3)
    H = osec.build_csr(a, 2, 1)
    ref = np.linalg.eigvalsh(H.toarray())
    sec = ed.ed_sector_create(ctx, a, 2, 1, "fp64")
    try:
        ev, info, st = ed.ed_lanczos(sec, k=len(ref), tol=1e-12, max_iter=100)
        assert ev_err(ev, ref) <= 1e-10, (ev, ref)
    finally:
        ed.ed_sector_destroy(sec)


def test_without_reorthogonalisation_ground_state(env):
    """Two-pass ground state with 3 resident vectors (the large-sector mode)."""
    ed, ctx, torch = env
    m = W.kanamori(10, seed=3)
    H = osec.build_csr(m, 5, 5)
    ref, refv = spectrum.lowest(H, 1, vectors=True)
    sec = ed.ed_sector_create(ctx, m, 5, 5, "fp64")
    try:
        n = H.shape[0]
        v = torch.empty(n, dtype=torch.float64, device="cuda")
        ev, info, st = ed.ed_lanczos(sec, k=1, tol=1e-11, max_iter=300, reorth=False, evecs=v)
        assert ev_err(ev, ref) <= 1e-10
        assert 0.0 < info.apply_ms < info.total_ms
        vv = v.cpu().numpy()
        assert abs(abs(vv @ refv[:, 0]) - 1.0) <= 1e-9
    finally:
        ed.ed_sector_destroy(sec)


_C1 = {}


def c1_reference():
    if not _C1:
        m = W.kanamori(12, seed=0)
        H = osec.build_csr(m, 6, 6)
        w, v = spectrum.lowest(H, 1, vectors=True)
        _C1.update(m=m, H=H, e0=w[0], v0=v[:, 0])
    return _C1


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_c1_ground_state_three_vectors(env, prec):
    """C1 ground state with three resident vectors (fused H*v + <q, Hq>, fused
    update + norm) and the regenerated Ritz vector."""
    ed, ctx, torch = env
    r = c1_reference()
    sec = ed.ed_sector_create(ctx, r["m"], 6, 6, prec)
    try:
        n = r["H"].shape[0]
        v = empty_vec(n, prec, ed, torch)
        ev, info, st = ed.ed_lanczos(sec, k=1, tol=1e-11, max_iter=400, reorth=False, evecs=v)
        assert abs(ev[0] - r["e0"]) <= 1e-10 * abs(r["e0"]), (ev[0], r["e0"])
        vv = to_host(v, prec, n, ed, torch)
        assert abs(abs(vv @ r["v0"]) - 1.0) <= 1e-8
    finally:
        ed.ed_sector_destroy(sec)


def test_c1_fp32_every_natural_order_variant(env):
    """Each launch shape of the float natural-order kernel (four or two rows per
    block, 256 to 1024 threads) inside the three-vector Lanczos step, where
    H*v also returns its per-block parts of <q, Hq>: ground energy within 1e-6
    relative of the oracle's."""
    ed, ctx, torch = env
    r = c1_reference()
    sec = ed.ed_sector_create(ctx, r["m"], 6, 6, "fp32")
    try:
        for v in range(10, 16):
            ed.ed_sector_set_variant(sec, v)
            ev, info, st = ed.ed_lanczos(sec, k=1, tol=1e-7, max_iter=400, reorth=False, allow_not_converged=True)
            assert ed.ed_sector_get_info(sec).kernel == 4
            assert abs(ev[0] - r["e0"]) <= 1e-6 * abs(r["e0"]), (v, ev[0], r["e0"])
    finally:
        ed.ed_sector_destroy(sec)


def test_c1_fp32_vectors_ground_energy(env):
    """FP32 Lanczos vectors, double-float products: ground energy within 1e-6 relative."""
    ed, ctx, torch = env
    r = c1_reference()
    sec = ed.ed_sector_create(ctx, r["m"], 6, 6, "fp32")
    try:
        ev, info, st = ed.ed_lanczos(sec, k=1, tol=1e-7, max_iter=400, reorth=False, allow_not_converged=True)
        assert abs(ev[0] - r["e0"]) <= 1e-6 * abs(r["e0"]), (ev[0], r["e0"])
    finally:
        ed.ed_sector_destroy(sec)
