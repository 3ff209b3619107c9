"""Thick-restart Lanczos (ed_lanczos_tr) on the GPU vs the oracle's exact spectra.

Eigenvalues: |theta - lambda| <= 1e-10 max(1, |lambda|) for FP64 and DF64
vectors (FP32 vectors: 1e-6 relative); Ritz vectors: ||H v - theta v|| <= 1e-8,
orthonormal.  Small bases force several restarts; degenerate atomic multiplets
need fresh directions after the Krylov space closes.
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


_C1 = {}


def c1_reference():
    if "H" not in _C1:
        m = W.kanamori(12, seed=0)
        H = osec.build_csr(m, 6, 6)
        _C1.update(m=m, H=H, ref=spectrum.lowest(H, 8))
    return _C1["m"], _C1["H"], _C1["ref"]


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("basis,keep", [(20, 12), (14, 10), (40, 0)])
def test_eight_lowest_small_sector(env, prec, basis, keep):
    """Kanamori N_s=8, (4,3), dim 3920: 8 lowest with bases of 14..40 vectors."""
    ed, ctx, torch = env
    m = W.kanamori(8, seed=1)
    H = osec.build_csr(m, 4, 3)
    ref = spectrum.lowest(H, 8)
    sec = ed.ed_sector_create(ctx, m, 4, 3, prec)
    try:
        n = H.shape[0]
        vecs = empty_vec(n, prec, ed, torch, count=8)
        ev, info, st = ed.ed_lanczos_tr(sec, k=8, tol=1e-11, max_basis=basis, keep=keep, max_iter=3000,
                                        evecs=vecs)
        assert ev_err(ev, ref) <= 1e-10, (ev, ref)
        assert info.n_converged == 8
        if basis < 40:
            assert info.restarts >= 1
        V = to_host(vecs, prec, 8 * n, ed, torch).reshape(8, n)
        for i in range(8):
            r = H @ V[i] - ev[i] * V[i]
            assert np.linalg.norm(r) <= 1e-8 * max(1, abs(ev[i])), (i, np.linalg.norm(r))
        G = V @ V.T
        assert np.max(np.abs(G - np.eye(8))) <= 1e-10
    finally:
        ed.ed_sector_destroy(sec)


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_c1_eight_lowest_bounded_basis(env, prec):
    """C1 (N_s=12, (6,6), dim 853,776): 8 lowest with a 32-vector basis."""
    ed, ctx, torch = env
    m, H, ref = c1_reference()
    sec = ed.ed_sector_create(ctx, m, 6, 6, prec)
    try:
        tol = 1e-7 if prec == "fp32" else 1e-10
        ev, info, st = ed.ed_lanczos_tr(sec, k=8, tol=tol, max_basis=32, keep=16, max_iter=3000,
                                        allow_not_converged=(prec == "fp32"))
        if prec == "fp32":
            assert np.max(np.abs(ev - ref) / np.abs(ref)) <= 1e-6
        else:
            assert ev_err(ev, ref) <= 1e-10, (ev, ref)
            assert info.n_converged == 8
        assert info.restarts >= 1
        eb = 4 if prec == "fp32" else 8
        # m + 2 + keep slots, each padded to a multiple of 32 elements
        ld = (H.shape[0] + 31) // 32 * 32
        assert info.basis_bytes == (32 + 2 + 16) * ld * eb
    finally:
        ed.ed_sector_destroy(sec)


def test_agrees_with_full_reorthogonalisation(env):
    ed, ctx, torch = env
    m = W.aim(6, seed=0)
    sec = ed.ed_sector_create(ctx, m, 3, 3, "fp64")
    try:
        a, _, _ = ed.ed_lanczos(sec, k=4, tol=1e-12, max_iter=400)
        b, info, _ = ed.ed_lanczos_tr(sec, k=4, tol=1e-12, max_basis=12, max_iter=2000)
        assert np.max(np.abs(a - b)) <= 1e-11 * max(1, np.max(np.abs(a)))
        assert info.restarts >= 1
    finally:
        ed.ed_sector_destroy(sec)


def test_degenerate_multiplets_and_small_sectors(env):
    ed, ctx, torch = env
    # atomic t2g Kanamori: degenerate multiplets, the Krylov space closes early
    a = W.atom(3)
    for nu, nd in ((2, 1), (2, 2)):
        H = osec.build_csr(a, nu, nd)
        ref = np.linalg.eigvalsh(H.toarray())
        k = min(len(ref), 12)
        sec = ed.ed_sector_create(ctx, a, nu, nd, "fp64")
        try:
            ev, info, st = ed.ed_lanczos_tr(sec, k=k, tol=1e-12, max_basis=min(len(ref), k + 6), max_iter=500)
            assert ev_err(ev, ref[:k]) <= 1e-10, (nu, nd, ev, ref[:k])
        finally:
            ed.ed_sector_destroy(sec)
    # dimension 1, and k larger than the dimension
    m = W.kanamori(8, seed=2)
    for nu, nd, k in ((0, 0, 1), (1, 8, 12)):
        H = osec.build_csr(m, nu, nd)
        ref = np.linalg.eigvalsh(H.toarray())
        sec = ed.ed_sector_create(ctx, m, nu, nd, "fp64")
        try:
            ev, info, st = ed.ed_lanczos_tr(sec, k=k, tol=1e-12, max_basis=min(40, len(ref)), max_iter=100)
            nn = len(ref)
            assert ev_err(ev[:nn], ref[:k]) <= 1e-10
            assert np.all(np.isnan(ev[nn:]))
        finally:
            ed.ed_sector_destroy(sec)


def test_invalid_arguments(env):
    ed, ctx, torch = env
    m = W.aim(6, seed=0)
    sec = ed.ed_sector_create(ctx, m, 3, 3, "fp64")
    try:
        for kw in (dict(k=4, max_basis=129), dict(k=8, max_basis=9), dict(k=4, max_basis=20, keep=3),
                   dict(k=4, max_basis=20, keep=19), dict(k=0), dict(k=65, max_basis=128)):
            with pytest.raises(ed.EdError):
                ed.ed_lanczos_tr(sec, **kw)
    finally:
        ed.ed_sector_destroy(sec)


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("solver", ["full_basis", "thick_restart"])
def test_odd_dimension_padded_basis(env, solver, prec):
    """Kanamori N_s=7 (3,4), dim 35^2 = 1225 (odd, 1 mod 4): the basis slots are
    padded to 32 elements and the CGS2 kernels read sixteen-byte vectors with
    an element-wise tail.  8 lowest eigenpairs against dense diagonalisation."""
    ed, ctx, torch = env
    m = W.kanamori(7, seed=5)
    H = osec.build_csr(m, 3, 4)
    n = H.shape[0]
    assert n == 1225
    ref = spectrum.lowest(H, 8)
    sec = ed.ed_sector_create(ctx, m, 3, 4, prec)
    try:
        vecs = empty_vec(n, prec, ed, torch, count=8)
        tol = 1e-7 if prec == "fp32" else 1e-11
        if solver == "full_basis":
            ev, info, st = ed.ed_lanczos(sec, k=8, tol=tol, max_iter=600, evecs=vecs,
                                         allow_not_converged=(prec == "fp32"))
        else:
            ev, info, st = ed.ed_lanczos_tr(sec, k=8, tol=tol, max_basis=24, keep=12, max_iter=4000,
                                            evecs=vecs, allow_not_converged=(prec == "fp32"))
        if prec == "fp32":
            assert np.max(np.abs(ev - ref) / np.abs(ref)) <= 1e-6, (ev, ref)
            return
        assert ev_err(ev, ref) <= 1e-10, (ev, ref)
        V = to_host(vecs, prec, 8 * n, ed, torch).reshape(8, n)
        for i in range(8):
            r = H @ V[i] - ev[i] * V[i]
            assert np.linalg.norm(r) <= 1e-8 * max(1, abs(ev[i])), (i, np.linalg.norm(r))
        assert np.max(np.abs(V @ V.T - np.eye(8))) < 1e-9
    finally:
        ed.ed_sector_destroy(sec)
