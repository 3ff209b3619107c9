"""Sector tables built by the CUDA library vs the oracle, bit-exact: basis strings
(ascending), hop targets (ranks), fermion signs and hop values; stored CSR
column indices and off-diagonal values."""
import numpy as np
import pytest

import workloads as W
from oracle import sector as osec
from tests._gpu import ensure_built, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    ed = ensure_built()
    ctx = ed.ed_ctx_create(0)
    yield ed, ctx, torch
    ed.ed_ctx_destroy(ctx)


def oracle_spin_hops(model, n, spin):
    """One spin's hop table from the oracle's sector H with the other spin empty."""
    H = osec.build_csr(model, n, 0) if spin == 0 else osec.build_csr(model, 0, n)
    ptr = [0]
    tgt, val = [], []
    for r in range(H.shape[0]):
        cols = H.indices[H.indptr[r]:H.indptr[r + 1]]
        vals = H.data[H.indptr[r]:H.indptr[r + 1]]
        keep = cols != r
        tgt += list(cols[keep])
        val += list(vals[keep])
        ptr.append(len(tgt))
    return np.array(ptr), np.array(tgt, dtype=np.int64), np.array(val)


CASES = [
    ("C0 AIM N_s=6", lambda: W.aim(6, seed=0), 3, 3),
    ("Kanamori N_s=8", lambda: W.kanamori(8, seed=1), 4, 3),
    ("Hubbard ring N_s=10", lambda: W.hubbard_cluster(10, tp=0.3), 5, 4),
    ("C1 Kanamori N_s=12", lambda: W.kanamori(12, seed=0), 6, 6),
    ("C3 Kanamori N_s=15", lambda: W.kanamori(15, seed=0), 7, 8),
]


@pytest.mark.parametrize("name,mk,nu,nd", CASES, ids=[c[0] for c in CASES])
def test_basis_and_hops_bit_exact(env, name, mk, nu, nd):
    ed, ctx, torch = env
    m = mk()
    sec = ed.ed_sector_create(ctx, m, nu, nd, "fp64")
    try:
        info = ed.ed_sector_get_info(sec)
        for spin, n in ((0, nu), (1, nd)):
            b = ed.ed_sector_basis(sec, spin)
            ref = osec.spin_basis(m.n_s, n)
            assert np.array_equal(b.astype(np.uint64), ref)
            ptr, tgt, val = ed.ed_sector_hops(sec, spin)
            rp, rt, rv = oracle_spin_hops(m, n, spin)
            assert np.array_equal(ptr.astype(np.int64), rp)
            assert np.array_equal(tgt.astype(np.int64), rt)
            assert np.array_equal(val, rv)          # T_ij * sign, bit for bit
        assert info.dim == len(osec.spin_basis(m.n_s, nu)) * len(osec.spin_basis(m.n_s, nd))
    finally:
        ed.ed_sector_destroy(sec)


CSR_CASES = [
    ("C0 AIM N_s=6", lambda: W.aim(6, seed=0), 3, 3),
    ("Kanamori N_s=8", lambda: W.kanamori(8, seed=1), 4, 3),
    ("Kanamori M=2 N_s=7", lambda: W.kanamori(7, seed=5, n_orb=2), 3, 4),
    ("Hubbard ring N_s=10", lambda: W.hubbard_cluster(10, tp=0.3), 5, 4),
    ("atom t2g", lambda: W.atom(3), 2, 1),
    ("empty up spin", lambda: W.kanamori(8, seed=2), 0, 3),
    ("full down spin", lambda: W.kanamori(8, seed=2), 3, 8),
]


@pytest.mark.parametrize("name,mk,nu,nd", CSR_CASES, ids=[c[0] for c in CSR_CASES])
def test_stored_csr_matches_oracle(env, name, mk, nu, nd):
    ed, ctx, torch = env
    m = mk()
    sec = ed.ed_sector_create(ctx, m, nu, nd, "fp64", ed.ED_SECTOR_CSR)
    try:
        H = osec.build_csr(m, nu, nd)
        rp, cols, vals = ed.ed_sector_csr_rows(sec, 0, H.shape[0])
        assert np.array_equal(rp, H.indptr.astype(np.int64))
        assert np.array_equal(cols, H.indices.astype(np.int64))
        rows = np.repeat(np.arange(H.shape[0]), np.diff(H.indptr))
        off = cols != rows
        assert np.array_equal(vals[off], H.data[off])          # hops, spin-flip, pair-hop: exact
        scale = max(1.0, np.abs(H.data[~off]).max())
        assert np.max(np.abs(vals[~off] - H.data[~off])) <= 1e-14 * scale   # diagonal sums
    finally:
        ed.ed_sector_destroy(sec)


def test_sector_argument_errors(env):
    ed, ctx, torch = env
    m = W.aim(6)
    for nu, nd in ((-1, 2), (7, 1), (2, 9)):
        with pytest.raises(ed.EdError) as e:
            ed.ed_sector_create(ctx, m, nu, nd)
        assert e.value.status == ed.ED_ERR_INVALID
    bad = W.aim(6)
    bad.T[0, 1] += 1e-3          # not symmetric
    with pytest.raises(ed.EdError):
        ed.ed_sector_create(ctx, bad, 3, 3)
    with pytest.raises(ed.EdError):
        ed.ed_sector_create(ctx, m, 3, 3, "df64", ed.ED_SECTOR_CSR)   # CSR is FP64 only
    small = ed.ed_ctx_create(0, hbm_budget=1 << 20)
    try:
        with pytest.raises(ed.EdError) as e:
            ed.ed_sector_create(small, W.kanamori(12), 6, 6, "fp64", ed.ED_SECTOR_CSR)
        assert e.value.status == ed.ED_ERR_OOM
        before = ed.ed_ctx_bytes_in_use(small)
        sec = ed.ed_sector_create(small, W.aim(6), 3, 3)     # still usable after the failure
        ed.ed_sector_destroy(sec)
        assert ed.ed_ctx_bytes_in_use(small) == before
    finally:
        ed.ed_ctx_destroy(small)
