"""Continued-fraction G(i w_n) on the GPU vs the oracle's continued fraction from
the same states and depth (|G - G_ref| <= 1e-8 on every frequency), and the
oracle's Lehmann sum where the CF is complete."""
import numpy as np
import pytest

import workloads as W
from oracle import sector as osec, greens as og, fock
from tests._gpu import ensure_built, torch_cuda, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    ed = ensure_built()
    ctx = ed.ed_ctx_create(0)
    yield ed, ctx, torch
    ed.ed_ctx_destroy(ctx)


@pytest.mark.parametrize("spin", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_c0_ground_state_gf(env, spin, prec):
    ed, ctx, torch = env
    m = W.aim(6, seed=0)
    H = osec.build_csr(m, 3, 3)
    w, v = np.linalg.eigh(H.toarray())
    states = [(3, 3, w[0], v[:, 0])]
    beta, nw, depth = 40.0, 1024, 60
    ref = og.greens_cf(m, states, beta, nw, m.orb0, spin, depth=depth)
    dv = to_dev(v[:, 0], prec, ed, torch)
    G = ed.ed_greens_cf(ctx, m, prec, [(3, 3, w[0], dv)], beta, nw, orbital=m.orb0, spin=spin, depth=depth)
    assert np.max(np.abs(G - ref)) <= 1e-8, np.max(np.abs(G - ref))
    assert np.all(G.imag < 0)


def test_thermal_mix_and_cutoff(env):
    """Several states from several sectors, Boltzmann weights, a cutoff that drops some."""
    ed, ctx, torch = env
    m = W.kanamori(6, seed=7, n_orb=2)
    states, dstates = [], []
    for nu, nd in ((3, 3), (3, 2), (2, 3), (4, 3)):
        H = osec.build_csr(m, nu, nd)
        w, v = np.linalg.eigh(H.toarray())
        for i in range(2):
            states.append((nu, nd, w[i], v[:, i]))
            dstates.append((nu, nd, w[i], to_dev(v[:, i], "fp64", ed, torch)))
    beta, nw, depth = 8.0, 256, 80
    for cut in (0.0, 1e-3):
        ref = og.greens_cf(m, states, beta, nw, m.orb0 + 1, 0, depth=depth, boltz_cut=cut)
        G = ed.ed_greens_cf(ctx, m, "fp64", dstates, beta, nw, orbital=m.orb0 + 1, spin=0, depth=depth,
                            boltz_cut=cut)
        assert np.max(np.abs(G - ref)) <= 1e-8


def test_complete_cf_equals_lehmann(env):
    """All eigenstates of every sector, CF deeper than any Krylov space: Eq. 3."""
    ed, ctx, torch = env
    m = W.aim(4, seed=11, U=2.5)
    beta, nw = 5.0, 32
    dstates = []
    for nu in range(5):
        for nd in range(5):
            H = osec.build_csr(m, nu, nd)
            w, v = np.linalg.eigh(H.toarray())
            for i in range(len(w)):
                dstates.append((nu, nd, w[i], to_dev(v[:, i], "fp64", ed, torch)))
    G = ed.ed_greens_cf(ctx, m, "fp64", dstates, beta, nw, 0, 0, depth=40, boltz_cut=0.0)
    ref = og.lehmann(m, beta, nw, 0, fock.UP)
    assert np.max(np.abs(G - ref)) <= 1e-9, np.max(np.abs(G - ref))
