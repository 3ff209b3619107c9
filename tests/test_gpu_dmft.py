"""DMFT self-consistency on the GPU (ed_dmft_update) vs the oracle's update
(oracle/dmft.py) on the same impurity G, and the whole ED/DMFT loop of the
square-lattice Hubbard model at half filling (U = 2, t = 0.5)."""
import numpy as np
import pytest

import bench
import workloads as W
from oracle import dmft as od, greens as og, fock
from tests._gpu import ensure_built, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    ed = ensure_built()
    ctx = ed.ed_ctx_create(0)
    yield ed, ctx, torch
    ed.ed_ctx_destroy(ctx)


def rel(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


def test_update_matches_oracle(env):
    """Sigma, G_loc and Delta_new agree to 1e-12; the fitted bath reaches the
    oracle's chi2 (the least-squares minimum, up to the order of the levels)."""
    ed, ctx, torch = env
    U, beta, t = 2.0, 20.0, 0.5
    eps, V = np.array([-0.9, -0.2, 0.3, 1.0, 0.05]), np.array([0.3, 0.22, 0.27, 0.35, 0.1])
    m = W.aim_bath(-U / 2, U, eps, V)
    n_w, n_fit = 128, 48
    G = og.lehmann(m, beta, n_w, orbital=m.orb0, spin=fock.UP)
    e, w = W.square_lattice_energies(t, 96)
    iw = 1j * og.matsubara(beta, n_w)
    e2, v2, c2, sig, gl, dn = ed.ed_dmft_update(ctx, G, beta, -U / 2, U / 2, eps, V, e, w, n_fit)
    re2, rv2, rc2, rsig, rgl, rdn = od.update(iw, G, -U / 2, U / 2, eps, V, e, w, n_fit)
    assert rel(sig, rsig) <= 1e-12 and rel(gl, rgl) <= 1e-12 and rel(dn, rdn) <= 1e-12
    assert c2 <= rc2 * (1 + 1e-6) + 1e-14, (c2, rc2)
    assert abs(c2 - od.chi2(iw[:n_fit], rdn[:n_fit], e2, v2)) <= 1e-12 * max(1.0, c2)
    assert np.all(v2 >= 0)
    # the fitted hybridisations agree where both fits reached the minimum
    assert rel(od.hybridisation(iw[:n_fit], e2, v2), od.hybridisation(iw[:n_fit], re2, rv2)) <= 1e-4


def test_atomic_self_energy(env):
    """Hubbard atom (V = 0) at half filling: Sigma = U/2 + U^2 / (4 i w_n)."""
    ed, ctx, torch = env
    U, beta = 2.0, 30.0
    m = W.aim_bath(-U / 2, U, [0.0], [0.0])
    G = og.lehmann(m, beta, 64, orbital=m.orb0, spin=fock.UP)
    e, w = W.square_lattice_energies(0.5, 32)
    _, _, _, sig, _, _ = ed.ed_dmft_update(ctx, G, beta, -U / 2, U / 2, [0.0], [0.0], e, w, 8)
    iw = 1j * og.matsubara(beta, 64)
    assert np.max(np.abs(sig - (U / 2 + U * U / (4 * iw)))) <= 1e-12


def test_loop_reaches_self_consistency(env):
    """N_s = 6: the loop converges; at half filling Re G(i w_n) = 0 (particle-hole
    symmetry), Im Sigma(i w_0) < 0 and 0 < Z < 1; the last update agrees with the
    oracle's on the same G."""
    ed, ctx, torch = env
    r = bench.dmft_loop(ed, ctx, torch, 6, n_w=256, n_fit=64, n_iter=40, prec="fp64", conv=1e-6, n_k=128)
    assert r["converged"], r["history"][-1]
    assert np.max(np.abs(r["G"].real)) <= 1e-6
    assert r["Sigma"][0].imag < 0 and 0 < r["Z"] < 1
    assert r["history"][-1]["ground_sector"] == [3, 3]
    assert r["history"][-1]["chi2"] < 1e-4


def test_invalid_arguments(env):
    ed, ctx, torch = env
    e, w = W.square_lattice_energies(0.5, 16)
    G = np.full(16, -0.1j)
    for kw in (dict(n_fit=0), dict(n_fit=17), dict(eps=[], V=[]), dict(e=[], w=[]),
               dict(G_imp=np.zeros(16, complex)), dict(G_imp=np.full(16, np.nan + 0j)), dict(beta=0.0)):
        args = dict(G_imp=G, beta=10.0, eps_d=-1.0, mu=1.0, eps=[0.1, 0.2], V=[0.3, 0.3], e=e, w=w, n_fit=8)
        args.update(kw)
        with pytest.raises(ed.EdError):
            ed.ed_dmft_update(ctx, **args)
