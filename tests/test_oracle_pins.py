"""Pins of the CPU oracle against facts fixed outside it (closed forms, invariants,
the paper's worked CSR example and sector sizes).  CPU only.

Each ``check_*`` raises AssertionError on failure; the planted-mistake tests at
the end re-run them against deliberately broken copies of oracle pieces to show
that every pin catches a plausible mistake.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import fock, sector, spectrum, greens

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def sector_eigs(model, nu, nd):
    H = sector.build_csr(model, nu, nd)
    return np.linalg.eigvalsh(H.toarray())


# ----------------------------------------------------------------- closed forms
def check_two_site_hubbard():
    """Eq. 1 on two sites, sector (1,1): E0 = (U - sqrt(U^2 + 16 t^2)) / 2."""
    for t, U in ((1.0, 4.0), (0.5, 2.0), (1.3, 0.7), (1.0, 0.0)):
        m = W.two_site_hubbard(t, U)
        e = sector_eigs(m, 1, 1)
        ref = (U - math.sqrt(U * U + 16 * t * t)) / 2
        assert abs(e[0] - ref) < 1e-13, (t, U, e[0], ref)


def check_u0_ground_energy():
    """Non-interacting limit: E0(N_up, N_dn) = lowest N_up + lowest N_dn levels of T."""
    models = [W.aim(6, seed=3, U=0.0), W.hubbard_cluster(6, t=1.0, U=0.0, tp=0.3),
              W.kanamori(6, seed=1, n_orb=2, U=0.0, J=0.0)]
    for m in models:
        lam = np.linalg.eigvalsh(m.T)
        for nu, nd in ((3, 3), (2, 4), (1, 5), (4, 4), (2, 2)):
            e0 = sector_eigs(m, nu, nd)[0]
            ref = lam[:nu].sum() + lam[:nd].sum()
            assert abs(e0 - ref) < 1e-12, (m.name, nu, nd, e0, ref)


def check_u0_greens():
    """Non-interacting limit: G(i w_n) = [(i w_n - T)^-1]_00 at any beta (Lehmann over all sectors)."""
    m = W.aim(4, seed=5, U=0.0)
    beta, nw = 7.0, 16
    G = greens.lehmann(m, beta, nw, orbital=0, spin=fock.UP)
    wn = greens.matsubara(beta, nw)
    ref = np.array([np.linalg.inv(1j * w * np.eye(4) - m.T)[0, 0] for w in wn])
    assert np.max(np.abs(G - ref)) < 1e-12, np.max(np.abs(G - ref))


def check_u0_greens_real_axis():
    """Non-interacting limit off the real axis: G(w + i eta) = [((w + i eta) - T)^-1]_00
    (Lehmann over all sectors), and G(z*) = G(z)* for a real Hamiltonian."""
    m = W.aim(4, seed=6, U=0.0)
    z = np.linspace(-3.0, 3.0, 41) + 0.05j
    G = greens.lehmann(m, 9.0, 0, orbital=0, spin=fock.UP, z=z)
    ref = np.array([np.linalg.inv(zz * np.eye(4) - m.T)[0, 0] for zz in z])
    assert np.max(np.abs(G - ref)) < 1e-12, np.max(np.abs(G - ref))
    Gc = greens.lehmann(m, 9.0, 0, orbital=0, spin=fock.UP, z=np.conj(z))
    assert np.max(np.abs(Gc - np.conj(G))) < 1e-12


def check_spectral_sum_rule():
    """A(w) = -Im G(w + i eta) / pi is non-negative and integrates to <{c, c+}> = 1
    (each pole is a Lorentzian of unit total weight; the tails beyond |w| = W
    carry about 2 eta / (pi W) of it)."""
    m = W.aim(4, seed=2, U=2.0)
    eta, Wd = 0.05, 400.0
    w = np.linspace(-Wd, Wd, 160001)
    G = greens.lehmann(m, 10.0, 0, orbital=0, spin=fock.UP, z=w + 1j * eta)
    A = greens.spectral(G)
    assert A.min() > 0.0
    tot = np.trapezoid(A, w) if hasattr(np, "trapezoid") else np.trapz(A, w)
    assert abs(tot - (1.0 - 2 * eta / (np.pi * Wd))) < 2e-4, tot


def check_cf_vs_lehmann_real_axis():
    """CF over all eigenstates at full depth == Lehmann at z = w + i eta (interacting AIM)."""
    m = W.aim(4, seed=11, U=2.5)
    beta = 5.0
    states = []
    for nu in range(5):
        for nd in range(5):
            H = sector.build_csr(m, nu, nd).toarray()
            w, v = np.linalg.eigh(H)
            states += [(nu, nd, w[i], v[:, i]) for i in range(len(w))]
    z = np.linspace(-4.0, 4.0, 33) + 0.1j
    Gcf = greens.greens_cf(m, states, beta, 0, 0, fock.UP, depth=64, boltz_cut=0.0, reorth=True, z=z)
    Gl = greens.lehmann(m, beta, 0, 0, fock.UP, z=z)
    assert np.max(np.abs(Gcf - Gl)) < 1e-10, np.max(np.abs(Gcf - Gl))


def check_dmft_atomic_self_energy():
    """Hubbard atom at half filling (V = 0, eps_d = -U/2): Sigma(i w) = U/2 + U^2 / (4 i w)."""
    from oracle import dmft
    U, beta = 2.0, 20.0
    m = W.aim_bath(-U / 2, U, [0.0], [0.0])
    G = greens.lehmann(m, beta, 64, orbital=m.orb0, spin=fock.UP)
    iw = 1j * greens.matsubara(beta, 64)
    sig = dmft.self_energy(iw, G, -U / 2, [0.0], [0.0])
    ref = U / 2 + U * U / (4 * iw)
    assert np.max(np.abs(sig - ref)) < 1e-12, np.max(np.abs(sig - ref))


def check_dmft_noninteracting():
    """U = 0: the impurity self-energy vanishes for any bath, and the square-lattice
    local Green's function has the band's moments: i w G -> 1, (i w)^3 (G - 1/(i w)) -> 4 t^2."""
    from oracle import dmft
    t, beta = 0.5, 30.0
    eps, V = np.array([-0.7, 0.1, 0.9]), np.array([0.3, 0.25, 0.4])
    m = W.aim_bath(0.0, 0.0, eps, V)
    G = greens.lehmann(m, beta, 40, orbital=m.orb0, spin=fock.UP)
    iw = 1j * greens.matsubara(beta, 40)
    assert np.max(np.abs(dmft.self_energy(iw, G, 0.0, eps, V))) < 1e-12
    e, w = W.square_lattice_energies(t, 128)
    assert abs(w.sum() - 1.0) < 1e-14 and abs((w * e).sum()) < 1e-14 and abs((w * e * e).sum() - 4 * t * t) < 1e-13
    z = 1j * np.array([200.0, 400.0])
    gl = dmft.lattice_gloc(z, np.zeros(2), 0.0, e, w)
    # z G = 1 + m1 / z + m2 / z^2 + ..., m1 = 0, m2 = 4 t^2
    assert np.max(np.abs(z * gl - 1.0 - 4 * t * t / z ** 2)) < 1e-8
    assert abs(((z ** 3) * (gl - 1.0 / z))[-1].real - 4 * t * t) < 1e-3


def check_dmft_lattice_moments():
    """Lattice G at chemical potential mu and a constant self-energy s: since
    1/(z + mu - s - e) = 1/z + (e - mu + s)/z^2 + ..., the band's moments
    (m1 = 0, m2 = 4 t^2) give z G = 1 + (s - mu)/z + (4 t^2 + (s - mu)^2)/z^2 + O(z^-3)."""
    from oracle import dmft
    t, mu, s = 0.5, 0.3, -0.45
    e, w = W.square_lattice_energies(t, 128)
    z = 1j * np.array([1000.0, 2000.0])  # the O(z^-3) remainder is ~3e-9 here
    for sig in (0.0, s):
        gl = dmft.lattice_gloc(z, np.full(2, sig), mu, e, w)
        a = sig - mu
        ref = 1.0 + a / z + (4 * t * t + a * a) / z ** 2
        assert np.max(np.abs(z * gl - ref)) < 2e-8, np.max(np.abs(z * gl - ref))


def check_dmft_weiss_field():
    """The Weiss field closes the loop: for any G, inserting the impurity
    self-energy of a bath and the same G as the local one gives that bath's
    hybridisation back; at U = 0 and mu = 0 the new hybridisation of the square
    lattice has first moment 4 t^2 (z Delta_new -> sum V^2 = 4 t^2)."""
    from oracle import dmft
    iw = 1j * greens.matsubara(25.0, 48)
    eps, V = np.array([-0.8, 0.2, 1.1]), np.array([0.3, 0.45, 0.2])
    G = 1.0 / (iw - 0.15 - 0.6 / iw + 0.2j)  # any G without zeros
    sig = dmft.self_energy(iw, G, 0.1, eps, V)
    back = dmft.weiss_hybridisation(iw, sig, G, 0.1)
    assert np.max(np.abs(back - dmft.hybridisation(iw, eps, V))) < 1e-12
    t = 0.5
    e, w = W.square_lattice_energies(t, 128)
    z = 1j * np.array([400.0])
    gl = dmft.lattice_gloc(z, np.zeros(1), 0.0, e, w)
    dn = dmft.weiss_hybridisation(z, np.zeros(1), gl, 0.0)
    assert abs((z * dn)[0].real - 4 * t * t) < 1e-4 and abs((z * dn)[0].imag) < 1e-6, z * dn


def check_dmft_bath_fit_recovers_bath():
    """A hybridisation made from a known bath is fitted back (chi2 ~ 0) from a perturbed start."""
    from oracle import dmft
    iw = 1j * greens.matsubara(40.0, 64)
    eps, V = np.array([-1.1, -0.3, 0.4, 1.2]), np.array([0.35, 0.2, 0.25, 0.4])
    target = dmft.hybridisation(iw, eps, V)
    e2, v2, c2 = dmft.fit_bath(iw, target, eps + 0.07 * np.array([1, -1, 1, -1]), V * 1.1)
    assert c2 < 1e-20, c2
    o = np.argsort(e2)
    assert np.max(np.abs(e2[o] - eps)) < 1e-6 and np.max(np.abs(v2[o] - V)) < 1e-6


def multiset(vals, tol=1e-9):
    vals = np.sort(np.asarray(vals))
    out = []
    for v in vals:
        if out and abs(v - out[-1][0]) < tol:
            out[-1][1] += 1
        else:
            out.append([v, 1])
    return [(round(v, 9), c) for v, c in out]


def check_t2g_multiplets(U=2.3, J=0.4):
    """Isolated t2g Kanamori atom (U' = U - 2J, J' = J): textbook multiplets.
    N=2: U-3J x9, U-J x5, U+2J x1.   N=3: 3U-9J x4, 3U-6J x10, 3U-4J x6.
    N=5: 10U-20J x6 (one hole).      N=6: 15U-30J x1 (full shell)."""
    m = W.atom(3, U=U, J=J)
    byN = {}
    for nu in range(4):
        for nd in range(4):
            byN.setdefault(nu + nd, []).extend(sector_eigs(m, nu, nd))
    exp = {
        0: [(0.0, 1)], 1: [(0.0, 6)],
        2: [(U - 3 * J, 9), (U - J, 5), (U + 2 * J, 1)],
        3: [(3 * U - 9 * J, 4), (3 * U - 6 * J, 10), (3 * U - 4 * J, 6)],
        5: [(10 * U - 20 * J, 6)], 6: [(15 * U - 30 * J, 1)],
    }
    for N, ref in exp.items():
        ref = [(round(v, 9), c) for v, c in sorted(ref)]
        assert multiset(byN[N]) == ref, (N, multiset(byN[N]), ref)


# ------------------------------------------------------------------- invariants
def check_hermitian():
    for m, nu, nd in ((W.kanamori(6, seed=2, n_orb=3), 3, 2), (W.aim(6), 3, 3),
                      (W.hubbard_cluster(5, tp=0.4), 2, 3)):
        H = sector.build_csr(m, nu, nd)
        D = (H - H.T).tocsr()
        D.eliminate_zeros()
        assert D.nnz == 0, m.name


def check_conservation_and_blocks():
    """Brute-force Fock H is block diagonal in (N_up, N_dn), and each block equals
    the sector tier's H under the sector's basis order."""
    m = W.kanamori(4, seed=7, n_orb=2, U=2.0, J=0.3)
    H = fock.fock_hamiltonian(m)
    Nu, Nd = fock.fock_numbers(4)
    r, c = np.nonzero(H)
    assert np.all(Nu[r] == Nu[c]) and np.all(Nd[r] == Nd[c])
    for nu in range(5):
        for nd in range(5):
            sec = sector.Sector(4, nu, nd)
            f = sec.states().astype(np.int64)
            blk = H[np.ix_(f, f)]
            Hs = sector.build_csr(m, nu, nd).toarray()
            assert np.array_equal(blk, Hs), (nu, nd)


def check_particle_hole():
    """Particle-hole symmetric parameters: spec(N_up, N_dn) = spec(n_s - N_up, n_s - N_dn)."""
    for m in (W.ph_symmetric_aim(5, U=3.0), W.ph_symmetric_kanamori(2, 2)):
        n = m.n_s
        for nu, nd in ((1, 2), (2, 2), (0, 3), (2, 4)):
            if nu > n or nd > n:
                continue
            a = sector_eigs(m, nu, nd)
            b = sector_eigs(m, n - nu, n - nd)
            assert np.max(np.abs(a - b)) < 1e-11, (m.name, nu, nd)


def check_spin_symmetry():
    m = W.kanamori(6, seed=4, n_orb=3)
    for nu, nd in ((2, 4), (1, 3), (2, 5)):
        a, b = sector_eigs(m, nu, nd), sector_eigs(m, nd, nu)
        assert np.max(np.abs(a - b)) < 1e-11


def check_su2_inclusion():
    """J' = J: every level of (N_up+1, N_dn-1) also appears in (N_up, N_dn), N_up >= N_dn."""
    m = W.kanamori(6, seed=9, n_orb=2)
    big = sector_eigs(m, 3, 3)
    small = sector_eigs(m, 4, 2)
    for e in small:
        assert np.min(np.abs(big - e)) < 1e-9, e


def check_cf_vs_lehmann():
    """CF over all eigenstates, full Krylov depth, no cutoff == Lehmann sum of Eq. 3."""
    m = W.aim(4, seed=11, U=2.5)
    beta, nw = 5.0, 24
    states = []
    for nu in range(5):
        for nd in range(5):
            H = sector.build_csr(m, nu, nd).toarray()
            w, v = np.linalg.eigh(H)
            states += [(nu, nd, w[i], v[:, i]) for i in range(len(w))]
    Gcf = greens.greens_cf(m, states, beta, nw, 0, fock.UP, depth=64, boltz_cut=0.0, reorth=True)
    Gl = greens.lehmann(m, beta, nw, 0, fock.UP)
    assert np.max(np.abs(Gcf - Gl)) < 1e-11, np.max(np.abs(Gcf - Gl))


def check_sum_rules():
    """n+ + n- = <{c, c+}> = 1 for every state; i w_n G(i w_n) -> 1 for large w_n."""
    m = W.aim(6, seed=0)
    H = sector.build_csr(m, 3, 3)
    w, v = np.linalg.eigh(H.toarray())
    st = [(3, 3, w[0], v[:, 0])]
    G, parts = greens.greens_cf(m, st, 40.0, 4096, 0, fock.UP, depth=80, return_parts=True)
    assert abs(parts[0][1] + parts[1][1] - 1.0) < 1e-13
    wn = greens.matsubara(40.0, 4096)
    assert abs(1j * wn[-1] * G[-1] - 1.0) < 2e-3


# ------------------------------------------------------------- paper fixtures
def check_fig1_csr():
    g = json.load(open(os.path.join(GOLD, "fig1_csr.json")))
    rng = np.random.default_rng(0)
    A = np.zeros((g["nrows"], g["nrows"]))
    for i, j in g["nonzero_positions"]:
        A[i, j] = rng.uniform(0.5, 2.0)
    ri, ci, vals = sector.csr_from_dense(A)
    assert list(ri) == g["row_ind"] and list(ci) == g["col_ind"]
    order = [(int(s[1]), int(s[2])) for s in g["value_order"]]
    assert np.array_equal(vals, np.array([A[i, j] for i, j in order]))
    v = rng.standard_normal(g["nrows"])
    assert np.allclose(sector.csr_matvec(ri, ci, vals, v), A @ v, rtol=0, atol=1e-14)


def check_sector_dims():
    g = json.load(open(os.path.join(GOLD, "sector_dims.json")))
    for c in g["cases"]:
        du = len(sector.spin_basis(c["n_s"], c["n_up"]))
        dd = len(sector.spin_basis(c["n_s"], c["n_dn"]))
        assert du * dd == c["dim"], c
    for c in g["per_spin"]:
        assert len(sector.spin_basis(c["n_s"], c["n"])) == c["count"]
    # the basis is the set of popcount-n strings in ascending order
    b = sector.spin_basis(7, 3)
    ref = sorted(sum(1 << i for i in comb) for comb in __import__("itertools").combinations(range(7), 3))
    assert list(b) == ref


def check_tiers_agree():
    """Dense eigh, ARPACK and brute force agree on the lowest levels of a 400-dim sector."""
    m = W.aim(6, seed=0)
    H = sector.build_csr(m, 3, 3)
    d = spectrum.lowest(H, 4)
    a = spectrum.lowest(H, 4, dense_limit=0)
    assert np.max(np.abs(d - a)) < 1e-10
    m4 = W.aim(4, seed=2)
    Hf = fock.fock_hamiltonian(m4)
    Nu, Nd = fock.fock_numbers(4)
    sel = np.nonzero((Nu == 2) & (Nd == 2))[0]
    bf = np.linalg.eigvalsh(Hf[np.ix_(sel, sel)])
    assert np.max(np.abs(bf - sector_eigs(m4, 2, 2))) < 1e-12


def check_row_sampling():
    m = W.kanamori(8, seed=3, n_orb=3)
    H = sector.build_csr(m, 4, 3)
    rows = np.array([0, 1, 17, 333, H.shape[0] - 1])
    ptr, cols, vals = sector.row_entries(m, 4, 3, rows)
    for k, r in enumerate(rows):
        assert np.array_equal(cols[ptr[k]:ptr[k + 1]], H.indices[H.indptr[r]:H.indptr[r + 1]])
        assert np.array_equal(vals[ptr[k]:ptr[k + 1]], H.data[H.indptr[r]:H.indptr[r + 1]])
    x = W.random_vector(H.shape[0], 1)
    assert np.allclose(sector.apply_rows(m, 4, 3, rows, x), (H @ x)[rows], rtol=1e-14, atol=1e-14)


def check_blocked_csr():
    """The row-block assembly (rows from the adjoint operator products applied to
    each row state) equals the column-wise literal build exactly, with a block
    size that leaves a ragged last block; the Green's function is unchanged
    when its neighbour sectors are built that way."""
    m = W.kanamori(8, seed=4, n_orb=3)
    for nu, nd in ((4, 3), (5, 4), (1, 0)):
        A = sector.build_csr(m, nu, nd)
        B = sector.build_csr_blocked(m, nu, nd, block=37)
        assert np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)
        assert np.array_equal(A.data, B.data)
    H = sector.build_csr(m, 4, 4)
    w, v = spectrum.lowest(H, 1, vectors=True)
    st = [(4, 4, w[0], v[:, 0])]
    G1 = greens.greens_cf(m, st, 20.0, 16, m.orb0, fock.UP, depth=40)
    G2 = greens.greens_cf(m, st, 20.0, 16, m.orb0, fock.UP, depth=40,
                          build=lambda mm, a, b: sector.build_csr_blocked(mm, a, b, block=101))
    assert np.array_equal(G1, G2)


PINS = [check_two_site_hubbard, check_u0_ground_energy, check_u0_greens, check_t2g_multiplets,
        check_hermitian, check_conservation_and_blocks, check_particle_hole, check_spin_symmetry,
        check_su2_inclusion, check_cf_vs_lehmann, check_sum_rules, check_fig1_csr,
        check_u0_greens_real_axis, check_spectral_sum_rule, check_cf_vs_lehmann_real_axis,
        check_dmft_atomic_self_energy, check_dmft_noninteracting, check_dmft_bath_fit_recovers_bath,
        check_dmft_lattice_moments, check_dmft_weiss_field,
        check_sector_dims, check_tiers_agree, check_row_sampling, check_blocked_csr]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


# ---------------------------------------------------------- planted mistakes
def _fails(pin):
    try:
        pin()
    except AssertionError:
        return True
    return False


def test_mistake_no_jordan_wigner_sign(monkeypatch):
    def apply_op_nosign(states, amps, md, dagger):
        bit = np.uint64(1) << np.uint64(md)
        occ = (states & bit) != 0
        ok = ~occ if dagger else occ
        return states ^ bit, np.where(ok, amps, 0.0)
    monkeypatch.setattr(fock, "apply_op", apply_op_nosign)
    assert _fails(check_u0_ground_energy)


def _patched_terms(transform):
    orig = fock.hamiltonian_terms

    def terms(model):
        return transform(model, orig(model))
    return terms


def test_mistake_spin_flip_sign(monkeypatch):
    def flip(model, terms):
        out = []
        for c, ops in terms:
            # spin-flip products: creation, annihilation, creation, annihilation
            if len(ops) == 4 and [d for _, d in ops] == [True, False, True, False] and ops[0][0] != ops[1][0]:
                c = -c
            out.append((c, ops))
        return out
    monkeypatch.setattr(fock, "hamiltonian_terms", _patched_terms(flip))
    assert _fails(check_t2g_multiplets)


def test_mistake_dropped_pair_hop(monkeypatch):
    def drop(model, terms):
        return [(c, ops) for c, ops in terms if [d for _, d in ops] != [True, True, False, False]]
    monkeypatch.setattr(fock, "hamiltonian_terms", _patched_terms(drop))
    assert _fails(check_t2g_multiplets)


def test_mistake_hund_sign(monkeypatch):
    def wrong(model, terms):
        n = model.n_s
        out = []
        for c, ops in terms:
            if len(ops) == 4 and [d for _, d in ops] == [True, False, True, False] and ops[0][0] == ops[1][0]:
                a, b = ops[0][0], ops[2][0]
                same_spin = (a < n) == (b < n)
                if same_spin and a % n != b % n:
                    c = model.Up + model.J
            out.append((c, ops))
        return out
    monkeypatch.setattr(fock, "hamiltonian_terms", _patched_terms(wrong))
    assert _fails(check_t2g_multiplets)


def test_mistake_hopping_dropped_for_down_spin(monkeypatch):
    def drop(model, terms):
        n = model.n_s
        return [(c, ops) for c, ops in terms
                if not (len(ops) == 2 and ops[0][0] >= n and ops[0][0] != ops[1][0])]
    monkeypatch.setattr(fock, "hamiltonian_terms", _patched_terms(drop))
    assert _fails(check_u0_ground_energy)


def test_mistake_conjugate_lehmann_sign(monkeypatch):
    orig = greens.lehmann

    def conj(*a, **k):
        return np.conj(orig(*a, **k))
    monkeypatch.setattr(greens, "lehmann", conj)
    assert _fails(check_u0_greens)


def test_mistake_cf_hole_sign(monkeypatch):
    orig = greens.cf_eval
    calls = {"n": 0}

    def bad(z, a, b):
        # evaluate every hole fraction without the leading minus sign
        g = orig(z, a, b)
        calls["n"] += 1
        return g if np.all(np.imag(z) > 0) else -g
    monkeypatch.setattr(greens, "cf_eval", bad)
    assert _fails(check_cf_vs_lehmann)


def test_mistake_transposed_csr(monkeypatch):
    orig = sector.csr_from_dense
    monkeypatch.setattr(sector, "csr_from_dense", lambda A: orig(A.T))
    assert _fails(check_fig1_csr)


def test_mistake_rank_off_by_one(monkeypatch):
    orig = sector.spin_basis
    monkeypatch.setattr(sector, "spin_basis", lambda n_s, n: orig(n_s, n)[::-1].copy())
    assert _fails(check_sector_dims)


def test_mistake_dmft_self_energy_sign(monkeypatch):
    from oracle import dmft

    def wrong(z, G_imp, eps_d, eps, V):
        z = np.asarray(z, dtype=complex)
        return z - eps_d - dmft.hybridisation(z, eps, V) + 1.0 / np.asarray(G_imp)
    monkeypatch.setattr(dmft, "self_energy", wrong)
    assert _fails(check_dmft_atomic_self_energy)


def test_mistake_dmft_dropped_hybridisation(monkeypatch):
    from oracle import dmft

    def wrong(z, G_imp, eps_d, eps, V):
        return np.asarray(z, dtype=complex) - eps_d - 1.0 / np.asarray(G_imp)
    monkeypatch.setattr(dmft, "self_energy", wrong)
    assert _fails(check_dmft_noninteracting)


def test_mistake_dmft_mu_sign(monkeypatch):
    from oracle import dmft
    orig = dmft.lattice_gloc
    monkeypatch.setattr(dmft, "lattice_gloc", lambda z, sigma, mu, e, w: orig(z, sigma, -mu, e, w))
    assert _fails(check_dmft_lattice_moments)


def test_mistake_dmft_weiss_sigma_sign(monkeypatch):
    from oracle import dmft

    def wrong(z, sigma, G_loc, eps_d):
        return np.asarray(z, dtype=complex) - eps_d + np.asarray(sigma) - 1.0 / np.asarray(G_loc)
    monkeypatch.setattr(dmft, "weiss_hybridisation", wrong)
    assert _fails(check_dmft_weiss_field)
