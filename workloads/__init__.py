"""Seeded synthetic model parameters and vectors for the impurity Hamiltonians.

This module only draws random numbers and lays the drawn parameters out as the
one-body matrix ``T`` and the interaction constants of a ``Model``.  It holds no
part of the Hamiltonian-vector product, the eigensolver or the Green's function:
both the CUDA library's Python binding and the CPU oracle consume the same
``Model`` objects, so both sides see bit-identical doubles.

Model (all energies in the same unit):

    H = sum_{ij,s} T_ij c+_is c_js + sum_i U_i n_iu n_id
      + sum_{m<m'<M, s s'} (Up - J delta_ss') n_ms n_m's'
      - sum_{m != m' < M} [ Jsf d+_mu d_md d+_m'd d_m'u + Jph d+_mu d+_md d_m'u d_m'd ]

which covers the Hubbard cluster of Eq. 1 (T = -t, U_i = U), the single-orbital
Anderson impurity of Eq. 2 (star-shaped T, U on the impurity only) and the
three-orbital Kanamori impurity of the Sec. 4 Hamiltonian (Jsf = Jph = J').

Site conventions: site i is bit i of a spin string.  By default the impurity
orbitals are the highest sites (orb0 = n_s - M .. n_s - 1) and the bath sites
0 .. n_s - M - 1 are grouped by the orbital they couple to; ``imp_first=True``
puts the impurity on sites 0..M-1 instead.  With the impurity on the high bits,
ascending numeric order of the spin strings lists them grouped by impurity
occupation.  The chemical potential shifts impurity levels only (Sec. 4 writes
eps_m - mu for d levels and bare eps_k for the bath).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Model", "aim", "kanamori", "two_site_hubbard", "hubbard_cluster", "atom",
    "ph_symmetric_aim", "ph_symmetric_kanamori", "random_vector", "binom",
    "sector_dim", "kanamori_half_filling_mu", "serving_stream",
]


@dataclass
class Model:
    n_s: int
    T: np.ndarray            # (n_s, n_s) float64, symmetric
    U_site: np.ndarray       # (n_s,) float64
    n_orb: int = 0           # M: sites orb0..orb0+M-1 carry Up/J/Jsf/Jph terms
    Up: float = 0.0
    J: float = 0.0
    Jsf: float = 0.0
    Jph: float = 0.0
    name: str = ""
    params: dict = field(default_factory=dict)
    orb0: int = 0            # first impurity-orbital site

    def __post_init__(self):
        self.T = np.ascontiguousarray(np.asarray(self.T, dtype=np.float64))
        self.U_site = np.ascontiguousarray(np.asarray(self.U_site, dtype=np.float64))
        assert self.T.shape == (self.n_s, self.n_s)
        assert self.U_site.shape == (self.n_s,)


def binom(n: int, k: int) -> int:
    return math.comb(n, k) if 0 <= k <= n else 0


def sector_dim(n_s: int, n_up: int, n_dn: int) -> int:
    return binom(n_s, n_up) * binom(n_s, n_dn)


def _bath_layout(n_orb: int, n_bath: int) -> list[int]:
    """Orbital index of each bath site, bath sites grouped by orbital.

    Orbital m receives n_bath // M baths, plus one more for m < n_bath % M.
    """
    counts = [n_bath // n_orb + (1 if m < n_bath % n_orb else 0) for m in range(n_orb)]
    owner = []
    for m, c in enumerate(counts):
        owner += [m] * c
    return owner


def _sites(n_s: int, n_orb: int, imp_first: bool):
    """(impurity sites, bath sites) for the two layouts."""
    if imp_first:
        return list(range(n_orb)), list(range(n_orb, n_s))
    return list(range(n_s - n_orb, n_s)), list(range(n_s - n_orb))


def aim(n_s: int = 6, seed: int = 0, U: float = 4.0, eps_d: float = 0.0, mu: float = 0.0,
        eps_range=(-2.0, 2.0), v_range=(0.1, 0.5), imp_first: bool = False) -> Model:
    """Single-orbital Anderson impurity (Eq. 2) with n_s - 1 bath levels.

    Draw order: eps_k for bath 0..N_b-1, then V_k in the same order.
    """
    rng = np.random.default_rng(seed)
    nb = n_s - 1
    eps = rng.uniform(eps_range[0], eps_range[1], nb)
    V = rng.uniform(v_range[0], v_range[1], nb)
    imp, bath = _sites(n_s, 1, imp_first)
    d = imp[0]
    T = np.zeros((n_s, n_s))
    T[d, d] = eps_d - mu
    for k in range(nb):
        s = bath[k]
        T[s, s] = eps[k]
        T[d, s] = T[s, d] = V[k]
    Us = np.zeros(n_s)
    Us[d] = U
    return Model(n_s, T, Us, n_orb=1, name=f"aim{n_s}", orb0=d,
                 params=dict(kind="aim", seed=seed, U=U, eps_d=eps_d, mu=mu, imp_first=imp_first,
                             eps_range=list(eps_range), v_range=list(v_range)))


def aim_bath(eps_d: float, U: float, eps, V, imp_first: bool = False) -> Model:
    """Single-orbital Anderson impurity (Eq. 2) with the given bath levels eps_k
    and hybridisations V_k (a DMFT iteration's bath); eps_d is the impurity
    level including any chemical potential."""
    eps = np.asarray(eps, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    nb = len(eps)
    n_s = nb + 1
    imp, bath = _sites(n_s, 1, imp_first)
    d = imp[0]
    T = np.zeros((n_s, n_s))
    T[d, d] = eps_d
    for k in range(nb):
        s = bath[k]
        T[s, s] = eps[k]
        T[d, s] = T[s, d] = V[k]
    Us = np.zeros(n_s)
    Us[d] = U
    return Model(n_s, T, Us, n_orb=1, name=f"aim_bath{n_s}", orb0=d,
                 params=dict(kind="aim_bath", U=U, eps_d=eps_d, eps=eps.tolist(), V=V.tolist(),
                             imp_first=imp_first))


def square_lattice_energies(t: float = 0.5, n_k: int = 256):
    """Band energies e(k) = -2t (cos kx + cos ky) of the square lattice with
    nearest-neighbour hopping t (the Sec. 3.2 test model) on an n_k x n_k grid
    of the Brillouin zone, as distinct values with their weights (summing to 1)."""
    k = 2.0 * np.pi * (np.arange(n_k) + 0.5) / n_k
    c = np.cos(k)
    e = (-2.0 * t * (c[:, None] + c[None, :])).ravel()
    e = np.round(e, 14)
    vals, counts = np.unique(e, return_counts=True)
    return vals, counts / float(n_k * n_k)


def dmft_initial_bath(n_bath: int, half_width: float = 1.0, v: float = 0.3):
    """Starting bath of a DMFT loop: levels spread evenly over [-w, w], equal V."""
    eps = np.linspace(-half_width, half_width, n_bath) if n_bath > 1 else np.zeros(1)
    return eps, np.full(n_bath, v)


def kanamori_half_filling_mu(U: float, Up: float, J: float, n_orb: int) -> float:
    """mu placing the isolated Kanamori atom (eps_m = 0) at its particle-hole point."""
    return (U + (n_orb - 1) * (2.0 * Up - J)) / 2.0


def kanamori(n_s: int = 12, seed: int = 0, n_orb: int = 3, U: float = 2.3, J: float = 0.4,
             Up: float | None = None, Jp: float | None = None, eps_m: float = 0.0,
             mu: float | None = None, eps_range=(-1.5, 1.5), v_range=(0.1, 0.4),
             spin_flip: bool = True, pair_hop: bool = True, imp_first: bool = False) -> Model:
    """Multi-orbital Kanamori impurity of the Sec. 4 Hamiltonian with random baths.

    Defaults: U' = U - 2J, J' = J, eps_m = 0, mu at the atom's half-filling point.
    Draw order: eps_k for bath 0..N_b-1 (site order), then V_k in the same order.
    """
    if Up is None:
        Up = U - 2.0 * J
    if Jp is None:
        Jp = J
    if mu is None:
        mu = kanamori_half_filling_mu(U, Up, J, n_orb)
    rng = np.random.default_rng(seed)
    nb = n_s - n_orb
    owner = _bath_layout(n_orb, nb)
    eps = rng.uniform(eps_range[0], eps_range[1], nb)
    V = rng.uniform(v_range[0], v_range[1], nb)
    imp, bath = _sites(n_s, n_orb, imp_first)
    T = np.zeros((n_s, n_s))
    for m in range(n_orb):
        T[imp[m], imp[m]] = eps_m - mu
    for k in range(nb):
        s = bath[k]
        T[s, s] = eps[k]
        T[imp[owner[k]], s] = T[s, imp[owner[k]]] = V[k]
    Us = np.zeros(n_s)
    Us[imp] = U
    return Model(n_s, T, Us, n_orb=n_orb, Up=Up, J=J,
                 Jsf=Jp if spin_flip else 0.0, Jph=Jp if pair_hop else 0.0,
                 name=f"kanamori{n_orb}o{n_s}s", orb0=imp[0],
                 params=dict(kind="kanamori", seed=seed, n_orb=n_orb, U=U, J=J, Up=Up, Jp=Jp,
                             eps_m=eps_m, mu=mu, eps_range=list(eps_range), imp_first=imp_first,
                             v_range=list(v_range), spin_flip=spin_flip, pair_hop=pair_hop))


def two_site_hubbard(t: float = 1.0, U: float = 4.0) -> Model:
    """Eq. 1 on two sites: T_01 = T_10 = -t, U on both sites."""
    T = np.array([[0.0, -t], [-t, 0.0]])
    return Model(2, T, np.array([U, U]), n_orb=0, name="hubbard2",
                 params=dict(kind="hubbard", t=t, U=U))


def hubbard_cluster(n_s: int, t: float = 1.0, U: float = 4.0, periodic: bool = True,
                    tp: float = 0.0) -> Model:
    """Eq. 1 on a ring of n_s sites (nearest neighbour -t, next-nearest -tp)."""
    T = np.zeros((n_s, n_s))
    for i in range(n_s):
        for d, tt in ((1, t), (2, tp)):
            j = i + d
            if j >= n_s:
                if not periodic:
                    continue
                j -= n_s
            if tt != 0.0 and j != i:
                T[i, j] = T[j, i] = -tt
    return Model(n_s, T, np.full(n_s, U), n_orb=0, name=f"hubbard{n_s}",
                 params=dict(kind="hubbard", t=t, tp=tp, U=U, periodic=periodic))


def atom(n_orb: int = 3, U: float = 2.3, J: float = 0.4, Up: float | None = None,
         Jp: float | None = None, eps_m: float = 0.0) -> Model:
    """Isolated Kanamori atom (t = V = 0): n_s = n_orb, no bath."""
    if Up is None:
        Up = U - 2.0 * J
    if Jp is None:
        Jp = J
    T = np.diag(np.full(n_orb, eps_m))
    return Model(n_orb, T, np.full(n_orb, U), n_orb=n_orb, Up=Up, J=J, Jsf=Jp, Jph=Jp,
                 name=f"atom{n_orb}", params=dict(kind="atom", U=U, J=J, Up=Up, Jp=Jp))


def ph_symmetric_aim(n_s: int = 5, U: float = 3.0, seed: int = 0) -> Model:
    """Eq. 2 with a particle-hole symmetric bath (levels in +-a pairs plus a zero level
    when n_s - 1 is odd, equal V for each pair) and eps_d = -U/2."""
    rng = np.random.default_rng(seed)
    nb = n_s - 1
    npair = nb // 2
    a = rng.uniform(0.2, 2.0, npair)
    v = rng.uniform(0.1, 0.6, npair)
    levels, hyb = [], []
    for p in range(npair):
        levels += [a[p], -a[p]]
        hyb += [v[p], v[p]]
    if nb % 2:
        levels.append(0.0)
        hyb.append(rng.uniform(0.1, 0.6))
    T = np.zeros((n_s, n_s))
    T[0, 0] = -U / 2.0
    for k in range(nb):
        T[1 + k, 1 + k] = levels[k]
        T[0, 1 + k] = T[1 + k, 0] = hyb[k]
    Us = np.zeros(n_s)
    Us[0] = U
    return Model(n_s, T, Us, n_orb=1, name=f"phaim{n_s}", params=dict(kind="ph_aim", U=U, seed=seed))


def ph_symmetric_kanamori(n_orb: int = 2, baths_per_orb: int = 2, U: float = 2.3, J: float = 0.4,
                          seed: int = 0) -> Model:
    """Kanamori impurity with +-a symmetric baths per orbital and
    eps_m - mu = -[U + (M-1)(2U' - J)]/2 (the particle-hole symmetric point)."""
    assert baths_per_orb % 2 == 0
    rng = np.random.default_rng(seed)
    Up = U - 2.0 * J
    n_s = n_orb * (1 + baths_per_orb)
    T = np.zeros((n_s, n_s))
    shift = -kanamori_half_filling_mu(U, Up, J, n_orb)
    for m in range(n_orb):
        T[m, m] = shift
    s = n_orb
    for m in range(n_orb):
        for _ in range(baths_per_orb // 2):
            a = rng.uniform(0.2, 1.5)
            v = rng.uniform(0.1, 0.5)
            for lev in (a, -a):
                T[s, s] = lev
                T[m, s] = T[s, m] = v
                s += 1
    Us = np.zeros(n_s)
    Us[:n_orb] = U
    return Model(n_s, T, Us, n_orb=n_orb, Up=Up, J=J, Jsf=J, Jph=J, name="phkan",
                 params=dict(kind="ph_kanamori", U=U, J=J, seed=seed))


def random_vector(dim: int, seed: int = 1) -> np.ndarray:
    """Seeded N(0,1) float64 vector."""
    return np.random.default_rng(seed).standard_normal(dim)


def serving_stream(n_requests: int = 200, seed: int = 0, rate: float = 1.0,
                   ns_range=(10, 16)) -> list[dict]:
    """Poisson arrival stream of impurity-solve requests: N_s ~ U{ns_range}, seeded baths.

    Each request: arrival time (in units of 1/rate), N_s, model seed, sector
    (ceil(N_s/2), floor(N_s/2)).
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    ns = rng.integers(ns_range[0], ns_range[1] + 1, n_requests)
    out = []
    for i in range(n_requests):
        n = int(ns[i])
        out.append(dict(id=i, t_arrive=float(t[i]), n_s=n, model_seed=1000 + i,
                        n_up=(n + 1) // 2, n_dn=n // 2))
    return out
