"""Green's function: Lehmann sum (Eq. 3) and Lanczos continued fractions, at the
Matsubara points or at any complex frequency off the real axis (z = w + i eta
gives the real-frequency spectral function A(w) = -Im G(w + i eta) / pi that
Figs. 3 and 5 of the paper plot).

Test infrastructure (see ``oracle/__init__``).

Sign reading of Eq. 3.  The printed denominator E_nu - E_mu - i w_n is the
complex conjugate of the usual Lehmann form; this oracle uses

    G(i w_n) = (1/Z) sum_{nu,mu} |<mu| c+ |nu>|^2 (e^{-b E_nu} + e^{-b E_mu})
                                  / (i w_n + E_nu - E_mu),

so that Im G(i w_n) < 0 for w_n > 0, with w_n = (2n+1) pi / beta.

Continued fraction for a kept state |nu> with weight w_nu (Sec. 2 notes that at
large beta only the lowest states matter; Sec. 4 keeps those whose Boltzmann
factor exceeds a cutoff, 1e-5 in the paper):

    particle:  phi = c+ |nu>, n+ = <phi|phi>, Lanczos (a_i, b_i) of H from phi,
               G+(z) = n+ / (z + E_nu - a_0 - b_1^2 / (z + E_nu - a_1 - ...))
    hole:      phi = c |nu>,  n- = <phi|phi>, Lanczos (a_i, b_i) of H from phi,
               G-(z) = n- / (z - E_nu + a_0 - b_1^2 / (z - E_nu + a_1 - ...))
    G(z) = sum_nu w_nu [G+(z) + G-(z)],  w_nu = e^{-b (E_nu - E_min)} / Z.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fock
from .sector import Sector, build_csr


def matsubara(beta: float, n_w: int) -> np.ndarray:
    return (2.0 * np.arange(n_w) + 1.0) * np.pi / beta


def op_matrix(n_s: int, n_up: int, n_dn: int, orbital: int, spin: int, dagger: bool):
    """Sparse matrix of c+_{orbital,spin} (or c) from sector (n_up, n_dn) to its
    neighbour sector, by literal operator application.  Returns (matrix,
    (n_up', n_dn')), or (None, None) when the target sector is empty."""
    dn_up = (1 if dagger else -1) if spin == fock.UP else 0
    dn_dn = (1 if dagger else -1) if spin == fock.DN else 0
    tu, td = n_up + dn_up, n_dn + dn_dn
    if not (0 <= tu <= n_s and 0 <= td <= n_s):
        return None, None
    src = Sector(n_s, n_up, n_dn)
    dst = Sector(n_s, tu, td)
    f = src.states()
    tgt, amp = fock.apply_term(f, [(fock.mode(orbital, spin, n_s), dagger)], 1.0)
    nz = amp != 0.0
    rows = dst.index(tgt[nz])
    cols = np.arange(src.dim)[nz]
    C = sp.csr_matrix((amp[nz], (rows, cols)), shape=(dst.dim, src.dim))
    return C, (tu, td)


def lehmann(model, beta: float, n_w: int, orbital: int = 0, spin: int = fock.UP,
            sectors=None, z=None) -> np.ndarray:
    """Eq. 3 (standard sign) summed over all eigenstates of the given sectors
    (default: every sector) by full diagonalisation, at z = i w_n (n < n_w) or,
    if given, at the complex frequencies z (n_w is then ignored)."""
    n = model.n_s
    if sectors is None:
        sectors = [(a, b) for a in range(n + 1) for b in range(n + 1)]
    eig = {}
    for (a, b) in sectors:
        H = build_csr(model, a, b)
        w, v = np.linalg.eigh(H.toarray())
        eig[(a, b)] = (w, v)
    E0 = min(w.min() for w, _ in eig.values())
    Z = sum(np.exp(-beta * (w - E0)).sum() for w, _ in eig.values())
    iw = 1j * matsubara(beta, n_w) if z is None else np.asarray(z, dtype=complex)
    G = np.zeros(len(iw), dtype=complex)
    for (a, b), (w_nu, v_nu) in eig.items():
        C, tgt = op_matrix(n, a, b, orbital, spin, True)
        if C is None or tgt not in eig:
            continue
        w_mu, v_mu = eig[tgt]
        M = v_mu.T @ (C @ v_nu)            # <mu| c+ |nu>
        M2 = M * M
        fac = np.exp(-beta * (w_nu - E0))[None, :] + np.exp(-beta * (w_mu - E0))[:, None]
        den = iw[:, None, None] + w_nu[None, None, :] - w_mu[None, :, None]
        G += ((M2 * fac)[None, :, :] / den).sum(axis=(1, 2))
    return G / Z


def lanczos_coeffs(H, phi: np.ndarray, L: int, reorth: bool = False, tol: float = 1e-12):
    """Lanczos recurrence from phi: returns (n2, a, b) with n2 = <phi|phi>,
    a_0..a_{k-1} the diagonal and b_1..b_{k-1} the off-diagonal of the
    tridiagonal matrix (b[0] = 0 as a placeholder).  Stops early when
    b_j <= tol * |H| estimate (Krylov space exhausted)."""
    n2 = float(phi @ phi)
    a, b = [], [0.0]
    if n2 == 0.0:
        return 0.0, np.zeros(0), np.zeros(0)
    v_prev = np.zeros_like(phi)
    v = phi / np.sqrt(n2)
    basis = [v] if reorth else None
    scale = 0.0
    for j in range(L):
        w = H @ v
        alpha = float(v @ w)
        w = w - alpha * v - b[-1] * v_prev
        if reorth:
            for _ in range(2):
                for q in basis:
                    w -= (q @ w) * q
        a.append(alpha)
        beta = float(np.sqrt(w @ w))
        scale = max(scale, abs(alpha), beta)
        if j == L - 1 or beta <= tol * max(scale, 1.0):
            break
        b.append(beta)
        v_prev, v = v, w / beta
        if reorth:
            basis.append(v)
    return n2, np.array(a), np.array(b[:len(a)])


def cf_eval(z: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """1 / (z - a_0 - b_1^2 / (z - a_1 - b_2^2 / ( ... / (z - a_{k-1})))), bottom up."""
    z = np.asarray(z, dtype=complex)
    g = 1.0 / (z - a[-1])
    for i in range(len(a) - 2, -1, -1):
        g = 1.0 / (z - a[i] - b[i + 1] ** 2 * g)
    return g


def greens_cf(model, states, beta: float, n_w: int, orbital: int = 0, spin: int = fock.UP,
              depth: int = 150, boltz_cut: float = 1e-5, reorth: bool = False,
              return_parts: bool = False, z=None, build=build_csr):
    """Continued-fraction G(i w_n) (or G(z) at the given complex z) from a list
    of states (n_up, n_dn, E, vector).

    Z is the sum of e^{-beta (E - E_min)} over the states passed; states whose
    factor is below ``boltz_cut`` are left out of the sum over nu.  ``build``
    makes the neighbour sectors' H (``sector.build_csr`` or, for sectors of tens
    of millions of states, ``sector.build_csr_blocked``)."""
    E = np.array([s[2] for s in states])
    E0 = E.min()
    fac = np.exp(-beta * (E - E0))
    Z = fac.sum()
    iw = 1j * matsubara(beta, n_w) if z is None else np.asarray(z, dtype=complex)
    G = np.zeros(len(iw), dtype=complex)
    parts = []
    n = model.n_s
    Hcache = {}

    def ham(a, b):
        if (a, b) not in Hcache:
            Hcache[(a, b)] = build(model, a, b)
        return Hcache[(a, b)]

    for (nu_, nd_, En, vec), f in zip(states, fac):
        if f < boltz_cut:
            continue
        w = f / Z
        for dag in (True, False):
            C, tgt = op_matrix(n, nu_, nd_, orbital, spin, dag)
            if C is None:
                parts.append((dag, 0.0, np.zeros(0), np.zeros(0)))
                continue
            phi = C @ vec
            n2, a, b = lanczos_coeffs(ham(*tgt), phi, depth, reorth=reorth)
            parts.append((dag, n2, a, b))
            if n2 == 0.0:
                continue
            if dag:
                G += w * n2 * cf_eval(iw + En, a, b)
            else:
                G += w * n2 * (-cf_eval(-(iw - En), a, b))
    return (G, parts) if return_parts else G


def spectral(G: np.ndarray) -> np.ndarray:
    """A(w) = -Im G(w + i eta) / pi from G on the line z = w + i eta."""
    return -np.imag(G) / np.pi
