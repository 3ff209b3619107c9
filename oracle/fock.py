"""Second-quantised operators on Fock integers and the Hamiltonian as a term list.

Test infrastructure (see ``oracle/__init__``).

Mode order for Jordan-Wigner signs: all spin-up modes first (mode i = site i),
then all spin-down modes (mode n_s + i).  A Fock state is the integer whose bit
``mode`` is the occupation of that mode, i.e. ``u | (d << n_s)`` for the up
string u and down string d.

c_mode |f>  = (-1)^{#occupied modes below mode} |f - mode>   if mode occupied, else 0
c+_mode |f> = (-1)^{#occupied modes below mode} |f + mode>   if mode empty,    else 0
"""
from __future__ import annotations

import numpy as np

UP, DN = 0, 1


def popcount(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a, dtype=np.uint64)
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a).astype(np.int64)
    out = np.zeros(a.shape, dtype=np.int64)   # byte-table fallback for older numpy
    tab = np.array([bin(i).count("1") for i in range(256)], dtype=np.int64)
    x = a.copy()
    for _ in range(8):
        out += tab[(x & np.uint64(0xFF)).astype(np.int64)]
        x >>= np.uint64(8)
    return out


def mode(site: int, spin: int, n_s: int) -> int:
    return site + (n_s if spin == DN else 0)


def apply_op(states: np.ndarray, amps: np.ndarray, md: int, dagger: bool):
    """Apply c+_md (dagger) or c_md to a batch of basis states with amplitudes."""
    bit = np.uint64(1) << np.uint64(md)
    occ = (states & bit) != 0
    ok = ~occ if dagger else occ
    below = states & (bit - np.uint64(1))
    sign = 1.0 - 2.0 * (popcount(below) & 1)
    return states ^ bit, np.where(ok, amps * sign, 0.0)


def apply_term(states: np.ndarray, ops, coef: float):
    """Apply coef * (op_0 op_1 ... op_{k-1}) to each state; op_{k-1} acts first.

    ``ops`` is a sequence of (mode, dagger).  Returns (new_states, amplitudes);
    amplitude 0 marks states annihilated by the product.
    """
    s = np.asarray(states, dtype=np.uint64).copy()
    a = np.full(s.shape, float(coef))
    for md, dag in reversed(ops):
        s, a = apply_op(s, a, md, dag)
    return s, a


def adjoint(ops):
    """Hermitian adjoint of an operator product (real coefficient)."""
    return [(md, not dag) for md, dag in reversed(ops)]


def hamiltonian_terms(model):
    """All operator products of H with their coefficients.

    One-body (Eq. 1, Eq. 2 and the first line of the Sec. 4 Hamiltonian):
        T_ij c+_is c_js                        for every T_ij != 0, both spins
    On-site Hubbard U (Eq. 1, Eq. 2, Sec. 4):
        U_i n_iu n_id
    The impurity orbitals m of Sec. 4 are the sites orb0 .. orb0 + n_orb - 1.
    Inter-orbital density-density (Sec. 4, m < m'):
        (Up - J delta_ss') n_ms n_m's'
    Spin-flip and pair-hopping (Sec. 4, every ordered m != m'):
        -Jsf d+_mu d_md d+_m'd d_m'u
        -Jph d+_mu d+_md d_m'u d_m'd
    Number operators are written as c+ c and applied literally.
    """
    n = model.n_s
    T = model.T
    terms = []
    for s in (UP, DN):
        for i in range(n):
            for j in range(n):
                if T[i, j] != 0.0:
                    terms.append((T[i, j], [(mode(i, s, n), True), (mode(j, s, n), False)]))
    for i in range(n):
        if model.U_site[i] != 0.0:
            a, b = mode(i, UP, n), mode(i, DN, n)
            terms.append((model.U_site[i], [(a, True), (a, False), (b, True), (b, False)]))
    M = model.n_orb
    orbs = [model.orb0 + m for m in range(M)]   # impurity orbitals d_m sit on these sites
    for ia, m in enumerate(orbs):
        for mp in orbs[ia + 1:]:
            for s in (UP, DN):
                for sp in (UP, DN):
                    c = model.Up - (model.J if s == sp else 0.0)
                    if c != 0.0:
                        a, b = mode(m, s, n), mode(mp, sp, n)
                        terms.append((c, [(a, True), (a, False), (b, True), (b, False)]))
    for m in orbs:
        for mp in orbs:
            if m == mp:
                continue
            if model.Jsf != 0.0:
                terms.append((-model.Jsf, [(mode(m, UP, n), True), (mode(m, DN, n), False),
                                           (mode(mp, DN, n), True), (mode(mp, UP, n), False)]))
            if model.Jph != 0.0:
                terms.append((-model.Jph, [(mode(m, UP, n), True), (mode(m, DN, n), True),
                                           (mode(mp, UP, n), False), (mode(mp, DN, n), False)]))
    return terms


def fock_hamiltonian(model) -> np.ndarray:
    """Dense H on the full 4^n_s Fock space (tier i, brute force; n_s <= 6)."""
    n = model.n_s
    assert n <= 6, "brute-force Fock space is limited to n_s <= 6"
    nf = 1 << (2 * n)
    states = np.arange(nf, dtype=np.uint64)
    H = np.zeros((nf, nf))
    for coef, ops in hamiltonian_terms(model):
        tgt, amp = apply_term(states, ops, coef)
        nz = amp != 0.0
        np.add.at(H, (tgt[nz].astype(np.int64), states[nz].astype(np.int64)), amp[nz])
    return H


def fock_numbers(n_s: int):
    """(N_up, N_dn) of every Fock state in the order of ``fock_hamiltonian``."""
    nf = 1 << (2 * n_s)
    states = np.arange(nf, dtype=np.uint64)
    mask = np.uint64((1 << n_s) - 1)
    return popcount(states & mask), popcount(states >> np.uint64(n_s))
