"""(N_up, N_dn) sector basis, explicit sector CSR, row-sampled H*v, Fig. 1 CSR.

Test infrastructure (see ``oracle/__init__``).

Basis convention: per spin, all n_s-bit strings with the sector's particle
number in ascending numeric order; the rank of a string is its position in that
list, found here by binary search (``np.searchsorted``).  A sector state is the
pair (r_up, r_dn) at flat index r_up * D_dn + r_dn.

H is built by applying every operator product of ``fock.hamiltonian_terms``
literally to every basis state (tier ii); nothing here uses a factorised hop
formula.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fock


def spin_basis(n_s: int, n: int) -> np.ndarray:
    """All n_s-bit strings with popcount n, ascending (uint64)."""
    allv = np.arange(1 << n_s, dtype=np.uint64)
    return allv[fock.popcount(allv) == n]


class Sector:
    def __init__(self, n_s: int, n_up: int, n_dn: int):
        if not (0 <= n_up <= n_s and 0 <= n_dn <= n_s):
            raise ValueError("particle numbers out of range")
        self.n_s, self.n_up, self.n_dn = n_s, n_up, n_dn
        self.up = spin_basis(n_s, n_up)
        self.dn = spin_basis(n_s, n_dn)
        self.D_up, self.D_dn = len(self.up), len(self.dn)
        self.dim = self.D_up * self.D_dn

    def states(self, idx=None) -> np.ndarray:
        """Fock integers u | d << n_s of the sector states (all, or at flat indices idx)."""
        if idx is None:
            idx = np.arange(self.dim, dtype=np.int64)
        idx = np.asarray(idx, dtype=np.int64)
        u = self.up[idx // self.D_dn]
        d = self.dn[idx % self.D_dn]
        return u | (d << np.uint64(self.n_s))

    def index(self, f: np.ndarray) -> np.ndarray:
        """Flat indices of Fock integers that lie in this sector (checked)."""
        f = np.asarray(f, dtype=np.uint64)
        mask = np.uint64((1 << self.n_s) - 1)
        u, d = f & mask, f >> np.uint64(self.n_s)
        iu = np.searchsorted(self.up, u)
        idn = np.searchsorted(self.dn, d)
        if len(f):
            if iu.max() >= self.D_up or idn.max() >= self.D_dn:
                raise AssertionError("state outside the sector")
            if not (np.all(self.up[iu] == u) and np.all(self.dn[idn] == d)):
                raise AssertionError("state outside the sector")
        return iu.astype(np.int64) * self.D_dn + idn.astype(np.int64)


def build_csr(model, n_up: int, n_dn: int, terms=None) -> sp.csr_matrix:
    """Explicit sector Hamiltonian in CSR (tier ii).

    Entry H[row, col] = <row| H |col>, accumulated from every operator product
    applied to every basis state |col>.  Exact zeros are omitted off the
    diagonal; the diagonal is always stored; columns ascend within a row.
    """
    sec = Sector(model.n_s, n_up, n_dn)
    src = sec.states()
    cols = np.arange(sec.dim, dtype=np.int64)
    R, C, V = [cols], [cols], [np.zeros(sec.dim)]
    for coef, ops in (terms if terms is not None else fock.hamiltonian_terms(model)):
        tgt, amp = fock.apply_term(src, ops, coef)
        nz = amp != 0.0
        if not nz.any():
            continue
        R.append(sec.index(tgt[nz]))
        C.append(cols[nz])
        V.append(amp[nz])
    r, c, v = np.concatenate(R), np.concatenate(C), np.concatenate(V)
    H = sp.coo_matrix((v, (r, c)), shape=(sec.dim, sec.dim)).tocsr()
    H.sum_duplicates()
    coo = H.tocoo()
    keep = (coo.data != 0.0) | (coo.row == coo.col)
    H = sp.csr_matrix((coo.data[keep], (coo.row[keep], coo.col[keep])), shape=H.shape)
    H.sort_indices()
    return H


def row_entries(model, n_up: int, n_dn: int, rows, terms=None):
    """Rows of the sector H without building it: for each flat index i in ``rows``,
    the (column, value) pairs of <i|H|j> != 0, the diagonal always included.

    <i|H|j> = <j|H^+|i>, so every operator product's adjoint is applied to |i>.
    Returns (row_ptr, cols, vals) for the sampled rows, columns ascending.
    """
    sec = Sector(model.n_s, n_up, n_dn)
    rows = np.asarray(rows, dtype=np.int64)
    f = sec.states(rows)
    k = np.arange(len(rows), dtype=np.int64)
    R, C, V = [k], [rows], [np.zeros(len(rows))]
    for coef, ops in (terms if terms is not None else fock.hamiltonian_terms(model)):
        tgt, amp = fock.apply_term(f, fock.adjoint(ops), coef)
        nz = amp != 0.0
        if not nz.any():
            continue
        R.append(k[nz])
        C.append(sec.index(tgt[nz]))
        V.append(amp[nz])
    r, c, v = np.concatenate(R), np.concatenate(C), np.concatenate(V)
    A = sp.coo_matrix((v, (r, c)), shape=(len(rows), sec.dim)).tocsr()
    A.sum_duplicates()
    coo = A.tocoo()
    keep = (coo.data != 0.0) | (coo.col == rows[coo.row])
    A = sp.csr_matrix((coo.data[keep], (coo.row[keep], coo.col[keep])), shape=A.shape)
    A.sort_indices()
    return A.indptr.astype(np.int64), A.indices.astype(np.int64), A.data


def build_csr_blocked(model, n_up: int, n_dn: int, block: int = 1 << 21, terms=None) -> sp.csr_matrix:
    """The same sector CSR as ``build_csr``, assembled block of rows by block of
    rows from ``row_entries`` (each row's <i|H|j> from the adjoint operator
    products applied to |i>).  Peak memory is one block's entries plus the
    finished matrix, so sectors of tens of millions of states fit host RAM."""
    sec = Sector(model.n_s, n_up, n_dn)
    ptrs, cols, vals = [np.zeros(1, dtype=np.int64)], [], []
    base = 0
    for r0 in range(0, sec.dim, block):
        rows = np.arange(r0, min(sec.dim, r0 + block), dtype=np.int64)
        p, c, v = row_entries(model, n_up, n_dn, rows, terms)
        ptrs.append(p[1:] + base)
        cols.append(c.astype(np.int32))
        vals.append(v)
        base += len(v)
    return sp.csr_matrix((np.concatenate(vals), np.concatenate(cols), np.concatenate(ptrs)),
                         shape=(sec.dim, sec.dim))


def apply_rows(model, n_up: int, n_dn: int, rows, x: np.ndarray, terms=None) -> np.ndarray:
    """(H x)[rows] for a sector too large to build: y_i = sum_j <i|H|j> x_j."""
    ptr, cols, vals = row_entries(model, n_up, n_dn, rows, terms)
    y = np.zeros(len(rows))
    np.add.at(y, np.repeat(np.arange(len(rows)), np.diff(ptr)), vals * x[cols])
    return y


# ---------------------------------------------------------------- Fig. 1 CSR
def csr_from_dense(A: np.ndarray):
    """CSR arrays (row_ind, col_ind, values) of a dense matrix as laid out in Fig. 1:
    row_ind[i] is where row i starts in the nonzero list (length nrows + 1),
    col_ind the column of each stored entry, entries row by row, columns ascending."""
    row_ind = [0]
    col_ind, vals = [], []
    for i in range(A.shape[0]):
        for j in range(A.shape[1]):
            if A[i, j] != 0.0 or i == j:
                col_ind.append(j)
                vals.append(A[i, j])
        row_ind.append(len(col_ind))
    return np.array(row_ind, dtype=np.int64), np.array(col_ind, dtype=np.int64), np.array(vals)


def csr_matvec(row_ind, col_ind, vals, v) -> np.ndarray:
    """y = H v from CSR arrays, one row at a time, one stored entry at a time
    (the product Listing 1 describes), starting from y = 0."""
    n = len(row_ind) - 1
    y = np.zeros(n)
    for i in range(n):
        acc = 0.0
        for j in range(row_ind[i], row_ind[i + 1]):
            acc += vals[j] * v[col_ind[j]]
        y[i] = acc
    return y
