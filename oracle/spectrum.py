"""Lowest eigenpairs of a sector Hamiltonian (tier iii).

Test infrastructure (see ``oracle/__init__``).

Dense ``numpy.linalg.eigh`` up to dimension 4900 (the full-diagonalisation limit
the paper states in Sec. 1, C(8,4)^2); above it ARPACK ``eigsh``, the
implicitly-restarted Arnoldi/Lanczos family the paper's solver belongs to
(abstract, Sec. 3).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

DENSE_LIMIT = 4900


def lowest(H, k: int = 1, vectors: bool = False, dense_limit: int = DENSE_LIMIT):
    n = H.shape[0]
    k = min(k, n)
    if n <= dense_limit:
        A = H.toarray() if sp.issparse(H) else np.asarray(H)
        w, v = np.linalg.eigh(A)
        return (w[:k], v[:, :k]) if vectors else w[:k]
    v0 = np.random.default_rng(12345).standard_normal(n)
    w, v = spla.eigsh(H, k=k, which="SA", tol=1e-14, v0=v0, ncv=max(2 * k + 1, 40))
    order = np.argsort(w)
    w, v = w[order], v[:, order]
    return (w, v) if vectors else w


def full_spectrum(H) -> np.ndarray:
    A = H.toarray() if sp.issparse(H) else np.asarray(H)
    return np.linalg.eigvalsh(A)
