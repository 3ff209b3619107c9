"""DMFT self-consistency for the one-band Hubbard model (Sec. 2: the lattice
problem is mapped onto the Anderson impurity of Eq. 2, whose Green's function
closes the loop).  Test infrastructure (see ``oracle/__init__``).

One update, from the impurity G(i w_n) of the AIM with level eps_d and bath
(eps_k, V_k):

    Delta(z)   = sum_k V_k^2 / (z - eps_k)                  bath hybridisation
    Sigma      = z - eps_d - Delta - 1 / G_imp              impurity self-energy
    G_loc      = sum_j w_j / (z + mu - e_j - Sigma)         lattice local Green's function
    Delta_new  = z - eps_d - Sigma - 1 / G_loc              new Weiss field as a hybridisation

and the new bath is the least-squares fit of Delta_new on the first n_fit
Matsubara points, chi2 = (1/n_fit) sum_n |Delta_new - Delta_fit|^2.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import least_squares


def hybridisation(z, eps, V):
    z = np.asarray(z, dtype=complex)
    return ((np.asarray(V) ** 2)[None, :] / (z[:, None] - np.asarray(eps)[None, :])).sum(axis=1)


def self_energy(z, G_imp, eps_d, eps, V):
    z = np.asarray(z, dtype=complex)
    return z - eps_d - hybridisation(z, eps, V) - 1.0 / np.asarray(G_imp)


def lattice_gloc(z, sigma, mu, e, w):
    z = np.asarray(z, dtype=complex)
    return (np.asarray(w)[None, :] / ((z + mu - np.asarray(sigma))[:, None] - np.asarray(e)[None, :])).sum(axis=1)


def weiss_hybridisation(z, sigma, G_loc, eps_d):
    return np.asarray(z, dtype=complex) - eps_d - np.asarray(sigma) - 1.0 / np.asarray(G_loc)


def chi2(z, target, eps, V):
    return float(np.mean(np.abs(np.asarray(target) - hybridisation(z, eps, V)) ** 2))


def fit_bath(z, target, eps0, V0):
    """Least-squares bath (eps_k, V_k) for the hybridisation `target` at z."""
    z = np.asarray(z, dtype=complex)
    nb = len(eps0)

    def res(p):
        d = np.asarray(target) - hybridisation(z, p[:nb], p[nb:])
        return np.concatenate([d.real, d.imag]) / np.sqrt(len(z))

    r = least_squares(res, np.concatenate([eps0, V0]), method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15,
                      max_nfev=20000)
    eps, V = r.x[:nb], np.abs(r.x[nb:])
    return eps, V, chi2(z, target, eps, V)


def update(iw, G_imp, eps_d, mu, eps, V, e, w, n_fit):
    """One self-consistency step; returns (eps_new, V_new, chi2, Sigma, G_loc, Delta_new)."""
    sig = self_energy(iw, G_imp, eps_d, eps, V)
    gl = lattice_gloc(iw, sig, mu, e, w)
    dn = weiss_hybridisation(iw, sig, gl, eps_d)
    e2, v2, c2 = fit_bath(iw[:n_fit], dn[:n_fit], np.asarray(eps, float), np.asarray(V, float))
    return e2, v2, c2, sig, gl, dn
