"""Writes tests/golden/c3_ground.json from the CPU oracle alone.

The three-orbital Kanamori impurity with 12 bath sites (N_s = 15, seeded random
bath, seed 0), half-filled sector (N_up, N_dn) = (7, 8), dim 6435^2 =
41,409,225: the sector size the paper gives as the workstation limit of sparse
methods (Sec. 1).  Stored: the ground energy (ARPACK on the oracle's sector
CSR, built by literal second-quantised operator application, Sec. 4
Hamiltonian), and G(i w_n) of orbital 0 spin up from that ground state by the
oracle's Lanczos continued fractions (Eq. 3 with the standard sign, beta = 40,
1024 Matsubara points) at depth 100, on the first 64 points and every 32nd
after them.

Run once on a host with ~40 GB of free RAM (about half an hour on one core):

    python tests/golden/make_c3_golden.py

It imports only ``oracle`` and ``workloads`` (the seeded parameter draws).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import greens as og, sector as osec, spectrum  # noqa: E402

N_S, N_UP, N_DN, SEED = 15, 7, 8, 0
BETA, N_W, DEPTH = 40.0, 1024, 100


def stored_points():
    return list(range(64)) + list(range(64, N_W, 32))


def main(out_path=os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_ground.json")):
    m = W.kanamori(N_S, seed=SEED)
    t0 = time.time()
    H = osec.build_csr_blocked(m, N_UP, N_DN)
    t_build = time.time() - t0
    w, v = spectrum.lowest(H, 1, vectors=True)
    E0, psi = float(w[0]), v[:, 0].copy()
    res = float(np.linalg.norm(H @ psi - E0 * psi))
    t_eig = time.time() - t0 - t_build
    del H, v
    G = og.greens_cf(m, [(N_UP, N_DN, E0, psi)], BETA, N_W, orbital=m.orb0, spin=0, depth=DEPTH,
                     build=osec.build_csr_blocked)
    t_g = time.time() - t0 - t_build - t_eig
    pts = stored_points()
    out = {
        "what": "oracle ground energy and continued-fraction G(i w_n) of the N_s=15 three-orbital Kanamori "
                "impurity, sector (7,8), dim 41409225 (Sec. 1 workstation-limit sector; Sec. 4 Hamiltonian; "
                "Eq. 3 standard sign)",
        "model": {"kind": "kanamori", "n_s": N_S, "seed": SEED, "U": 2.3, "J": 0.4, "Up": "U-2J", "Jp": "J"},
        "sector": [N_UP, N_DN], "dim": int(len(psi)),
        "E0": E0, "residual_norm": res,
        "greens": {"beta": BETA, "n_w": N_W, "orbital": "orb0 (first impurity orbital)", "spin": "up",
                   "depth": DEPTH, "boltz_cut": 1e-5, "states": "ground state only",
                   "n": pts, "re": [float(G[i].real) for i in pts], "im": [float(G[i].imag) for i in pts]},
        "made_by": "tests/golden/make_c3_golden.py (oracle.sector.build_csr_blocked, oracle.spectrum.lowest, "
                   "oracle.greens.greens_cf)",
        "seconds": {"build": t_build, "eigsh": t_eig, "greens": t_g},
    }
    with open(out_path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("E0", "residual_norm", "seconds")}))


if __name__ == "__main__":
    main()
