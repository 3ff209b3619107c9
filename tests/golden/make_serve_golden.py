"""Writes tests/golden/serve_stream.json from the CPU oracle alone.

The impurity-solve request stream the benchmark serves: three-orbital
Kanamori impurities with seeded random baths, N_s uniform in 10..16, sector
(ceil(N_s/2), floor(N_s/2)), Poisson arrivals (``workloads.serving_stream``,
seed 0).  For the first 16 requests with N_s <= 14 it stores the 4 lowest
energies of the sector (oracle sector CSR by literal operator application,
Sec. 4 Hamiltonian; ARPACK) and G(i w_n) of orbital 0 spin up from those four
states with Boltzmann weights at beta = 40 and the 1e-5 weight cutoff of
Sec. 4 (oracle continued fractions, depth 100, Eq. 3 with the standard sign)
on the first 64 of 1024 Matsubara points and every 32nd after them.

Run once (about an hour on one core, ~25 GB of RAM at N_s = 14):

    python tests/golden/make_serve_golden.py

It imports only ``oracle`` and ``workloads`` (the seeded parameter draws).
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import greens as og, sector as osec, spectrum  # noqa: E402

N_REQ, K, NS_MAX = 16, 4, 14
BETA, N_W, DEPTH, CUT = 40.0, 1024, 100, 1e-5


def stored_points():
    return list(range(64)) + list(range(64, N_W, 32))


def main(out_path=os.path.join(os.path.dirname(os.path.abspath(__file__)), "serve_stream.json")):
    stream = W.serving_stream(N_REQ, seed=0, rate=1.0, ns_range=(10, 16))
    pts = stored_points()
    out = {"what": "oracle lowest energies and G(i w_n) of the served request stream (Sec. 2 impurity solves, "
                   "Sec. 4 Hamiltonian and state cutoff, Eq. 3 standard sign)",
           "stream": {"n_requests": N_REQ, "seed": 0, "rate": 1.0, "ns_range": [10, 16]},
           "k": K, "greens": {"beta": BETA, "n_w": N_W, "depth": DEPTH, "boltz_cut": CUT, "orbital": "orb0",
                              "spin": "up", "n": pts},
           "requests": []}
    for r in stream:
        if r["n_s"] > NS_MAX:
            continue
        t0 = time.time()
        m = W.kanamori(r["n_s"], seed=r["model_seed"])
        H = osec.build_csr_blocked(m, r["n_up"], r["n_dn"])
        w, v = spectrum.lowest(H, K, vectors=True)
        del H
        states = [(r["n_up"], r["n_dn"], float(w[j]), v[:, j].copy()) for j in range(len(w))]
        del v
        G = og.greens_cf(m, states, BETA, N_W, orbital=m.orb0, spin=0, depth=DEPTH, boltz_cut=CUT,
                         build=osec.build_csr_blocked)
        out["requests"].append({"id": r["id"], "n_s": r["n_s"], "model_seed": r["model_seed"],
                                "sector": [r["n_up"], r["n_dn"]], "E": [float(e) for e in w],
                                "G_re": [float(G[i].real) for i in pts], "G_im": [float(G[i].imag) for i in pts],
                                "seconds": time.time() - t0})
        print(json.dumps({"id": r["id"], "n_s": r["n_s"], "E0": float(w[0]), "s": time.time() - t0}), flush=True)
    with open(out_path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
