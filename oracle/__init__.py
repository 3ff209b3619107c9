"""CPU oracle for the sector Hamiltonian-vector product, Lanczos spectra and
continued-fraction Green's functions.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import it.  It shares no code
with the CUDA library under ``paper_1004_3354_gb300/`` and never imports it; the
only module both sides use is ``workloads`` (seeded parameter draws).

Everything here is plain, slow and float64:

* ``fock``      second-quantised c / c+ on Fock integers with Jordan-Wigner signs,
                the Hamiltonian as an explicit list of operator products, and the
                brute-force Fock-space matrix (tier i).
* ``sector``    the (N_up, N_dn) sector basis (sorted strings, ranks by binary
                search), the explicit sector CSR built by literal operator
                application (tier ii), row-sampled H*v for large sectors, and the
                CSR layout of Fig. 1 with the Listing 1 product.
* ``spectrum``  lowest eigenvalues: dense eigh up to dim 4900 (the paper's stated
                full-diagonalisation limit, Sec. 1), ARPACK (eigsh) above (tier iii).
* ``greens``    Lehmann Green's function (Eq. 3, standard sign reading),
                c / c+ sector maps, Lanczos continued fractions.

Pins (tests/test_oracle_*.py, ``-m "not gpu"``): closed forms (two-site Hubbard,
U = 0 spectra and Green's function, Kanamori atomic multiplets), invariants
(Hermiticity, particle-number conservation, particle-hole and spin symmetry),
the worked CSR example of Fig. 1, brute force against the sector tier, CF
against Lehmann, and planted-mistake tests showing that each pin bites.
"""
