"""Oracle: plain, slow, FP64 CPU reference for SU(2) two-site DMRG H.psi.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The library (``paper_2309_16724_gb300``) never imports it,
and this package never imports the library: the two share no code.  The one
shared module is ``synth`` (seeded inputs, no method arithmetic).

Each function cites the passage of arXiv:2309.16724 it follows:

* ``su2``      Wigner 6j (Eq. A3/A4), 9j (Eq. A2), the scalar factor C~
               (Eq. a), plus Clebsch-Gordan coefficients by Racah's formula
               (the "directly from Clebsch-Gordan" route of Appendix A).
* ``model``    reduced site operators (Sec. II.B, three-state orbital site
               and spin-1/2 site), the operator-table of Eq. 2.
* ``sectors``  the block-sparse two-site wavefunction (sector-table, Sec. II.A).
* ``heff``     sector-task-table (Eq. 3), sector-value table (Sec. II.C),
               H.psi as the sum of Eq. 2, diagonal of H_eff.
* ``env``      block operators A_i, D_i: Heisenberg renormalisation from a
               seeded MPS (W9j^(l), W9j^(r) factors, Sec. II.C) and the
               synthetic-entry ab initio skeleton.
* ``expand``   independent definitions used as pins: Clebsch-Gordan
               expansion to the m-resolved (U(1)) basis, explicit full-space
               projection P^T H P for small spin chains.
* ``abinitio`` the ab initio Hamiltonian (Eq. 1) from integrals: spin-adapted
               normal/complementary block operators renormalised from a
               seeded MPS (Sec. II.A, II.C) and the operator-table at the
               two-site bond.
* ``fci``      full configuration interaction of small ab initio problems.
* ``sweep``    the two-site sweep (Sec. II): Davidson at every bond, SVD of
               the reduced wavefunction per bond sector, truncation to D
               multiplets, block growth with the kept singular vectors.
* ``davidson`` Davidson eigensolver (the diagonalisation of Sec. II).
* ``ed``       exact diagonalisation of small Heisenberg chains.

Parity status per function is stated in each module header.
"""
