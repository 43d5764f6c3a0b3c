"""CPU FP64 oracle for ROM-enhanced SISA on the parametric RTE (arXiv 2402.10488).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.  It shares no code with the CUDA library; the two meet only in the
seeded problem descriptions of ``paper_2402_10488_gb300.inputs``.

Everything here is plain numpy / scipy in float64, written to be checked against the paper by
eye: DG matrices are assembled from their integral definitions by Gauss quadrature, the
transport sweep is a sparse direct solve of the block-triangular system, DSA is a sparse
direct solve of the moment system, POD is a dense thin SVD.

Modules (each function cites the passage it follows):
  quadrature  -- S_N rules: normalised Gauss-Legendre (1D), Chebyshev-Legendre CL (2D)   Sec. 2.1
  dg          -- upwind DG matrices D_j, Sigma_t, Sigma_s, G, g^bc; D^+/D^-, D_C, D_J      Sec. 2.2, App. B
  transport   -- transport sweep, L and b-bar, coupled system A f = b, residual R^rho      Sec. 2.3, 2.3.1
  dsa         -- consistent DSA (1D as printed in App. B; 2D by the same derivation)      App. B
  rom         -- POD, affine reduced operators, ROMIG, correction snapshots, ROMSA         Sec. 3
  sisa        -- Alg. 1 (SISA) with SA in {none, exact, DSA, ROMSA, ROMSAD (Alg. 2)}       Sec. 2.3, 3.2.2

Parity status: every function is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``
against closed forms, printed formulas, invariants or brute force; none is "parity unpinned".
"""
