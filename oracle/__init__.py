"""Oracle: plain, slow, FP64 CPU implementation of the FFT-VIE hot path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import anything here.  The
library under ``paper_2508_16471_gb300/`` never does, and the oracle imports
nothing from the library (the seeded input generators in
``paper_2508_16471_gb300.inputs`` hold no arithmetic of the method).

Modules:
  vie  -- discrete VIE (kernel, direct / dense / FFT operator, GMRES,
          incident field, far field, detector projection)
  hom  -- g2 (Eq. 10 and Eq. 11 by brute force), path amplitudes, coincidence
          counts, visibility, classical P2
  mie  -- Lorenz-Mie series (physics validation, not a parity pin)

Parity status: every function is pinned by a ``-m "not gpu"`` test against
closed forms, brute force or invariants (tests/test_oracle_*.py).
"""
