"""Plain FP64 CPU oracle for the disconnected-loop hot path (TEST INFRASTRUCTURE).

This package is test infrastructure only.  It is imported by `tests/`, by
`__graft_entry__.smoke()` and by the CPU-baseline leg of `bench.py`, never by the
product path (`paper_1309_2256_gb300`), and it imports nothing from that path.
It is written for a reader checking it against the paper by eye: full-lattice
numpy arrays, `np.roll` for neighbours, `einsum` for the colour and spin
products, LAPACK (`np.linalg.solve`) for dense exact inversion.  No blocking,
fusion or reordering beyond what each cited equation states.

Modules:
  lattice   site indexing, gamma matrices, the 16 Gamma, momentum list
  noise     Z4 (Z2 x iZ2) noise from a counter-based generator (Sec. 2.1)
  operator  twisted-mass Wilson-Dirac operator and its even-odd form (App. A)
  solver    CG on the normal equations; dense LU at small volume (Sec. 2.2)
  loops     bilinears, estimators (Eqs. loopSt, loopVv, loopStD, loopHPE1),
            momentum projection, HPE exact terms (Eq. HPE), TSM (Eq. estiTSM)
  network   the gauge-covariant parallel-transport network of the learned
            preconditioner (no counterpart in the paper), forward and exact backward

Parity status: every function here is pinned by a `-m "not gpu"` test
(tests/test_oracle_*.py) except the statements about the B55.32 physics,
which are out of scope (parity unpinned: no ensemble).
"""
from . import lattice, noise, operator, solver, loops, network  # noqa: F401
