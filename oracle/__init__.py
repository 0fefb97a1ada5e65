"""Plain FP64 CPU oracle for arXiv 0910.0992's temporally preconditioned Wilson solve.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The library (``paper_0910_0992_gb300``) never imports it, and it never
imports the library: the two share only the seeded input generators in
``synthetic/``.

Modules:
  wilson  -- M, D_t, D_s, T, T^-1 by Sherman-Morrison-Woodbury, C_L, C_R, M~, M-hat,
             S_L, S_R, the 4-D Schur comparator (§II)
  solve   -- CGNR and the four solve methods, FP64 true residual
  dense   -- dense matrices and singular values on tiny lattices
  flops   -- the paper's FLOP-count model (App. B, App. C)
  force   -- pseudofermion action phi^dag (M-hat^dag M-hat)^-1 phi and its force dS/dU (FP64 adjoint
             through the six factors of M-hat), pinned by central finite differences
  determinant -- log det(mu - D_t) = log|det M| - log|det M-hat| from Polyakov products, and its
             force; the extra Hamiltonian term of the temporal preconditioner in HMC (§IV)
  clover  -- the SW clover term (clover-leaf field strength), M_SW = M + A, partial temporal
             preconditioning with 3-D ILU (Eq. TPrecPartial, App. B's apply sequence), the 4-D Schur
             clover comparator, full SW temporal preconditioning (the line inverse of A + mu - D_t,
             also by the appendix's Woodbury form) and their solves

Every function is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``
except where its docstring says "parity unpinned".
"""

from . import wilson, solve, dense, flops, force, determinant, clover  # noqa: F401
