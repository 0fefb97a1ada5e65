"""Seeded synthetic inputs for the anisotropic Wilson operator.

This module is the only code shared by the CPU oracle and the CUDA path. It
draws random numbers and builds input fields; it holds none of the
preconditioner's arithmetic (no hopping terms, no time-line solves, no
projectors).

Field conventions (the library's C-ABI uses the same layouts):

* spinor field  ``psi[t, z, y, x, spin, colour]``   complex128, shape ``(T, L, L, L, 4, 3)``
* gauge field   ``U[t, z, y, x, mu, row, col]``     complex128, shape ``(T, L, L, L, 4, 3, 3)``
  with ``mu = 0, 1, 2, 3`` for the x, y, z and t directions.
* gauge transformation ``g[t, z, y, x, row, col]``  complex128, shape ``(T, L, L, L, 3, 3)``

The paper's ensembles (quenched Wilson gauge action, Table I) are not
available; the links are the stand-in ``U = exp(i eps H)`` with ``H`` a
Gaussian Hermitian traceless matrix, which gives SU(3) links whose distance
from the unit matrix is set by ``eps``.
"""

from .fields import (
    gell_mann,
    random_su3,
    random_gauge,
    unit_gauge,
    random_gauge_transform,
    gaussian_source,
    point_sources,
    kappa_critical_free,
    workload,
    WORKLOADS,
)

__all__ = [
    "gell_mann",
    "random_su3",
    "random_gauge",
    "unit_gauge",
    "random_gauge_transform",
    "gaussian_source",
    "point_sources",
    "kappa_critical_free",
    "workload",
    "WORKLOADS",
]
