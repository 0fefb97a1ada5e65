"""Dense matrices of the oracle's operators on tiny lattices (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/wilson.py``).

Builds the matrix of a linear operator column by column by applying it to unit
vectors, so that identities of the paper can be checked with dense linear
algebra (inverse, Schur complement, singular values) from NumPy.
"""

import numpy as np

from . import wilson as W


def basis(L, T, mask=None):
    """Unit vectors on the sites where ``mask`` is true (all sites if None), all 12 components.

    Returns (E, idx) with E of shape (n, T, L, L, L, 4, 3) and idx the flat
    positions of the chosen degrees of freedom in a lattice field.
    """
    full = np.ones((T, L, L, L), dtype=bool) if mask is None else mask.astype(bool)
    sel = np.broadcast_to(full[..., None, None], (T, L, L, L, 4, 3)).ravel()
    idx = np.flatnonzero(sel)
    E = np.zeros((idx.size, T * L ** 3 * 12), dtype=np.complex128)
    E[np.arange(idx.size), idx] = 1.0
    return E.reshape((idx.size, T, L, L, L, 4, 3)), idx


def matrix(op, L, T, mask_in=None, mask_out=None, chunk=256):
    """Dense matrix of ``op`` from the dofs on ``mask_in`` to the dofs on ``mask_out``."""
    E, idx_in = basis(L, T, mask_in)
    _, idx_out = basis(L, T, mask_out)
    cols = []
    for k in range(0, E.shape[0], chunk):
        y = op(E[k:k + chunk])
        cols.append(y.reshape(y.shape[0], -1)[:, idx_out])
    return np.concatenate(cols, axis=0).T


def sigma_ratio(A):
    """sigma_max / sigma_min of a dense matrix (sqrt of the condition number of A^dag A)."""
    s = np.linalg.svd(A, compute_uv=False)
    return s[0] / s[-1]


def temporal_matrix(U, p, x, y, z):
    """Dense N_t x N_t block matrix T (3x3 blocks) of one spatial site, built from its definition (§II.A)."""
    T = p.T
    U0 = U[:, z, y, x, W.MU_T]
    D = np.zeros((3 * T, 3 * T), dtype=np.complex128)
    for t in range(T):
        D[3 * t:3 * t + 3, 3 * t:3 * t + 3] = p.mu * np.eye(3)
        tp = (t + 1) % T
        sgn = p.bc if t == T - 1 else 1.0
        D[3 * t:3 * t + 3, 3 * tp:3 * tp + 3] -= sgn * U0[t]
    return D
