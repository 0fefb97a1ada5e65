"""FP64 oracle of the determinant of the temporal preconditioner and of its force.

TEST INFRASTRUCTURE ONLY (see ``oracle/wilson.py``).

The paper expects (§IV, closing paragraph) that hybrid Monte Carlo with the temporal
preconditioner acquires extra Hamiltonian terms from the determinants of the preconditioning
matrices, and does not derive them. For the Wilson operator of §II they follow from the
definitions:

* C_L = P_+ + P_- T^-1 and C_R = P_- + P_+ T^-dag (§II.A), so C_L^-1 C_R^-1 = P_- T + P_+ T^dag
  = mu - D_t, and M-tilde = C_L M C_R has unit diagonal blocks in the 3-D parity split, whose
  Schur complement is M-hat (§II.B). Hence det M = det(M-hat) det(mu - D_t).
* T acts on colour x time at one spatial site x: mu on the diagonal, -U_0(t) coupling t to t+1
  and the wrap entry -s U_0(N_t - 1) (§II.A). Eliminating the time slices one after the other
  gives det T(x) = det(mu^N_t 1 - s P(x)) with the ordered Polyakov product
  P(x) = U_0(x, 0) U_0(x, 1) ... U_0(x, N_t - 1).
* P_- and P_+ each hold two spin components, so det(mu - D_t) = prod_x |det T(x)|^4 >= 0.

This module evaluates

    log det(mu - D_t) = 4 sum_x log|det(mu^N_t 1 - s P(x))|
                      = 4 sum_x [3 N_t log mu + log|det(1 - s mu^-N_t P(x))|]

(the second form only avoids overflowing mu^N_t) and its derivative for
U_0(x, t) -> exp(i eps T_a) U_0(x, t), T_a = lambda_a / 2. With A(t) = U_0(0) ... U_0(t-1),
B(t) = U_0(t+1) ... U_0(N_t-1) and R = (mu^N_t 1 - s P)^-1 the product changes by
dP = A (i eps T_a) U_0(t) B, so

    d/d eps log|det(mu^N_t 1 - s P)| = Re Tr[R (-s) dP] / eps = -s Re Tr[i T_a Z(t)],
    Z(t) = U_0(t) B(t) R A(t),

and the force of log det(mu - D_t) is 4 times that; spatial links do not enter. Two flavours
of Wilson fermions carry the term -2 log det(mu - D_t) in their action beside the
pseudofermion action of M-hat. Pinned in ``tests/test_oracle_determinant.py`` against dense
determinants of mu - D_t, of M and of M-hat, the free field and finite differences.
"""

import numpy as np

from . import force as FO
from . import wilson as W


def polyakov(U, p):
    """P(x) = U_0(x, 0) U_0(x, 1) ... U_0(x, N_t - 1), shape (L, L, L, 3, 3) = [z, y, x]."""
    U0 = W.link(U, W.MU_T)
    P = np.broadcast_to(np.eye(3, dtype=np.complex128), U0.shape[1:]).copy()
    for t in range(p.T):
        P = P @ U0[t]
    return P


def logdet_per_site(U, p):
    """log|det(mu^N_t 1 - s P(x))| per spatial site, shape (L, L, L)."""
    c = p.bc * p.mu ** (-p.T)
    _, la = np.linalg.slogdet(np.eye(3) - c * polyakov(U, p))
    return 3 * p.T * np.log(p.mu) + la


def logdet_temporal(U, p):
    """log det(mu - D_t) = 4 sum_x log|det(mu^N_t 1 - s P(x))| (real; det(mu - D_t) >= 0)."""
    return float(4.0 * np.sum(logdet_per_site(U, p)))


def transported_resolvent(U, p):
    """Z(t) = U_0(t) B(t) (mu^N_t 1 - s P)^-1 A(t) per temporal link, shape (T, L, L, L, 3, 3)."""
    U0 = W.link(U, W.MU_T)
    T = p.T
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), U0.shape[1:])
    A = [eye.copy()]                       # A(t) = U_0(0) ... U_0(t-1)
    for t in range(T - 1):
        A.append(A[-1] @ U0[t])
    B = [None] * T                         # B(t) = U_0(t+1) ... U_0(N_t-1)
    B[T - 1] = eye.copy()
    for t in range(T - 2, -1, -1):
        B[t] = U0[t + 1] @ B[t + 1]
    P = A[T - 1] @ U0[T - 1]
    c = p.bc * p.mu ** (-T)
    R = p.mu ** (-T) * np.linalg.inv(np.eye(3) - c * P)   # (mu^N_t 1 - s P)^-1
    return np.stack([U0[t] @ B[t] @ R @ A[t] for t in range(T)])


def force_logdet_temporal(U, p):
    """F[t, z, y, x, mu, a] = d log det(mu - D_t) / d eps for U_mu -> exp(i eps T_a) U_mu (zero for mu < 3)."""
    Z = transported_resolvent(U, p)
    Ta = FO.generators()
    F = np.zeros(U.shape[:-2] + (8,))
    F[..., W.MU_T, :] = -4.0 * p.bc * np.real(np.einsum("aij,...ji->...a", 1j * Ta, Z))
    return F
