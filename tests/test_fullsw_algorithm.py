"""CPU check of the algorithm the full SW Q^-1 kernels use, written out in NumPy from its
definition (not from the kernels), against the oracle's dense line inverse ``oracle/clover.py``.

The appendix ("Full Preconditioning with Clover") writes Q = A + mu - D_t = T_0 + V W^dag and
inverts it by one Woodbury step. The GPU path solves the open chain T_0 by block LU: the Schur
complements Sigma_t = mu + A(t) - [P_+ (x) W_{t-1}^dag] Sigma_{t-1}^-1 [P_- (x) W_{t-1}] differ from
the diagonal blocks only in their (P_+, P_-) corner, a forward sweep needs only the P_+ rows of
Sigma^-1 and the backward sweep adds [P_- (x) W_t] y_{t+1}. Q^-1 b = chi - Z Lambda W^dag chi with
chi = T_0^-1 b, Z = T_0^-1 V and Lambda = (1 + W^dag Z)^-1. A dropped projector, a swapped sweep
direction or a wrong wrap sign in this derivation fails here, before any kernel runs.
"""

import numpy as np
import pytest

import synthetic as S
from oracle import clover as CL
from oracle import wilson as W
from test_oracle_pins import _params


def _k1(M):
    """1_2 (x) M on one spin half (two spins x three colours)."""
    return np.kron(np.eye(2), M)


def _line_qinv(D, links, s, b):
    """Q^-1 b on one time line: D[t] the 12x12 diagonal blocks mu + A(t), links[t] the temporal
    link from t to t + 1 (links[T-1] the wrap link), s the boundary sign, b[t] 12-vectors."""
    T = len(D)
    Sinv = []
    for t in range(T):
        Sg = D[t].copy()
        if t > 0:
            Sg[:6, 6:] -= _k1(links[t - 1].conj().T) @ Sinv[t - 1][:6, 6:] @ _k1(links[t - 1])
        Sinv.append(np.linalg.inv(Sg))

    def t0_solve(rhs):
        z = [rhs[0].copy()]
        for t in range(1, T):
            zt = rhs[t].copy()
            zt[:6] += _k1(links[t - 1].conj().T) @ (Sinv[t - 1][:6] @ z[t - 1])
            z.append(zt)
        y = [None] * T
        y[T - 1] = Sinv[T - 1] @ z[T - 1]
        for t in range(T - 2, -1, -1):
            v = z[t].copy()
            v[6:] += _k1(links[t]) @ y[t + 1][6:]
            y[t] = Sinv[t] @ v
        return np.array(y)

    Uw = links[T - 1]
    Z = np.zeros((T, 12, 12), dtype=np.complex128)
    for j in range(12):
        col = np.zeros((T, 12), dtype=np.complex128)
        if j < 6:  # V_0 = -s P_+ (x) U_w^dag
            col[0, :6] = (-s * _k1(Uw.conj().T))[:, j]
        else:      # V_{T-1} = -s P_- (x) U_w
            col[T - 1, 6:] = (-s * _k1(Uw))[:, j - 6]
        Z[:, :, j] = t0_solve(col)
    WdZ = np.concatenate([Z[T - 1, :6, :], Z[0, 6:, :]])  # W^dag Z: P_+ rows at T-1, P_- rows at 0
    Lam = np.linalg.inv(np.eye(12) + WdZ)
    chi = t0_solve(b)
    c = Lam @ np.concatenate([chi[T - 1, :6], chi[0, 6:]])
    return chi - np.einsum("tij,j->ti", Z, c)


@pytest.mark.parametrize("T,bc,seed", [(2, -1, 61), (4, 1, 62), (5, -1, 63), (8, 1, 64), (12, -1, 65)])
def test_block_lu_woodbury_equals_the_dense_line_inverse(T, bc, seed):
    L = 2
    p = _params(L, T, kappa_s=0.08, xi=3.0, bc=bc)
    U = S.random_gauge(L, T, 0.5, seed)
    Acl = CL.clover_term(U, 1.1, 0.9)
    psi = S.gaussian_source(L, T, seed + 100)
    ref = CL.Q_inverse(U, Acl, psi, p)
    for (x, y, z) in [(0, 0, 0), (1, 0, 1), (1, 1, 1)]:
        D = [p.mu * np.eye(12) + Acl[t, z, y, x].reshape(12, 12) for t in range(T)]
        links = [U[t, z, y, x, W.MU_T] for t in range(T)]
        b = psi[:, z, y, x].reshape(T, 12)
        got = _line_qinv(D, links, p.bc, b)
        want = ref[:, z, y, x].reshape(T, 12)
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_dropping_the_wrap_correction_fails():
    """Without the Woodbury correction the result is T_0^-1 b, not Q^-1 b (the test has teeth)."""
    L, T = 2, 6
    p = _params(L, T, kappa_s=0.08, xi=3.0, bc=-1)
    U = S.random_gauge(L, T, 0.5, 66)
    Acl = CL.clover_term(U, 1.0, 1.0)
    psi = S.gaussian_source(L, T, 166)
    ref = CL.Q_inverse(U, Acl, psi, p)
    D = [p.mu * np.eye(12) + Acl[t, 0, 0, 0].reshape(12, 12) for t in range(T)]
    links = [U[t, 0, 0, 0, W.MU_T] for t in range(T)]
    b = psi[:, 0, 0, 0].reshape(T, 12)
    want = ref[:, 0, 0, 0].reshape(T, 12)
    open_chain = _line_qinv(D, links, 0.0, b)  # s = 0 removes V: plain T_0^-1 b
    assert np.abs(open_chain - want).max() > 1e-3 * np.abs(want).max()
