"""Pins of the oracle's full SW temporal preconditioning (CPU only).

Q = A + mu - D_t per time line: its dense inverse against Q itself (built from the operators, not
the line matrix), against the Wilson C_R C_L when A = 0 (mu - D_t = C_L^-1 C_R^-1, §II.A), and the
appendix's single-step Woodbury form against the dense inverse (T = 2, where the wrap and bulk
couplings share blocks, included); M-hat_full against (Q^oo)^-1 times the dense 3-D Schur
complement of M_SW, its A = 0 similarity to the Wilson M-hat, its adjoint, and its solve.
"""

import numpy as np
import pytest

import synthetic as S
from oracle import clover as CL
from oracle import dense as D
from oracle import wilson as W
from test_oracle_pins import _params


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _setup(L=2, T=4, bc=-1, seed=91):
    p = _params(L, T, kappa_s=0.08, xi=3.0, bc=bc)
    U = S.random_gauge(L, T, 0.5, seed)
    return p, U, CL.clover_term(U, 1.1, 0.9)


@pytest.mark.parametrize("T,bc", [(4, -1), (5, 1), (2, -1), (2, 1)])
def test_line_inverse(T, bc):
    p, U, Acl = _setup(T=T, bc=bc)
    psi = S.gaussian_source(p.L, T, 92, nrhs=2)
    q = CL.Q_inverse(U, Acl, psi, p)
    assert _rel(CL.Q_apply(U, Acl, q, p), psi) < 1e-13
    assert _rel(CL.Q_inverse_woodbury(U, Acl, psi, p), q) < 1e-13
    zero = np.zeros_like(Acl)
    assert _rel(CL.Q_inverse(U, zero, psi, p), W.C_R(U, W.C_L(U, psi, p), p)) < 1e-13


def test_full_operator_is_the_preconditioned_schur_complement():
    p, U, Acl = _setup()
    par3 = W.parity3(p.L, p.T)
    ev, od = par3 == 0, par3 == 1
    blk = lambda a, b: D.matrix(lambda v: CL.M_sw(U, Acl, v, p), p.L, p.T, a, b)
    schur = blk(od, od) - blk(ev, od) @ np.linalg.solve(blk(ev, ev), blk(od, ev))
    Qoo = D.matrix(lambda v: CL.Q_apply(U, Acl, v, p), p.L, p.T, od, od)
    ref = np.linalg.solve(Qoo, schur)
    got = D.matrix(lambda v: CL.M_hat_full_sw(U, Acl, v, p, par3), p.L, p.T, od, od)
    assert _rel(got, ref) < 1e-12


def test_without_clover_term_it_is_similar_to_the_wilson_operator():
    """A = 0: (Q^oo)^-1 = C_R^o C_L^o, so M-hat_full = C_R^o M-hat (C_R^o)^-1."""
    p, U, _ = _setup(seed=93)
    zero = np.zeros(U.shape[:4] + (4, 3, 4, 3), dtype=np.complex128)
    par3 = W.parity3(p.L, p.T)
    od = par3 == 1
    psi = W.restrict(S.gaussian_source(p.L, p.T, 94), od)
    ref = W.restrict(W.C_R(U, W.M_hat(U, W.restrict(W.C_R_inv(U, psi, p), od), p, par3), p), od)
    assert _rel(CL.M_hat_full_sw(U, zero, psi, p, par3), ref) < 1e-12


def test_adjoint_and_solve():
    p, U, Acl = _setup(seed=95)
    par3 = W.parity3(p.L, p.T)
    od = par3 == 1
    a = W.restrict(S.gaussian_source(p.L, p.T, 96), od)
    b = W.restrict(S.gaussian_source(p.L, p.T, 97), od)
    lhs = np.vdot(a.ravel(), CL.M_hat_full_sw(U, Acl, b, p, par3).ravel())
    rhs = np.vdot(CL.M_hat_full_sw_dag(U, Acl, a, p, par3).ravel(), b.ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    eta = S.gaussian_source(p.L, p.T, 98)
    psi, it, rel = CL.solve_full_sw(U, Acl, eta, p, tol=1e-12)
    Ms = D.matrix(lambda v: CL.M_sw(U, Acl, v, p), p.L, p.T)
    assert rel <= 1e-12 and it > 0
    assert _rel(psi, np.linalg.solve(Ms, eta.ravel()).reshape(eta.shape)) < 1e-9
