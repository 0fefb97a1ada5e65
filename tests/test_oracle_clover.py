"""Pins of the oracle's clover operator, partial temporal preconditioning and 3-D ILU (CPU only).

``oracle/clover.py`` is tied to: closed forms of F and A for constant abelian fields in a spatial
and a temporal plane (derived by hand from the definitions), the reduction to the Wilson 3-D
Schur operator when A = 0, the product S_L M_SW S_R of dense matrices (Eq. TPrecPartial against
App. B's sequence), hermiticity, chirality and gauge covariance of A, gamma_5-hermiticity, dense LU
solves, and the 4-D Schur clover comparator against the dense Schur complement of M_SW.
"""

import numpy as np
import pytest

import synthetic as S
from oracle import clover as CL
from oracle import dense as D
from oracle import wilson as W
from test_oracle_pins import _gauge_transform, _params


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _abelian(L, T, mu, nu, b, su3=True):
    """Unit links except U_mu(x) = diag(e^{i b x_nu}, e^{-i b x_nu} or 1, 1): flux b per mu-nu plaquette."""
    U = S.unit_gauge(L, T)
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    coord = (x, y, z, t)[nu]
    U[..., mu, 0, 0] = np.exp(1j * b * coord)
    U[..., mu, 1, 1] = np.exp(-1j * b * coord) if su3 else 1.0
    return U


def test_abelian_field_strength_spatial_plane():
    """U_x = diag(e^{iby}, e^{-iby}, 1): every xy leaf is diag(e^{-ib}, e^{ib}, 1), so
    F_xy = i sin b diag(-1, 1, 0), F_yx = -F_xy, the other planes vanish, and
    A = (c_s / 2) sin b diag(1, -1, 1, -1) (x) diag(-1, 1, 0) (sigma_xy = i diag(s3, s3))."""
    L, T, b = 4, 4, 2 * np.pi / 4
    U = _abelian(L, T, 0, 1, b)
    F = CL.field_strength(U, 0, 1)
    ref = 1j * np.sin(b) * np.diag([-1.0, 1.0, 0.0])
    assert np.max(np.abs(F - ref)) < 1e-14
    assert np.max(np.abs(CL.field_strength(U, 1, 0) + ref)) < 1e-14
    for (m, n) in [(0, 2), (1, 2), (0, 3), (1, 3), (2, 3)]:
        assert np.max(np.abs(CL.field_strength(U, m, n))) < 1e-14
    c_s, c_t = 1.3, 0.7
    A = CL.clover_term(U, c_s, c_t)
    refA = 0.5 * c_s * np.sin(b) * np.einsum("ab,cd->acbd", np.diag([1.0, -1.0, 1.0, -1.0]), np.diag([-1.0, 1.0, 0.0]))
    assert np.max(np.abs(A - refA)) < 1e-14


def test_abelian_field_strength_temporal_plane():
    """U_t = diag(e^{ibx}, e^{-ibx}, 1): every xt leaf is diag(e^{ib}, e^{-ib}, 1), so
    F_xt = i sin b diag(1, -1, 0) and A = (c_t / 2) sin b [[0, s1], [s1, 0]] (x) diag(1, -1, 0)
    (sigma_xt = gamma_x gamma_t = [[0, i s1], [i s1, 0]])."""
    L, T, b = 4, 6, 2 * np.pi / 4
    U = _abelian(L, T, 3, 0, b)
    F = CL.field_strength(U, 0, 3)
    assert np.max(np.abs(F - 1j * np.sin(b) * np.diag([1.0, -1.0, 0.0]))) < 1e-14
    c_s, c_t = 1.3, 0.7
    A = CL.clover_term(U, c_s, c_t)
    s1 = np.array([[0, 1], [1, 0]], dtype=complex)
    spin = np.block([[np.zeros((2, 2)), s1], [s1, np.zeros((2, 2))]])
    refA = 0.5 * c_t * np.sin(b) * np.einsum("ab,cd->acbd", spin, np.diag([1.0, -1.0, 0.0]))
    assert np.max(np.abs(A - refA)) < 1e-14


def test_trace_is_removed():
    """U(3) flux diag(e^{iby}, 1, 1): (Q - Q^dag)/8 = diag(-i sin b, 0, 0) has a trace; F is its traceless part."""
    L, T, b = 4, 4, 2 * np.pi / 4
    U = _abelian(L, T, 0, 1, b, su3=False)
    F = CL.field_strength(U, 0, 1)
    ref = 1j * np.sin(b) * np.diag([-2.0, 1.0, 1.0]) / 3.0
    assert np.max(np.abs(F - ref)) < 1e-14


def test_clover_term_properties():
    """A(x) is hermitian, commutes with gamma_5 and is gauge covariant; F is anti-hermitian and traceless."""
    U = S.random_gauge(4, 6, 0.5, 71)
    A = CL.clover_term(U, 1.2, 0.9).reshape(U.shape[:4] + (12, 12))
    assert np.max(np.abs(A - np.conj(np.swapaxes(A, -1, -2)))) < 1e-15
    g5 = np.kron(W.GAMMA5, np.eye(3))
    assert np.max(np.abs(A @ g5 - g5 @ A)) < 1e-15
    assert np.max(np.abs(A)) > 1e-2
    for (m, n) in CL.SPATIAL_PLANES + CL.TEMPORAL_PLANES:
        F = CL.field_strength(U, m, n)
        assert np.max(np.abs(F + np.conj(np.swapaxes(F, -1, -2)))) < 1e-15
        assert np.max(np.abs(np.trace(F, axis1=-2, axis2=-1))) < 1e-15
    g = S.random_gauge_transform(4, 6, 72)
    Ag = CL.clover_term(_gauge_transform(U, g), 1.2, 0.9)
    G = np.einsum("ab,...cd->...acbd", np.eye(4), g).reshape(g.shape[:4] + (12, 12))  # 1_spin (x) g(x)
    ref = G @ A @ np.conj(np.swapaxes(G, -1, -2))
    assert np.max(np.abs(Ag.reshape(A.shape) - ref)) < 1e-13


@pytest.fixture(scope="module")
def tiny():
    p = _params(2, 4, kappa_s=0.08, xi=3.0, bc=-1)
    U = S.random_gauge(2, 4, 0.5, 73)
    Acl = CL.clover_term(U, 1.1, 0.9)
    return p, U, Acl


def test_without_clover_term_ilu_is_the_schur_operator(tiny):
    """A = 0: M-tilde_ILU = diag(1, M-hat) (the partial and full schemes coincide for Wilson)."""
    p, U, _ = tiny
    par3 = W.parity3(p.L, p.T)
    zero = np.zeros(U.shape[:4] + (4, 3, 4, 3), dtype=np.complex128)
    psi = S.gaussian_source(p.L, p.T, 74)
    got = CL.M_ilu(U, zero, psi, p, par3)
    ref = W.restrict(psi, par3 == 0) + W.M_hat(U, psi, p, par3)
    assert _rel(got, ref) < 1e-14


@pytest.mark.parametrize("bc", [-1, 1])
def test_ilu_sequence_is_S_L_M_S_R(bc):
    """App. B's sequence equals the dense product S_L M_SW S_R, and its (e, e) block is 1 + Abar^ee (Eq. TPrecPartial)."""
    p = _params(2, 4, kappa_s=0.08, xi=3.0, bc=bc)
    U = S.random_gauge(2, 4, 0.5, 75)
    Acl = CL.clover_term(U, 1.1, 0.9)
    par3 = W.parity3(p.L, p.T)
    Mi = D.matrix(lambda v: CL.M_ilu(U, Acl, v, p, par3), p.L, p.T)
    SL = D.matrix(lambda v: W.S_L(U, v, p, par3), p.L, p.T)
    Ms = D.matrix(lambda v: CL.M_sw(U, Acl, v, p), p.L, p.T)
    SR = D.matrix(lambda v: W.S_R(U, v, p, par3), p.L, p.T)
    assert _rel(Mi, SL @ Ms @ SR) < 1e-13
    ev = par3 == 0
    Mee = D.matrix(lambda v: CL.M_ilu(U, Acl, v, p, par3), p.L, p.T, ev, ev)
    Abee = D.matrix(lambda v: CL.Abar(U, Acl, v, p, 0, par3), p.L, p.T, ev, ev)
    assert _rel(Mee, np.eye(Mee.shape[0]) + Abee) < 1e-14


def test_gamma5_hermiticity(tiny):
    p, U, Acl = tiny
    par3 = W.parity3(p.L, p.T)
    a, b = S.gaussian_source(p.L, p.T, 76), S.gaussian_source(p.L, p.T, 77)
    for f, fd in [(lambda v: CL.M_sw(U, Acl, v, p), lambda v: CL.M_sw_dag(U, Acl, v, p)),
                  (lambda v: CL.M_ilu(U, Acl, v, p, par3), lambda v: CL.M_ilu_dag(U, Acl, v, p, par3))]:
        lhs = np.vdot(a.ravel(), f(b).ravel())
        rhs = np.vdot(fd(a).ravel(), b.ravel())
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("bc", [-1, 1])
def test_solve_matches_dense_lu(bc):
    p = _params(2, 4, kappa_s=0.08, xi=3.0, bc=bc)
    U = S.random_gauge(2, 4, 0.5, 78)
    Acl = CL.clover_term(U, 1.1, 0.9)
    eta = S.gaussian_source(p.L, p.T, 79)
    psi, it, rel = CL.solve(U, Acl, eta, p, tol=1e-12)
    Ms = D.matrix(lambda v: CL.M_sw(U, Acl, v, p), p.L, p.T)
    ref = np.linalg.solve(Ms, eta.ravel()).reshape(eta.shape)
    assert rel <= 1e-12 and it > 0
    assert _rel(psi, ref) < 1e-9


@pytest.mark.parametrize("bc", [-1, 1])
def test_clover_4d_schur_is_the_dense_schur_complement(bc):
    """M-hat_4 of M_SW equals M_oo - M_oe M_ee^-1 M_eo of the dense M_SW in 4-D parity order."""
    p = _params(2, 4, kappa_s=0.08, xi=3.0, bc=bc)
    U = S.random_gauge(2, 4, 0.5, 81)
    Acl = CL.clover_term(U, 1.1, 0.9)
    par4 = W.parity4(p.L, p.T)
    ev, od = par4 == 0, par4 == 1
    blk = lambda a, b: D.matrix(lambda v: CL.M_sw(U, Acl, v, p), p.L, p.T, a, b)
    ref = blk(od, od) - blk(ev, od) @ np.linalg.solve(blk(ev, ev), blk(od, ev))
    got = D.matrix(lambda v: CL.M_hat4_sw(U, Acl, v, p, par4), p.L, p.T, od, od)
    assert _rel(got, ref) < 1e-13
    zero = np.zeros_like(Acl)
    psi = S.gaussian_source(p.L, p.T, 82)
    assert _rel(CL.M_hat4_sw(U, zero, psi, p, par4), W.M_hat4(U, psi, p, par4)) < 1e-14


def test_clover_4d_schur_solve(tiny):
    p, U, Acl = tiny
    eta = S.gaussian_source(p.L, p.T, 83)
    psi, it, rel = CL.solve_eo4d(U, Acl, eta, p, tol=1e-12)
    Ms = D.matrix(lambda v: CL.M_sw(U, Acl, v, p), p.L, p.T)
    ref = np.linalg.solve(Ms, eta.ravel()).reshape(eta.shape)
    assert rel <= 1e-12 and it > 0
    assert _rel(psi, ref) < 1e-9
    par4 = W.parity4(p.L, p.T)
    a, b = S.gaussian_source(p.L, p.T, 84), S.gaussian_source(p.L, p.T, 85)
    lhs = np.vdot(a.ravel(), CL.M_hat4_sw(U, Acl, b, p, par4).ravel())
    rhs = np.vdot(CL.M_hat4_sw_dag(U, Acl, a, p, par4).ravel(), b.ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
