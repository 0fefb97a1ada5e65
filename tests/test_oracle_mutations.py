"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case patches one plausible error into the oracle (a flipped sign, a dropped
factor, a transposed link, a wrong recurrence sign, a reversed product) and checks
that at least one pin of ``test_oracle_pins``, ``test_oracle_determinant`` or
``test_oracle_clover`` then fails.
"""

import numpy as np
import pytest

import synthetic as S
from oracle import wilson as W
import test_oracle_pins as P


def _medium():
    p = P._params(4, 8, kappa_s=0.075, xi=3.5)
    return p, S.random_gauge(4, 8, 0.3, 21), S.gaussian_source(4, 8, 22)


def _small():
    p = P._params(2, 4)
    return p, S.random_gauge(2, 4, 0.3, 11), S.gaussian_source(2, 4, 12)


def test_flipped_wrap_sign_is_caught(monkeypatch):
    orig = W._vw

    def bad(U, p):
        V, Wm = orig(U, p)
        return -V, Wm

    monkeypatch.setattr(W, "_vw", bad)
    with pytest.raises(AssertionError):
        P.test_Tinv_matches_dense_inverse(-1)
    with pytest.raises(AssertionError):
        P.test_temporal_factorisation(_medium())


def test_backsub_sign_of_app_b_is_caught(monkeypatch):
    """The recurrence as printed in App. B (chi - U psi) is not T_0's inverse."""

    def bad(U0, rhs, mu):
        T = rhs.shape[W.AX_T]
        chi = np.zeros_like(rhs)
        chi[W._t_index(chi, T - 1)] = rhs[W._t_index(rhs, T - 1)] / mu
        for t in range(T - 2, -1, -1):
            chi[W._t_index(chi, t)] = (rhs[W._t_index(rhs, t)] - W.colour(U0[t], chi[W._t_index(chi, t + 1)])) / mu
        return chi

    monkeypatch.setattr(W, "T0_backsub", bad)
    with pytest.raises(AssertionError):
        P.test_Tinv_matches_dense_inverse(1)


def test_dropped_projector_half_is_caught(monkeypatch):
    def bad(U, psi, mu, bc):
        Umu = W.link(U, mu)
        fwd = W.colour(Umu, W.shift(psi, mu, +1, bc))
        bwd = W.colour(W.dag(W.shift(Umu, mu, -1, 1.0)), W.shift(psi, mu, -1, bc))
        return W.spin(W.I4 - W.GAMMA[mu], fwd) + W.spin(W.I4 + W.GAMMA[mu], bwd)

    monkeypatch.setattr(W, "hop", bad)
    with pytest.raises(AssertionError):
        P.test_free_field_momentum_space()


def test_untransposed_backward_link_is_caught(monkeypatch):
    def bad(U, psi, mu, bc):
        Umu = W.link(U, mu)
        fwd = W.colour(Umu, W.shift(psi, mu, +1, bc))
        bwd = W.colour(W.shift(Umu, mu, -1, 1.0), W.shift(psi, mu, -1, bc))
        return W.spin(0.5 * (W.I4 - W.GAMMA[mu]), fwd) + W.spin(0.5 * (W.I4 + W.GAMMA[mu]), bwd)

    monkeypatch.setattr(W, "hop", bad)
    with pytest.raises(AssertionError):
        P.test_gamma5_hermiticity(_medium())


def test_wrong_schur_sign_is_caught(monkeypatch):
    def bad(U, psi_o, p, par3=None):
        if par3 is None:
            par3 = W.parity3(p.L, p.T)
        x = W.restrict(psi_o, par3 == 1)
        return x + W.Dbar_s(U, W.Dbar_s(U, x, p, 0, par3), p, 1, par3) / p.gamma_f ** 2

    monkeypatch.setattr(W, "M_hat", bad)
    with pytest.raises(AssertionError):
        P.test_Mhat_is_dense_schur_complement(_small())
    with pytest.raises(AssertionError):
        P.test_tprec_full_block_form(_medium())


def test_swapped_projectors_in_CL_is_caught(monkeypatch):
    monkeypatch.setattr(W, "C_L", lambda U, psi, p: W.spin(W.P_MINUS, psi) + W.spin(W.P_PLUS, W.Tinv(U, psi, p)))
    with pytest.raises(AssertionError):
        P.test_temporal_factorisation(_medium())


# --------------------------------------------------------------------------- determinant of mu - D_t
def test_reversed_polyakov_order_is_caught(monkeypatch):
    import test_oracle_determinant as PD
    from oracle import determinant as DT

    def bad(U, p):
        U0 = W.link(U, W.MU_T)
        P_ = np.broadcast_to(np.eye(3, dtype=np.complex128), U0.shape[1:]).copy()
        for t in range(p.T):
            P_ = U0[t] @ P_
        return P_

    monkeypatch.setattr(DT, "polyakov", bad)
    with pytest.raises(AssertionError):
        PD.test_per_site_determinant_matches_dense_T(2, 4, -1)


def test_dropped_boundary_sign_in_determinant_is_caught(monkeypatch):
    import test_oracle_determinant as PD
    from oracle import determinant as DT

    def bad(U, p):
        _, la = np.linalg.slogdet(np.eye(3) - p.mu ** (-p.T) * DT.polyakov(U, p))
        return 3 * p.T * np.log(p.mu) + la

    monkeypatch.setattr(DT, "logdet_per_site", bad)
    with pytest.raises(AssertionError):
        PD.test_logdet_matches_dense_mu_minus_Dt(2, 4, -1)
    with pytest.raises(AssertionError):
        PD.test_det_M_is_det_M_hat_times_det_mu_minus_Dt(2, 4, -1)


def test_adjoint_resolvent_in_force_is_caught(monkeypatch):
    import test_oracle_determinant as PD
    from oracle import determinant as DT
    orig = DT.transported_resolvent
    monkeypatch.setattr(DT, "transported_resolvent", lambda U, p: np.conj(np.swapaxes(orig(U, p), -1, -2)))
    with pytest.raises(AssertionError):
        PD.test_force_matches_finite_differences_of_dense_determinants(-1)


def test_swapped_prefix_and_suffix_in_force_is_caught(monkeypatch):
    import test_oracle_determinant as PD
    from oracle import determinant as DT

    def bad(U, p):
        U0 = W.link(U, W.MU_T)
        T = p.T
        eye = np.broadcast_to(np.eye(3, dtype=np.complex128), U0.shape[1:])
        A = [eye.copy()]
        for t in range(T - 1):
            A.append(A[-1] @ U0[t])
        B = [None] * T
        B[T - 1] = eye.copy()
        for t in range(T - 2, -1, -1):
            B[t] = U0[t + 1] @ B[t + 1]
        R = p.mu ** (-T) * np.linalg.inv(np.eye(3) - p.bc * p.mu ** (-T) * (A[T - 1] @ U0[T - 1]))
        return np.stack([U0[t] @ A[t] @ R @ B[t] for t in range(T)])

    monkeypatch.setattr(DT, "transported_resolvent", bad)
    with pytest.raises(AssertionError):
        PD.test_force_matches_finite_differences_of_dense_determinants(-1)


# --------------------------------------------------------------------------- clover, partial preconditioning, ILU
def test_reversed_clover_leaf_is_caught(monkeypatch):
    import test_oracle_clover as PC
    from oracle import clover as CL
    orig = CL.clover_leaves

    def bad(U, mu, nu):
        Um, Un = W.link(U, mu), W.link(U, nu)
        first = Um @ CL._sh(Un, mu, 1) @ CL._dag(CL._sh(Um, nu, 1)) @ CL._dag(Un)
        return orig(U, mu, nu) - first + CL._dag(first)   # one leaf traversed the other way

    monkeypatch.setattr(CL, "clover_leaves", bad)
    with pytest.raises(AssertionError):
        PC.test_abelian_field_strength_spatial_plane()


def test_kept_trace_in_field_strength_is_caught(monkeypatch):
    import test_oracle_clover as PC
    from oracle import clover as CL
    monkeypatch.setattr(CL, "field_strength", lambda U, mu, nu: (CL.clover_leaves(U, mu, nu)
                                                                 - CL._dag(CL.clover_leaves(U, mu, nu))) / 8.0)
    with pytest.raises(AssertionError):
        PC.test_trace_is_removed()


def test_sigma_without_half_is_caught(monkeypatch):
    import test_oracle_clover as PC
    from oracle import clover as CL
    monkeypatch.setattr(CL, "sigma", lambda mu, nu: W.GAMMA[mu] @ W.GAMMA[nu] - W.GAMMA[nu] @ W.GAMMA[mu])
    with pytest.raises(AssertionError):
        PC.test_abelian_field_strength_temporal_plane()


def test_wrong_sign_in_ilu_sequence_is_caught(monkeypatch):
    import test_oracle_clover as PC
    from oracle import clover as CL

    def bad(U, Acl, psi, p, par3=None):
        if par3 is None:
            par3 = W.parity3(p.L, p.T)
        ev, od = par3 == 0, par3 == 1
        psi_e, psi_o = W.restrict(psi, ev), W.restrict(psi, od)
        t1 = W.Dbar_s(U, psi_o, p, 0, par3) / p.gamma_f
        t2 = CL.Abar(U, Acl, t1 + psi_e, p, 0, par3)
        chi_o = psi_o + CL.Abar(U, Acl, psi_o, p, 1, par3) + W.Dbar_s(U, t2 + t1, p, 1, par3) / p.gamma_f
        return psi_e + t2 + chi_o

    monkeypatch.setattr(CL, "M_ilu", bad)
    with pytest.raises(AssertionError):
        PC.test_ilu_sequence_is_S_L_M_S_R(-1)


# --------------------------------------------------------------------------- full SW temporal preconditioning
def test_swapped_projectors_in_woodbury_are_caught(monkeypatch):
    import test_oracle_full_sw as PF
    from oracle import clover as CL
    orig = CL.wrap_factors

    def bad(U0_last, p):
        V, Wd = orig(U0_last, p)
        T = p.T
        Wd = Wd.copy()
        Wd[:, 0:12], Wd[:, 12 * (T - 1):] = Wd[:, 12 * (T - 1):].copy(), Wd[:, 0:12].copy()
        return V, Wd

    monkeypatch.setattr(CL, "wrap_factors", bad)
    with pytest.raises(AssertionError):
        PF.test_line_inverse(4, -1)


def test_adjoint_in_the_wrong_order_is_caught(monkeypatch):
    import test_oracle_full_sw as PF
    from oracle import clover as CL
    monkeypatch.setattr(CL, "M_hat_full_sw_dag",
                        lambda U, Acl, v, p, par3=None: W.spin(W.GAMMA5, CL.M_hat_full_sw(U, Acl, W.spin(W.GAMMA5, v), p, par3)))
    with pytest.raises(AssertionError):
        PF.test_adjoint_and_solve()
