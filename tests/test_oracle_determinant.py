"""Pins of the oracle's temporal-preconditioner determinant and its force (CPU only).

Each pin ties ``oracle/determinant.py`` to something other than itself: the dense
determinant of one site's T (built entry by entry from §II.A), the dense determinant of
mu - D_t, the factorisation det M = det(M-hat) det(mu - D_t) checked with dense M and M-hat
(§II.A-B), the free field, central finite differences of dense determinants, and gauge
invariance.
"""

import numpy as np
import pytest

import synthetic as S
from oracle import dense as D
from oracle import determinant as DT
from oracle import force as FO
from oracle import wilson as W
from test_oracle_pins import _gauge_transform, _params

CASES = [(2, 4, -1), (2, 5, 1), (2, 3, -1)]


def _lattice(L, T, bc, seed=31, eps=0.5, kappa_s=0.07, xi=3.0):
    return _params(L, T, kappa_s=kappa_s, xi=xi, bc=bc), S.random_gauge(L, T, eps, seed)


def _dense_mu_minus_Dt(U, p):
    return D.matrix(lambda v: p.mu * v - W.D_t(U, v, p.bc), p.L, p.T)


def _logdet_M_over_M_hat(U, p):
    """(phase of det M / det M-hat, log|det M| - log|det M-hat|) from dense matrices."""
    par3 = W.parity3(p.L, p.T)
    sm, lm = np.linalg.slogdet(D.matrix(lambda v: W.M(U, v, p), p.L, p.T))
    sh, lh = np.linalg.slogdet(D.matrix(lambda v: W.M_hat(U, v, p, par3), p.L, p.T, par3 == 1, par3 == 1))
    return sm / sh, lm - lh


@pytest.mark.parametrize("L,T,bc", CASES + [(2, 16, -1)])
def test_per_site_determinant_matches_dense_T(L, T, bc):
    """log|det T(x)| of the dense 3N_t x 3N_t matrix of one site equals the Polyakov-loop form."""
    p, U = _lattice(L, T, bc, kappa_s=0.1, xi=3.5)
    per_site = DT.logdet_per_site(U, p)
    for (x, y, z) in [(0, 0, 0), (1, 0, 1), (1, 1, 1)]:
        _, ref = np.linalg.slogdet(D.temporal_matrix(U, p, x, y, z))
        assert abs(per_site[z, y, x] - ref) < 1e-11 * max(1.0, abs(ref))


@pytest.mark.parametrize("L,T,bc", CASES)
def test_logdet_matches_dense_mu_minus_Dt(L, T, bc):
    """det(mu - D_t) is real and positive and its log is the oracle's value."""
    p, U = _lattice(L, T, bc)
    sign, ref = np.linalg.slogdet(_dense_mu_minus_Dt(U, p))
    assert abs(sign - 1.0) < 1e-10
    assert abs(DT.logdet_temporal(U, p) - ref) < 1e-11 * abs(ref)


@pytest.mark.parametrize("L,T,bc", CASES)
def test_det_M_is_det_M_hat_times_det_mu_minus_Dt(L, T, bc):
    """det M = det(M-hat) det(mu - D_t) with dense M (whole lattice) and M-hat (odd 3-D sites)."""
    p, U = _lattice(L, T, bc)
    phase, diff = _logdet_M_over_M_hat(U, p)
    assert abs(phase - 1.0) < 1e-9
    assert abs(diff - DT.logdet_temporal(U, p)) < 1e-9 * abs(diff)


@pytest.mark.parametrize("bc", [1, -1])
def test_free_field(bc):
    """U = 1: P = 1, so log det(mu - D_t) = 4 L^3 * 3 log|mu^N_t - s|."""
    p = _params(4, 6, kappa_s=0.08, xi=2.5, bc=bc)
    U = S.unit_gauge(4, 6)
    ref = 4 * 4 ** 3 * 3 * np.log(abs(p.mu ** 6 - bc))
    assert abs(DT.logdet_temporal(U, p) - ref) < 1e-12 * abs(ref)
    F = DT.force_logdet_temporal(U, p)
    assert np.max(np.abs(F)) < 1e-13   # Z = (mu^N_t - s)^-1 times 1 has no traceless part


@pytest.mark.parametrize("bc", [1, -1])
def test_force_matches_finite_differences_of_dense_determinants(bc):
    """dF / d eps of log|det M| - log|det M-hat| (dense) is the oracle's force, temporal and spatial links."""
    p, U = _lattice(2, 4, bc, seed=41)
    F = DT.force_logdet_temporal(U, p)
    h = 1e-5
    for mu, site, a in [(3, (0, 0, 0, 0), 0), (3, (3, 1, 0, 1), 4), (3, (2, 0, 1, 1), 7), (3, (3, 0, 0, 0), 2),
                        (1, (1, 0, 1, 0), 3)]:
        plus = _logdet_M_over_M_hat(FO.perturb(U, mu, site, a, +h), p)[1]
        minus = _logdet_M_over_M_hat(FO.perturb(U, mu, site, a, -h), p)[1]
        fd = (plus - minus) / (2 * h)
        t, z, y, x = site
        assert abs(F[t, z, y, x, mu, a] - fd) < 2e-7 * max(1.0, abs(fd)), (mu, site, a, fd)
    # and against the dense determinant of mu - D_t on a longer lattice
    p, U = _lattice(2, 6, bc, seed=43, kappa_s=0.12, xi=3.0)
    F = DT.force_logdet_temporal(U, p)
    for site, a in [((5, 1, 1, 0), 1), ((0, 0, 1, 1), 5), ((3, 1, 0, 0), 6)]:
        ld = lambda V: np.linalg.slogdet(_dense_mu_minus_Dt(V, p))[1]
        fd = (ld(FO.perturb(U, 3, site, a, +h)) - ld(FO.perturb(U, 3, site, a, -h))) / (2 * h)
        t, z, y, x = site
        assert abs(F[t, z, y, x, 3, a] - fd) < 2e-7 * max(1.0, abs(fd)), (site, a, fd)
    assert abs(F[..., 3, :]).max() > 1e-3  # the check above is not vacuous


def test_gauge_invariance():
    """log det(mu - D_t) is gauge invariant; the force of each link rotates, keeping its length."""
    p, U = _lattice(4, 6, -1, seed=51, kappa_s=0.1, xi=3.0)
    Ug = _gauge_transform(U, S.random_gauge_transform(4, 6, 52))
    a, b = DT.logdet_temporal(U, p), DT.logdet_temporal(Ug, p)
    assert abs(a - b) < 1e-12 * abs(a)
    na = np.linalg.norm(DT.force_logdet_temporal(U, p), axis=-1)
    nb = np.linalg.norm(DT.force_logdet_temporal(Ug, p), axis=-1)
    assert np.max(np.abs(na - nb)) < 1e-12 * np.max(na)
