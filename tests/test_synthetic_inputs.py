"""The seeded input generators shared by the oracle and the GPU path (no method arithmetic).

Pins: links and gauge transformations are SU(3) to rounding; small eps gives links near the unit
matrix with the spread of exp(i eps H); the generators are reproducible from their seeds and the
point sources are the 12 spin-colour unit vectors at site 0; the workloads' couplings sit below
the free critical point except the deliberately supercritical 4^3 x 16 one.
"""

import numpy as np
import pytest

import synthetic as S


def _su3_defects(u):
    m = u.reshape(-1, 3, 3)
    unit = np.abs(np.einsum("nij,nkj->nik", m, m.conj()) - np.eye(3)).max()
    det = np.abs(np.linalg.det(m) - 1.0).max()
    return unit, det


def test_gell_mann_normalisation():
    lam = S.gell_mann()
    assert lam.shape == (8, 3, 3)
    for a in range(8):
        assert np.allclose(lam[a], lam[a].conj().T)
        assert abs(np.trace(lam[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(lam[a] @ lam[b]) - 2.0 * (a == b)) < 1e-14


@pytest.mark.parametrize("eps", [0.0, 0.2, 1.0])
def test_random_gauge_is_su3(eps):
    U = S.random_gauge(4, 6, eps, 11)
    assert U.shape == (6, 4, 4, 4, 4, 3, 3)
    unit, det = _su3_defects(U)
    assert unit < 1e-14 and det < 1e-14


def test_small_eps_links_are_near_unity():
    U = S.random_gauge(4, 8, 0.05, 12).reshape(-1, 3, 3)
    dev = np.linalg.norm(U - np.eye(3), axis=(1, 2))
    # |exp(i eps H) - 1| ~ eps |H|, |H|_F^2 = sum_a h_a^2 / 2 with E = 4: mean about eps sqrt(4)
    assert 0.03 < dev.mean() < 0.15
    assert dev.max() < 0.5


def test_gauge_transform_is_su3():
    g = S.random_gauge_transform(4, 6, 13)
    unit, det = _su3_defects(g)
    assert unit < 1e-14 and det < 1e-14


def test_generators_are_reproducible():
    assert np.array_equal(S.random_gauge(2, 4, 0.3, 7), S.random_gauge(2, 4, 0.3, 7))
    assert not np.array_equal(S.random_gauge(2, 4, 0.3, 7), S.random_gauge(2, 4, 0.3, 8))
    a = S.gaussian_source(2, 4, 9, nrhs=3)
    assert np.array_equal(a, S.gaussian_source(2, 4, 9, nrhs=3))


def test_gaussian_source_statistics():
    eta = S.gaussian_source(8, 16, 21)
    assert eta.shape == (16, 8, 8, 8, 4, 3)
    # Re, Im ~ N(0, 1/2): E|eta|^2 = 1 per component
    assert abs(np.mean(np.abs(eta) ** 2) - 1.0) < 0.02
    assert abs(np.mean(eta.real)) < 0.01 and abs(np.mean(eta.imag)) < 0.01


def test_point_sources():
    eta = S.point_sources(2, 4)
    assert eta.shape == (12, 4, 2, 2, 2, 4, 3)
    for k in range(12):
        s, c = divmod(k, 3)
        assert eta[k, 0, 0, 0, 0, s, c] == 1.0
        assert np.count_nonzero(eta[k]) == 1


def test_workload_couplings():
    for name, w in S.WORKLOADS.items():
        assert w["kappa_t"] == pytest.approx(w["xi"] * w["kappa_s"])
        kc = S.kappa_critical_free(w["xi"])
        if name == "wilson_4c16_xi3":
            assert w["kappa_s"] > kc  # the literal supercritical couplings of the smallest workload
        else:
            assert w["kappa_s"] < kc
    assert S.kappa_critical_free(3.5) == pytest.approx(1.0 / 13.0)
