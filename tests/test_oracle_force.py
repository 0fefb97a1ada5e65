"""Pins of the oracle's pseudofermion force (CPU only).

F_mu^a(x) = dS/d eps for U_mu(x) -> exp(i eps T_a) U_mu(x), S = phi^dag (M-hat^dag M-hat)^-1 phi,
is checked against central finite differences of S on random links (h = 1e-5), on a
degenerate 2^3 lattice and a 4^3 one, both boundary conditions. A planted mistake (one of
the six chain terms dropped) must fail the same comparison.
"""

import numpy as np
import pytest

import synthetic as S
from oracle import force as F
from oracle import wilson as W


def _setup(L, T, bc, seed):
    p = W.Params(L, T, 0.07, xi=3.0, bc=bc)
    U = S.random_gauge(L, T, 0.4, seed)
    phi = W.restrict(S.gaussian_source(L, T, seed + 50), W.parity3(L, T) == 1)
    return p, U, phi


def _samples(L, T, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        site = (int(rng.integers(0, T)), int(rng.integers(0, L)), int(rng.integers(0, L)), int(rng.integers(0, L)))
        out.append((int(rng.integers(0, 4)), site, int(rng.integers(0, 8))))
    # always include a time-boundary link and a spatial link of each direction
    out += [(3, (T - 1, 0, 0, 0), 3), (0, (0, 1, 0, 1), 1), (1, (1, 0, 1, 0), 5), (2, (2, 1, 1, 0), 7)]
    return out


@pytest.mark.parametrize("L,T,bc,seed", [(2, 4, -1, 3), (2, 6, 1, 4), (4, 4, -1, 5)])
def test_force_matches_finite_differences(L, T, bc, seed):
    p, U, phi = _setup(L, T, bc, seed)
    f = F.force(U, phi, p)
    for mu, site, a in _samples(L, T, 6, seed):
        fd = F.force_fd(U, phi, p, mu, site, a)
        assert abs(f[site + (mu, a)] - fd) < 5e-9 + 1e-6 * abs(fd), (mu, site, a, f[site + (mu, a)], fd)


def test_force_is_gauge_covariant_in_norm():
    """Under a gauge transformation the force rotates in the adjoint, so |F_mu(x)| per link is invariant."""
    p, U, phi = _setup(2, 4, -1, 6)
    g = S.random_gauge_transform(2, 4, 7)
    Ug = np.empty_like(U)
    for mu in range(4):
        gp = W.shift(g, mu, +1, 1.0)
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gp, -1, -2))
    f = F.force(U, phi, p)
    fg = F.force(Ug, W.colour(g, phi), p)
    assert np.allclose(np.linalg.norm(f, axis=-1), np.linalg.norm(fg, axis=-1), atol=1e-10)


def test_dropped_chain_term_is_caught(monkeypatch):
    orig = F._temporal_link_derivative_CR
    calls = {"n": 0}

    def drop_first(U, w, v, p):
        calls["n"] += 1
        z = orig(U, w, v, p)
        return z * 0 if calls["n"] == 1 else z

    monkeypatch.setattr(F, "_temporal_link_derivative_CR", drop_first)
    p, U, phi = _setup(2, 4, -1, 3)
    f = F.force(U, phi, p)
    bad = 0
    for mu, site, a in [(3, (0, 0, 0, 1), 0), (3, (1, 1, 0, 0), 2), (3, (2, 0, 1, 1), 4), (3, (3, 1, 1, 0), 6)]:
        fd = F.force_fd(U, phi, p, mu, site, a)
        bad += abs(f[site + (mu, a)] - fd) > 5e-9 + 1e-6 * abs(fd)
    assert bad > 0
