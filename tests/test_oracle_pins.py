"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: an identity the
paper states (mu - D_t = C_L^-1 C_R^-1, gamma_5 relation, S_L M S_R = diag(1, M-hat)),
a closed form (free-field spectrum, the SMW block X, Lambda), a library routine on a
dense matrix built from the definitions (inverse, Schur complement, linear solve,
singular values), or an invariance (gauge covariance).
"""

import numpy as np
import pytest

import synthetic as S
from oracle import dense as D
from oracle import flops as F
from oracle import solve as SV
from oracle import wilson as W


def _params(L=2, T=4, kappa_s=0.07, xi=3.0, bc=-1):
    return W.Params(L, T, kappa_s, xi=xi, bc=bc)


@pytest.fixture(scope="module")
def small():
    p = _params(2, 4)
    U = S.random_gauge(2, 4, 0.3, 11)
    eta = S.gaussian_source(2, 4, 12)
    return p, U, eta


@pytest.fixture(scope="module")
def medium():
    p = _params(4, 8, kappa_s=0.075, xi=3.5)
    U = S.random_gauge(4, 8, 0.3, 21)
    eta = S.gaussian_source(4, 8, 22)
    return p, U, eta


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _ip(a, b):
    return np.vdot(a.ravel(), b.ravel())


# --------------------------------------------------------------------------- spin algebra
def test_gamma_clifford_and_basis():
    """Euclidean Clifford algebra, hermiticity; gamma_t diagonal so P_+ / P_- pick upper / lower spins."""
    for m in range(4):
        assert np.allclose(W.GAMMA[m], W.GAMMA[m].conj().T)
        for n in range(4):
            ac = W.GAMMA[m] @ W.GAMMA[n] + W.GAMMA[n] @ W.GAMMA[m]
            assert np.allclose(ac, 2 * np.eye(4) * (m == n))
    assert np.allclose(W.P_PLUS, np.diag([1, 1, 0, 0]))
    assert np.allclose(W.P_MINUS, np.diag([0, 0, 1, 1]))
    assert np.allclose(W.GAMMA5, -np.block([[np.zeros((2, 2)), np.eye(2)], [np.eye(2), np.zeros((2, 2))]]))
    for m in range(4):
        assert np.allclose(W.GAMMA5 @ W.GAMMA[m], -W.GAMMA[m] @ W.GAMMA5)


# --------------------------------------------------------------------------- T and T^-1
@pytest.mark.parametrize("bc", [-1, 1])
def test_Tinv_matches_dense_inverse(bc):
    """SMW T^-1 and (T^dag)^-1 equal the library inverse of the dense T built from its definition."""
    p = _params(2, 6, bc=bc)
    U = S.random_gauge(2, 6, 0.5, 3)
    eta = S.gaussian_source(2, 6, 4)
    psi = W.Tinv(U, eta, p)
    psid = W.Tdag_inv(U, eta, p)
    for (x, y, z) in [(0, 0, 0), (1, 0, 1), (1, 1, 1)]:
        Td = D.temporal_matrix(U, p, x, y, z)
        for s in range(4):
            rhs = eta[:, z, y, x, s, :].reshape(-1)
            ref = np.linalg.solve(Td, rhs)
            assert np.allclose(psi[:, z, y, x, s, :].reshape(-1), ref, atol=1e-13, rtol=0)
            refd = np.linalg.solve(Td.conj().T, rhs)
            assert np.allclose(psid[:, z, y, x, s, :].reshape(-1), refd, atol=1e-13, rtol=0)


@pytest.mark.parametrize("bc", [-1, 1])
def test_Tinv_free_field_closed_form(bc):
    """Unit links: plane waves e^{i p0 t} are eigenvectors of T^-1 with eigenvalue 1/(mu - e^{i p0})."""
    T = 8
    p = _params(2, T, bc=bc)
    U = S.unit_gauge(2, T)
    rng = np.random.default_rng(0)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    for n in range(T):
        p0 = (2 * n + (1 if bc == -1 else 0)) * np.pi / T
        wave = np.exp(1j * p0 * np.arange(T))
        psi = wave[:, None, None, None, None, None] * np.broadcast_to(u, (T, 2, 2, 2, 4, 3))
        lam = 1.0 / (p.mu - np.exp(1j * p0))
        assert _rel(W.Tinv(U, psi, p), lam * psi) < 1e-13
        assert _rel(W.Tdag_inv(U, psi, p), np.conj(lam) * psi) < 1e-13


def test_smw_X_closed_form_and_cutoff_norm():
    """X(t) = -s mu^{-(N_t-t)} U_0(t)...U_0(N_t-1); ||X(t)||_F = sqrt(3) mu^{-(N_t-t)} (§II.A, Eq. cutoff)."""
    T = 6
    p = _params(2, T, bc=-1)
    U = S.random_gauge(2, T, 0.7, 8)
    X, Lam = W.smw_init(U, p)
    Xm = np.swapaxes(X, -1, -2)
    U0 = U[..., 3, :, :]
    for (x, y, z) in [(0, 0, 0), (1, 1, 0)]:
        prod = np.eye(3, dtype=complex)
        for t in range(T - 1, -1, -1):
            prod = U0[t, z, y, x] @ prod
            ref = -p.bc * p.mu ** (-(T - t)) * prod
            assert np.allclose(Xm[t, z, y, x], ref, atol=1e-15)
            assert np.isclose(np.linalg.norm(Xm[t, z, y, x]), np.sqrt(3) * p.mu ** (-(T - t)))
        # X(0) is the Polyakov loop up to -s mu^-N_t, so Lambda = (I - s mu^-N_t P)^-1
        P = prod
        assert np.allclose(Lam[z, y, x], np.linalg.inv(np.eye(3) - p.bc * p.mu ** (-T) * P))


def test_lambda_free_field():
    """Free field: Lambda = I / (1 - s mu^{-N_t})."""
    for bc in (-1, 1):
        p = _params(2, 4, bc=bc)
        _, Lam = W.smw_init(S.unit_gauge(2, 4), p)
        assert np.allclose(Lam, np.eye(3) / (1 - bc * p.mu ** (-4)))


def test_temporal_factorisation(medium):
    """mu - D_t = C_L^-1 C_R^-1 (§II.A, Eq. dt_clcr), and C_L, C_R invert C_L^-1, C_R^-1."""
    p, U, eta = medium
    lhs = p.mu * eta - W.D_t(U, eta, p.bc)
    rhs = W.C_L_inv(U, W.C_R_inv(U, eta, p), p)
    assert _rel(lhs, rhs) < 1e-14
    assert _rel(W.C_L(U, W.C_L_inv(U, eta, p), p), eta) < 1e-13
    assert _rel(W.C_R(U, W.C_R_inv(U, eta, p), p), eta) < 1e-13


def test_gamma5_relation(medium):
    """C_L^{dag -1} = gamma_5 C_R^-1 gamma_5 (§II.A): <a, C_L^-1 b> = <gamma_5 C_R^-1 gamma_5 a, b>."""
    p, U, eta = medium
    a = S.gaussian_source(p.L, p.T, 99)
    lhs = _ip(a, W.C_L_inv(U, eta, p))
    rhs = _ip(W.spin(W.GAMMA5, W.C_R_inv(U, W.spin(W.GAMMA5, a), p)), eta)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# --------------------------------------------------------------------------- M, D_s, D_t
def test_free_field_momentum_space():
    """Unit links: M e^{ipx} u = [mu - sum_mu w_mu (cos p_mu - i gamma_mu sin p_mu)] e^{ipx} u,
    with w_t = 1 and w_i = 1/gamma_f; eigenvalues a +- i sqrt(sum w^2 sin^2 p)."""
    L, T = 4, 8
    p = _params(L, T, kappa_s=0.08, xi=2.5, bc=-1)
    U = S.unit_gauge(L, T)
    rng = np.random.default_rng(1)
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    w = [1 / p.gamma_f] * 3 + [1.0]
    for trial in range(4):
        n = rng.integers(0, 8, size=4)
        pm = [2 * np.pi * n[0] / L, 2 * np.pi * n[1] / L, 2 * np.pi * n[2] / L, (2 * n[3] + 1) * np.pi / T]
        phase = np.exp(1j * (pm[0] * x + pm[1] * y + pm[2] * z + pm[3] * t))
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = phase[..., None, None] * u
        Mp = p.mu * np.eye(4) - sum(w[m] * (np.cos(pm[m]) * np.eye(4) - 1j * np.sin(pm[m]) * W.GAMMA[m])
                                   for m in range(4))
        ref = phase[..., None, None] * (Mp @ u)
        assert _rel(W.M(U, psi, p), ref) < 1e-13
        a = p.mu - sum(w[m] * np.cos(pm[m]) for m in range(4))
        b = np.sqrt(sum(w[m] ** 2 * np.sin(pm[m]) ** 2 for m in range(4)))
        ev = np.linalg.eigvals(Mp)
        assert np.allclose(ev.real, a, atol=1e-12)
        assert np.allclose(np.sort(ev.imag), [-b, -b, b, b], atol=1e-12)


def test_gamma5_hermiticity(medium):
    """Random gauge field: <a, M b> = <gamma_5 M gamma_5 a, b>, and the same for M~, M-hat, M-hat_4."""
    p, U, eta = medium
    a = S.gaussian_source(p.L, p.T, 98)
    par3, par4 = W.parity3(p.L, p.T), W.parity4(p.L, p.T)
    for op, opd, mask in [(W.M, W.M_dag, None), (W.M_tilde, W.M_tilde_dag, None),
                          (lambda U_, v, p_: W.M_hat(U_, v, p_, par3), lambda U_, v, p_: W.M_hat_dag(U_, v, p_, par3), par3 == 1),
                          (lambda U_, v, p_: W.M_hat4(U_, v, p_, par4), lambda U_, v, p_: W.M_hat4_dag(U_, v, p_, par4), par4 == 1)]:
        aa = a if mask is None else W.restrict(a, mask)
        bb = eta if mask is None else W.restrict(eta, mask)
        lhs = _ip(aa, op(U, bb, p))
        rhs = _ip(opd(U, aa, p), bb)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _gauge_transform(U, g, bc_unused=None):
    """U_mu(x) -> g(x) U_mu(x) g(x + mu)^dag with periodic g."""
    Ug = np.empty_like(U)
    for mu in range(4):
        gp = W.shift(g, mu, +1, 1.0)
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gp, -1, -2))
    return Ug


def test_gauge_covariance(medium):
    """M[U^g] (g psi) = g M[U] psi, and the same for T^-1, C_L, C_R and M-hat."""
    p, U, eta = medium
    g = S.random_gauge_transform(p.L, p.T, 5)
    Ug = _gauge_transform(U, g)
    geta = W.colour(g, eta)
    assert _rel(W.M(Ug, geta, p), W.colour(g, W.M(U, eta, p))) < 1e-13
    assert _rel(W.Tinv(Ug, geta, p), W.colour(g, W.Tinv(U, eta, p))) < 1e-13
    assert _rel(W.C_R(Ug, geta, p), W.colour(g, W.C_R(U, eta, p))) < 1e-13
    par3 = W.parity3(p.L, p.T)
    xo = W.restrict(eta, par3 == 1)
    assert _rel(W.M_hat(Ug, W.colour(g, xo), p, par3), W.colour(g, W.M_hat(U, xo, p, par3))) < 1e-13


# --------------------------------------------------------------------------- Schur operators
def test_tprec_full_block_form(medium):
    """S_L M S_R = diag(1, 1 - gamma_f^-2 D-bar^{oe} D-bar^{eo}) for Wilson (§II.B, Eq. TPrecFull)."""
    p, U, eta = medium
    par3 = W.parity3(p.L, p.T)
    lhs = W.S_L(U, W.M(U, W.S_R(U, eta, p, par3), p), p, par3)
    rhs = W.restrict(eta, par3 == 0) + W.M_hat(U, eta, p, par3)
    assert _rel(lhs, rhs) < 1e-13


def _dense_blocks(U, p, par):
    Md = D.matrix(lambda v: W.M(U, v, p), p.L, p.T)
    sel = np.broadcast_to(par[..., None, None], (p.T, p.L, p.L, p.L, 4, 3)).ravel()
    e, o = np.flatnonzero(sel == 0), np.flatnonzero(sel == 1)
    return Md, e, o


def test_Mhat_is_dense_schur_complement(small):
    """M-hat = C_L^o [M^oo - M^oe (M^ee)^-1 M^eo] C_R^o with p_3 ordering (§II.B), C's from dense inverses."""
    p, U, _ = small
    par3 = W.parity3(p.L, p.T)
    Md, e, o = _dense_blocks(U, p, par3)
    schur = Md[np.ix_(o, o)] - Md[np.ix_(o, e)] @ np.linalg.solve(Md[np.ix_(e, e)], Md[np.ix_(e, o)])
    CLinv = D.matrix(lambda v: W.C_L_inv(U, v, p), p.L, p.T, par3 == 1, par3 == 1)
    CRinv = D.matrix(lambda v: W.C_R_inv(U, v, p), p.L, p.T, par3 == 1, par3 == 1)
    ref = np.linalg.inv(CLinv) @ schur @ np.linalg.inv(CRinv)
    Mh = D.matrix(lambda v: W.M_hat(U, v, p, par3), p.L, p.T, par3 == 1, par3 == 1)
    assert np.abs(Mh - ref).max() < 1e-13 * np.abs(ref).max()


def test_Mhat4_is_dense_schur_complement(small):
    """M-hat_4 = M^oo - M^oe (M^ee)^-1 M^eo with p_4 ordering (§II.B, 4D-Schur)."""
    p, U, _ = small
    par4 = W.parity4(p.L, p.T)
    Md, e, o = _dense_blocks(U, p, par4)
    schur = Md[np.ix_(o, o)] - Md[np.ix_(o, e)] @ np.linalg.solve(Md[np.ix_(e, e)], Md[np.ix_(e, o)])
    Mh4 = D.matrix(lambda v: W.M_hat4(U, v, p, par4), p.L, p.T, par4 == 1, par4 == 1)
    assert np.abs(Mh4 - schur).max() < 1e-13 * np.abs(schur).max()


# --------------------------------------------------------------------------- solves
@pytest.mark.parametrize("method", SV.METHODS)
def test_solve_matches_dense_solve(small, method):
    """Every method reaches the unique solution of M psi = eta (dense LU) with true residual <= 1e-10."""
    p, U, eta = small
    Md = D.matrix(lambda v: W.M(U, v, p), p.L, p.T)
    ref = np.linalg.solve(Md, eta.ravel()).reshape(eta.shape)
    psi, it, rel = SV.solve(U, eta, p, method, tol=1e-10)
    assert rel <= 1e-10
    assert it > 0
    assert _rel(psi, ref) < 1e-8


def test_cgnr_on_dense_spd():
    """CGNR on a small dense system converges to the library solve."""
    rng = np.random.default_rng(3)
    A = np.eye(20) * 3 + 0.3 * (rng.standard_normal((20, 20)) + 1j * rng.standard_normal((20, 20)))
    b = rng.standard_normal(20) + 1j * rng.standard_normal(20)
    x, it, rel = SV.cgnr(lambda v: A @ v, lambda v: A.conj().T @ v, b, tol=1e-12)
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-10)


# --------------------------------------------------------------------------- conditioning
def _sigma_ratios(U, p):
    par3, par4 = W.parity3(p.L, p.T), W.parity4(p.L, p.T)
    r = {}
    r["unprec"] = D.sigma_ratio(D.matrix(lambda v: W.M(U, v, p), p.L, p.T))
    r["temporal"] = D.sigma_ratio(D.matrix(lambda v: W.M_tilde(U, v, p), p.L, p.T))
    r["eo4d"] = D.sigma_ratio(D.matrix(lambda v: W.M_hat4(U, v, p, par4), p.L, p.T, par4 == 1, par4 == 1))
    r["temporal_schur"] = D.sigma_ratio(D.matrix(lambda v: W.M_hat(U, v, p, par3), p.L, p.T, par3 == 1, par3 == 1))
    return r


def test_condition_ordering_anisotropic():
    """xi = 3, subcritical: kappa(unprec) > kappa(temporal), kappa(unprec) > kappa(4D eo) > kappa(temporal+Schur)."""
    p = _params(2, 4, kappa_s=0.07, xi=3.0)
    U = S.random_gauge(2, 4, 0.3, 1)
    r = _sigma_ratios(U, p)
    assert r["unprec"] > r["temporal"]
    assert r["unprec"] > r["eo4d"] > r["temporal_schur"]


def test_condition_isotropic_no_gain():
    """xi = 1 (§III.D: the paper finds no gain for isotropic lattices): kappa(temporal+Schur) >= kappa(4D eo)."""
    p = W.Params(2, 8, 0.11, kappa_t=0.11, bc=-1)
    U = S.random_gauge(2, 8, 0.3, 2)
    r = _sigma_ratios(U, p)
    assert r["temporal_schur"] >= r["eo4d"]


def test_condition_gauge_invariant():
    """Singular values, hence condition numbers, do not change under a random gauge transformation."""
    p = _params(2, 4, kappa_s=0.07, xi=3.0)
    U = S.random_gauge(2, 4, 0.3, 1)
    Ug = _gauge_transform(U, S.random_gauge_transform(2, 4, 9))
    a, b = _sigma_ratios(U, p), _sigma_ratios(Ug, p)
    for k in a:
        assert abs(a[k] - b[k]) < 1e-12 * a[k]


# --------------------------------------------------------------------------- FLOP model
def _golden(root):
    rows = {}
    with open(f"{root}/tests/golden/flop_model.txt") as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            vals = []
            for tok in parts[1:]:
                try:
                    vals.append(int(tok))
                except ValueError:
                    break
            rows[parts[0]] = vals
    return rows


def test_flop_model_matches_paper(root_dir):
    """The FLOP model rebuilt from unit costs gives the totals printed in App. B and App. C."""
    g = _golden(root_dir)
    assert F.dslash_site(4) == g["dslash4_site"][0]
    assert F.dslash_site(3) == g["dslash3_site"][0]
    lin = {
        "backsub": F.backsub, "woodbury": F.woodbury, "precond_per_line": F.c_precond_per_line,
        "clover_4d_schur_per_line": F.clover_4d_schur_per_line,
        "clover_temporal_ilu_per_line": F.clover_temporal_ilu_per_line,
        "wilson_4d_schur_per_line": F.wilson_4d_schur_per_line,
        "wilson_temporal_schur_per_line": F.wilson_temporal_schur_per_line,
        "wilson_temporal_schur_tricks_per_line": F.wilson_temporal_schur_tricks_per_line,
        "wilson_4d_schur_tricks_per_line": F.wilson_4d_schur_tricks_per_line,
    }
    for name, fn in lin.items():
        a, b = g[name]
        for nt in (1, 16, 128):
            assert fn(nt) == a * nt + b, name
