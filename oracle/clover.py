"""FP64 oracle of the clover (SW) operator with partial temporal preconditioning and 3-D ILU.

TEST INFRASTRUCTURE ONLY (see ``oracle/wilson.py``).

§II: the SW fermion matrix is M_SW = A + mu - D_t - D_s / gamma_f, the Wilson matrix plus the
site-diagonal clover term

    A(x) = -[ (c_t / 2) sum_i sigma_i0 F_i0(x) + (c_s / 2) sum_{i<j} sigma_ij F_ij(x) ],
    sigma_mu nu = [gamma_mu, gamma_nu] / 2,

with F_mu nu(x) the anti-hermitian clover-leaf field strength. §II.B: "partial" temporal
preconditioning keeps the Wilson C_L, C_R (and so the Wilson S_L, S_R); applied to M_SW they
give Eq. TPrecPartial,

    M-tilde_ILU = S_L M_SW S_R = [[1 + Abar^ee,            gamma_f^-1 Abar^ee Dbar^eo],
                                  [gamma_f^-1 Dbar^oe Abar^ee, 1 + Abar^oo - gamma_f^-2 Dbar^oe (1 - Abar^ee) Dbar^eo]],

Abar = C_L A C_R, Dbar = C_L D_s C_R, which App. B applies as the sequence t_1 = Dbar^eo psi_o,
t_2 = Abar^ee (t_1 + psi_e), chi_e = psi_e + t_2, chi_o = psi_o + Abar^oo psi_o + Dbar^oe (t_2 - t_1)
(the gamma_f factors, which App. B absorbs into Dbar, written out here). M_SW psi = eta is solved
as M-tilde_ILU y = S_L eta, psi = S_R y.

Readings where the paper is brief (each pinned in ``tests/test_oracle_clover.py``):
* F_mu nu(x) = [Q_mu nu(x) - Q_mu nu(x)^dag] / 8 with its trace removed, Q the sum of the four
  plaquette leaves in the mu nu plane that start and end at x, all with the orientation of
  U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag;
* the spatial sum runs over the three planes i < j, one term per plane like the temporal sum;
* c_s and c_t are inputs (Eq. ClovCoeffs gives them from the tadpole factor u_s, gamma_g, gamma_f, xi).
"""

import numpy as np

from . import solve as SV
from . import wilson as W

SPATIAL_PLANES = ((0, 1), (0, 2), (1, 2))
TEMPORAL_PLANES = ((0, 3), (1, 3), (2, 3))


def sigma(mu, nu):
    """sigma_mu nu = [gamma_mu, gamma_nu] / 2 (4x4, Dirac-Pauli basis of ``oracle/wilson.py``)."""
    return 0.5 * (W.GAMMA[mu] @ W.GAMMA[nu] - W.GAMMA[nu] @ W.GAMMA[mu])


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def _sh(f, mu, step):
    """f(x + step * mu) for a link or matrix field (periodic: the gauge field has no boundary sign)."""
    return W.shift(f, mu, step, 1.0)


def clover_leaves(U, mu, nu):
    """Q_mu nu(x): the four plaquettes in the mu nu plane that start and end at x, one orientation.

    Link and matrix fields have shape (T, L, L, L, 3, 3).
    """
    Um, Un = W.link(U, mu), W.link(U, nu)
    q = Um @ _sh(Un, mu, 1) @ _dag(_sh(Um, nu, 1)) @ _dag(Un)                       # x -> x+mu -> x+mu+nu -> x+nu -> x
    Um_m, Un_m = _sh(Um, mu, -1), _sh(Un, mu, -1)
    q = q + Un @ _dag(_sh(Um_m, nu, 1)) @ _dag(Un_m) @ Um_m                          # x -> x+nu -> x-mu+nu -> x-mu -> x
    Um_mn = _sh(Um_m, nu, -1)
    q = q + _dag(Um_m) @ _dag(_sh(Un_m, nu, -1)) @ Um_mn @ _sh(Un, nu, -1)           # x -> x-mu -> x-mu-nu -> x-nu -> x
    Un_n = _sh(Un, nu, -1)
    q = q + _dag(Un_n) @ _sh(Um, nu, -1) @ _sh(Un_n, mu, 1) @ _dag(Um)               # x -> x-nu -> x-nu+mu -> x+mu -> x
    return q


def field_strength(U, mu, nu):
    """F_mu nu(x) = (Q - Q^dag) / 8 with the trace removed: anti-hermitian and traceless."""
    Q = clover_leaves(U, mu, nu)
    F = (Q - _dag(Q)) / 8.0
    tr = np.trace(F, axis1=-2, axis2=-1)
    return F - tr[..., None, None] * np.eye(3) / 3.0


def clover_term(U, c_s, c_t):
    """A(x) as a (T, L, L, L, 4, 3, 4, 3) array [.., spin, colour, spin', colour'] (§II, Eq. for A)."""
    A = np.zeros(U.shape[:4] + (4, 3, 4, 3), dtype=np.complex128)
    for (i, j) in SPATIAL_PLANES:
        A -= 0.5 * c_s * np.einsum("ab,...cd->...acbd", sigma(i, j), field_strength(U, i, j))
    for (i, t) in TEMPORAL_PLANES:
        A -= 0.5 * c_t * np.einsum("ab,...cd->...acbd", sigma(i, t), field_strength(U, i, t))
    return A


def apply_A(Acl, psi):
    """(A psi)(x) = A(x) psi(x); psi of shape (..., T, L, L, L, 4, 3)."""
    return np.einsum("tzyxacbd,...tzyxbd->...tzyxac", Acl, psi)


def M_sw(U, Acl, psi, p):
    """M_SW = A + mu - D_t - D_s / gamma_f (§II)."""
    return W.M(U, psi, p) + apply_A(Acl, psi)


def M_sw_dag(U, Acl, psi, p):
    """M_SW^dag = gamma_5 M_SW gamma_5 (A is hermitian and commutes with gamma_5)."""
    return W.spin(W.GAMMA5, M_sw(U, Acl, W.spin(W.GAMMA5, psi), p))


def Abar(U, Acl, psi, p, par, par3):
    """Abar^{pp} = C_L^p A^pp C_R^p on the sites of 3-D parity ``par`` (§II.B notation K-bar)."""
    m = par3 == par
    return W.restrict(W.C_L(U, apply_A(Acl, W.restrict(W.C_R(U, W.restrict(psi, m), p), m)), p), m)


def M_ilu(U, Acl, psi, p, par3=None):
    """M-tilde_ILU psi by the sequence of App. B (both 3-D parities)."""
    if par3 is None:
        par3 = W.parity3(p.L, p.T)
    ev, od = par3 == 0, par3 == 1
    psi_e, psi_o = W.restrict(psi, ev), W.restrict(psi, od)
    t1 = W.Dbar_s(U, psi_o, p, 0, par3) / p.gamma_f
    t2 = Abar(U, Acl, t1 + psi_e, p, 0, par3)
    chi_e = psi_e + t2
    chi_o = psi_o + Abar(U, Acl, psi_o, p, 1, par3) + W.Dbar_s(U, t2 - t1, p, 1, par3) / p.gamma_f
    return chi_e + chi_o


def M_ilu_dag(U, Acl, psi, p, par3=None):
    """M-tilde_ILU^dag = gamma_5 M-tilde_ILU gamma_5 (S_R^dag = gamma_5 S_L gamma_5, M_SW gamma_5-hermitian)."""
    return W.spin(W.GAMMA5, M_ilu(U, Acl, W.spin(W.GAMMA5, psi), p, par3))


def true_residual(U, Acl, psi, eta, p):
    """||eta - M_SW psi||_2 / ||eta||_2 in FP64."""
    r = eta - M_sw(U, Acl, psi, p)
    return float(np.sqrt(np.vdot(r.ravel(), r.ravel()).real / np.vdot(eta.ravel(), eta.ravel()).real))


def solve(U, Acl, eta, p, tol=1e-10, maxiter=100000):
    """M_SW psi = eta by CGNR on M-tilde_ILU y = S_L eta, psi = S_R y (§II.B, partial preconditioning).

    The inner tolerance is tightened (restarting from the current iterate) until the FP64 true
    residual of M_SW is at most ``tol``. Returns (psi, CG iterations, true relative residual).
    """
    par3 = W.parity3(p.L, p.T)
    A = lambda v: M_ilu(U, Acl, v, p, par3)
    Ad = lambda v: M_ilu_dag(U, Acl, v, p, par3)
    b = W.S_L(U, eta, p, par3)
    inner, y, total, rel, psi = tol, None, 0, np.inf, None
    for _ in range(8):
        y, it, _ = SV.cgnr(A, Ad, b, x0=y, tol=inner, maxiter=maxiter - total)
        total += it
        psi = W.S_R(U, y, p, par3)
        rel = true_residual(U, Acl, psi, eta, p)
        if rel <= tol or total >= maxiter:
            break
        inner *= 0.5 * tol / rel
    return psi, total, rel


# ---------------------------------------------------------------------------
# The 4-D Schur (even-odd) clover operator: the paper's comparator for the clover case (§II.B,
# first display; App. B counts its apply as 2 (C(D) + C(A^-1)) per site pair)
# ---------------------------------------------------------------------------
def mu_plus_A(Acl, p):
    """mu + A(x) per site, (T, L, L, L, 4, 3, 4, 3)."""
    one = np.einsum("ab,cd->acbd", np.eye(4), np.eye(3))
    return p.mu * one + Acl


def mu_plus_A_inv(Acl, p):
    """(mu + A(x))^-1 per site (dense 12 x 12 inverse), (T, L, L, L, 4, 3, 4, 3)."""
    B = mu_plus_A(Acl, p)
    sh = B.shape
    return np.linalg.inv(B.reshape(sh[:4] + (12, 12))).reshape(sh)


def M_hat4_sw(U, Acl, psi_o, p, par4=None):
    """(mu + A)^oo - D_w^oe (mu + A)^-1_ee D_w^eo on odd-p_4 sites (D_w = D_t + D_s / gamma_f)."""
    if par4 is None:
        par4 = W.parity4(p.L, p.T)
    ev, od = par4 == 0, par4 == 1
    x = W.restrict(psi_o, od)
    he = W.restrict(W.D_w(U, x, p), ev)
    he = apply_A(mu_plus_A_inv(Acl, p), he)
    return W.restrict(apply_A(mu_plus_A(Acl, p), x) - W.D_w(U, he, p), od)


def M_hat4_sw_dag(U, Acl, psi_o, p, par4=None):
    return W.spin(W.GAMMA5, M_hat4_sw(U, Acl, W.spin(W.GAMMA5, psi_o), p, par4))


def solve_eo4d(U, Acl, eta, p, tol=1e-10, maxiter=100000):
    """M_SW psi = eta by CGNR on the 4-D Schur operator: b_o = eta_o + D_w^oe (mu + A)^-1_ee eta_e,
    psi_e = (mu + A)^-1_ee (eta_e + D_w^eo psi_o). Returns (psi, CG iterations, true relative residual)."""
    par4 = W.parity4(p.L, p.T)
    ev, od = par4 == 0, par4 == 1
    Minv = mu_plus_A_inv(Acl, p)
    eta_e = W.restrict(eta, ev)
    b = W.restrict(eta, od) + W.restrict(W.D_w(U, apply_A(Minv, eta_e), p), od)
    A = lambda v: M_hat4_sw(U, Acl, v, p, par4)
    Ad = lambda v: M_hat4_sw_dag(U, Acl, v, p, par4)
    inner, y, total, rel, psi = tol, None, 0, np.inf, None
    for _ in range(8):
        y, it, _ = SV.cgnr(A, Ad, b, x0=y, tol=inner, maxiter=maxiter - total)
        total += it
        psi_o = W.restrict(y, od)
        psi = apply_A(Minv, W.restrict(eta_e + W.D_w(U, psi_o, p), ev)) + psi_o
        rel = true_residual(U, Acl, psi, eta, p)
        if rel <= tol or total >= maxiter:
            break
        inner *= 0.5 * tol / rel
    return psi, total, rel
