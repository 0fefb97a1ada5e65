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


# ---------------------------------------------------------------------------
# Full SW temporal preconditioning (§II.A, the paragraphs on SW fermions; appendix "Full
# Preconditioning with Clover"): the temporal block Q = A + mu - D_t of each spatial line is
# inverted whole. Any split C_L^-1 C_R^-1 = Q gives Q-bar = 1 and the form of Eq. TPrecFull; read
# here with the one-sided split C_L = Q^-1, C_R = 1:
#   M-hat_full = 1 - gamma_f^-2 (Q^oo)^-1 D_s^oe (Q^ee)^-1 D_s^eo   on odd 3-D sites.
# ---------------------------------------------------------------------------
def Q_apply(U, Acl, psi, p):
    """Q psi = (A + mu - D_t) psi (§II, Eq. for M without its D_s term)."""
    return apply_A(Acl, psi) + p.mu * psi - W.D_t(U, psi, p.bc)


def Q_line_matrix(U, Acl, p, x, y, z, wrap=True):
    """Dense 12 N_t x 12 N_t matrix of Q on the time line of spatial site (x, y, z), from the
    definitions: mu + A(t) on the diagonal, -P_- U_0(t) coupling t to t+1, -P_+ U_0(t-1)^dag
    coupling t to t-1, the wrap couplings carrying the boundary sign s (left out with wrap=False:
    the open chain T_0 of the appendix)."""
    T = p.T
    U0 = U[:, z, y, x, W.MU_T]
    Qm = np.zeros((12 * T, 12 * T), dtype=np.complex128)
    for t in range(T):
        blk = slice(12 * t, 12 * t + 12)
        Qm[blk, blk] = p.mu * np.eye(12) + Acl[t, z, y, x].reshape(12, 12)
        tn, tb = (t + 1) % T, (t - 1) % T
        if wrap or t < T - 1:
            sf = p.bc if t == T - 1 else 1.0
            Qm[blk, 12 * tn:12 * tn + 12] -= sf * np.kron(W.P_MINUS, U0[t])
        if wrap or t > 0:
            sb = p.bc if t == 0 else 1.0
            Qm[blk, 12 * tb:12 * tb + 12] -= sb * np.kron(W.P_PLUS, np.conj(U0[tb]).T)
    return Qm


def wrap_factors(U0_last, p):
    """V (12 N_t x 12) and W^dag (12 x 12 N_t) of the appendix with V W^dag the two wrap couplings:
    V_0 = -s P_+ U_0(N_t-1)^dag, V_{N_t-1} = -s P_- U_0(N_t-1), W^dag = (P_-, 0, ..., 0, P_+)."""
    T = p.T
    V = np.zeros((12 * T, 12), dtype=np.complex128)
    Wd = np.zeros((12, 12 * T), dtype=np.complex128)
    V[0:12] = -p.bc * np.kron(W.P_PLUS, np.conj(U0_last).T)
    V[12 * (T - 1):] = -p.bc * np.kron(W.P_MINUS, U0_last)
    Wd[:, 0:12] = np.kron(W.P_MINUS, np.eye(3))
    Wd[:, 12 * (T - 1):] = np.kron(W.P_PLUS, np.eye(3))
    return V, Wd


def Q_inverse(U, Acl, psi, p):
    """Q^-1 psi, one dense solve per spatial line (the plain definition)."""
    T, L = p.T, p.L
    out = np.zeros_like(psi)
    for z in range(L):
        for y in range(L):
            for x in range(L):
                rhs = psi[..., :, z, y, x, :, :]                      # (..., T, 4, 3)
                lead = rhs.shape[:-3]
                b = rhs.reshape(lead + (12 * T,))
                sol = np.linalg.solve(Q_line_matrix(U, Acl, p, x, y, z), b.reshape(-1, 12 * T).T).T
                out[..., :, z, y, x, :, :] = sol.reshape(lead + (T, 4, 3))
    return out


def Q_inverse_woodbury(U, Acl, psi, p):
    """Q^-1 psi by the appendix's single-step Woodbury form, line by line: Q = T_0 + V W^dag with
    T_0 the open chain (Q without its two wrap couplings) and V, W^dag from ``wrap_factors``;
    Q^-1 = T_0^-1 - T_0^-1 V (1 + W^dag T_0^-1 V)^-1 W^dag T_0^-1 (T_0 solved densely here; the paper
    uses an inner CG for it)."""
    T, L = p.T, p.L
    out = np.zeros_like(psi)
    for z in range(L):
        for y in range(L):
            for x in range(L):
                T0 = Q_line_matrix(U, Acl, p, x, y, z, wrap=False)
                V, Wd = wrap_factors(U[T - 1, z, y, x, W.MU_T], p)
                rhs = psi[..., :, z, y, x, :, :]
                lead = rhs.shape[:-3]
                b = rhs.reshape(lead + (12 * T,)).reshape(-1, 12 * T).T
                chi = np.linalg.solve(T0, b)
                T0V = np.linalg.solve(T0, V)
                lam = np.linalg.inv(np.eye(12) + Wd @ T0V)
                sol = chi - T0V @ (lam @ (Wd @ chi))
                out[..., :, z, y, x, :, :] = sol.T.reshape(lead + (T, 4, 3))
    return out


def M_hat_full_sw(U, Acl, psi_o, p, par3=None):
    """1 - gamma_f^-2 (Q^oo)^-1 D_s^oe (Q^ee)^-1 D_s^eo on odd 3-D sites."""
    if par3 is None:
        par3 = W.parity3(p.L, p.T)
    ev, od = par3 == 0, par3 == 1
    x = W.restrict(psi_o, od)
    t = W.restrict(Q_inverse(U, Acl, W.restrict(W.D_s(U, x), ev), p), ev)
    return x - W.restrict(Q_inverse(U, Acl, W.restrict(W.D_s(U, t), od), p), od) / p.gamma_f ** 2


def M_hat_full_sw_dag(U, Acl, psi_o, p, par3=None):
    """Adjoint of M-hat_full: gamma_5 [Q^oo - gamma_f^-2 D_s^oe (Q^ee)^-1 D_s^eo] (Q^oo)^-1 gamma_5
    (Q and D_s are gamma_5-hermitian)."""
    if par3 is None:
        par3 = W.parity3(p.L, p.T)
    ev, od = par3 == 0, par3 == 1
    g = W.restrict(W.spin(W.GAMMA5, psi_o), od)
    u = W.restrict(Q_inverse(U, Acl, g, p), od)
    t = W.restrict(Q_inverse(U, Acl, W.restrict(W.D_s(U, u), ev), p), ev)
    r = W.restrict(Q_apply(U, Acl, u, p), od) - W.restrict(W.D_s(U, t), od) / p.gamma_f ** 2
    return W.spin(W.GAMMA5, r)


def solve_full_sw(U, Acl, eta, p, tol=1e-10, maxiter=100000):
    """M_SW psi = eta with full SW temporal preconditioning and 3-D Schur: CGNR on
    M-hat_full psi_o = (Q^oo)^-1 (eta_o + gamma_f^-1 D_s^oe (Q^ee)^-1 eta_e), then
    psi_e = (Q^ee)^-1 (eta_e + gamma_f^-1 D_s^eo psi_o). Returns (psi, CG iterations, true residual)."""
    par3 = W.parity3(p.L, p.T)
    ev, od = par3 == 0, par3 == 1
    g = p.gamma_f
    eta_e, eta_o = W.restrict(eta, ev), W.restrict(eta, od)
    qe = W.restrict(Q_inverse(U, Acl, eta_e, p), ev)
    b = W.restrict(Q_inverse(U, Acl, eta_o + W.restrict(W.D_s(U, qe), od) / g, p), od)
    A = lambda v: M_hat_full_sw(U, Acl, v, p, par3)
    Ad = lambda v: M_hat_full_sw_dag(U, Acl, v, p, par3)
    inner, y, total, rel, psi = tol, None, 0, np.inf, None
    for _ in range(8):
        y, it, _ = SV.cgnr(A, Ad, b, x0=y, tol=inner, maxiter=maxiter - total)
        total += it
        psi_o = W.restrict(y, od)
        psi = W.restrict(Q_inverse(U, Acl, eta_e + W.restrict(W.D_s(U, psi_o), ev) / g, p), ev) + psi_o
        rel = true_residual(U, Acl, psi, eta, p)
        if rel <= tol or total >= maxiter:
            break
        inner *= 0.5 * tol / rel
    return psi, total, rel
