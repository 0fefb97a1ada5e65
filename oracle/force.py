"""FP64 oracle of the pseudofermion force of the temporally preconditioned operator.

TEST INFRASTRUCTURE ONLY (see ``oracle/wilson.py``).

The paper proposes carrying the preconditioner into hybrid Monte Carlo (§IV, last
paragraph) without working it out. The hot path needs the force of the pseudofermion
action of the temporal + 3-D Schur operator,

    S(U) = phi^dag (M-hat^dag M-hat)^-1 phi,     phi on odd 3-D parity sites,

with respect to every link U_mu(x) -> exp(i eps T_a) U_mu(x), T_a = lambda_a / 2:

    F_mu^a(x) = dS / d eps at eps = 0.

With X = (M-hat^dag M-hat)^-1 phi and Y = M-hat X one has dS = -2 Re(Y^dag dM-hat X). M-hat =
1 - gamma_f^-2 C_L^o D_s^oe C_R^e C_L^e D_s^eo C_R^o (§II.B, Eq. TPrecFull), so dM-hat is the sum
of six terms, each with one factor differentiated:
  * a hopping factor D_s: for a link U_k(x) the derivative of w^dag D_s v is
    Tr[i T_a (Q - R)], Q = sum_spin (U v(x+k)) (P^-_k w(x))^dag, R = sum_spin v(x) (U P^+_k w(x+k))^dag;
  * a temporal factor: C_L = P_+ + P_- T^-1 and C_R = P_- + P_+ T^-dag, with
    d(T^-1) = -T^-1 dT T^-1, and (dT chi)(t) = -dU_0(t) chi(t+1) (sign s across the wrap).
The derivative of S is the sum of these traces over the six (left vector, right vector)
pairs of the chain, times 2 gamma_f^-2. This module evaluates them in plain NumPy and is
pinned against central finite differences of S (``tests/test_oracle_force.py``).
"""

import numpy as np

from . import solve as SV
from . import wilson as W

LAMBDA = None


def generators():
    """T_a = lambda_a / 2, the su(3) generators of the link perturbation."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return lam / 2


def action(U, phi_o, p, tol=1e-13):
    """S = phi^dag (M-hat^dag M-hat)^-1 phi (phi on odd 3-D parity sites, full-lattice array)."""
    X = normal_solve(U, phi_o, p, tol)
    return float(np.real(np.vdot(phi_o.ravel(), X.ravel())))


def normal_solve(U, phi_o, p, tol=1e-13, maxiter=100000):
    """X = (M-hat^dag M-hat)^-1 phi by CG on the normal operator."""
    par3 = W.parity3(p.L, p.T)
    A = lambda v: W.M_hat_dag(U, W.M_hat(U, v, p, par3), p, par3)
    b = W.restrict(phi_o, par3 == 1)
    x = np.zeros_like(b)
    r = b.copy()
    pd = r.copy()
    rr = np.vdot(r.ravel(), r.ravel()).real
    bn = np.sqrt(rr)
    for _ in range(maxiter):
        if np.sqrt(rr) <= tol * bn:
            break
        q = A(pd)
        alpha = rr / np.vdot(pd.ravel(), q.ravel()).real
        x = x + alpha * pd
        r = r - alpha * q
        rr_new = np.vdot(r.ravel(), r.ravel()).real
        pd = r + (rr_new / rr) * pd
        rr = rr_new
    return x


def _outer(a, b):
    """sum over spin of a_s b_s^dag: (..., 4, 3) x (..., 4, 3) -> (..., 3, 3)."""
    return np.einsum("...sa,...sb->...ab", a, b.conj())


def _hop_link_derivative(U, w, v, k):
    """Z_k(x) with d(w^dag D_s v)/d eps_a(k, x) = Tr[i T_a Z_k(x)] for the spatial direction k."""
    Uk = W.link(U, k)
    Pm = 0.5 * (W.I4 - W.GAMMA[k])
    Pp = 0.5 * (W.I4 + W.GAMMA[k])
    v_fwd = W.shift(v, k, +1, 1.0)               # v(x + k)
    w_fwd = W.shift(w, k, +1, 1.0)               # w(x + k)
    Q = _outer(W.colour(Uk, v_fwd), W.spin(Pm, w))
    R = _outer(v, W.colour(Uk, W.spin(Pp, w_fwd)))
    return Q - R


def _temporal_link_derivative_CL(U, w, v, p):
    """Z_0(x) with d(w^dag C_L v) = Tr[i T_a Z_0]: a = T^-dag P_- w, b = T^-1 P_- v,
    Z_0(t) = s(t) sum_spin (U_0(t) b(t+1)) a(t)^dag."""
    a = W.Tdag_inv(U, W.spin(W.P_MINUS, w), p)
    b = W.Tinv(U, W.spin(W.P_MINUS, v), p)
    U0 = W.link(U, W.MU_T)
    return _outer(W.colour(U0, W.shift(b, W.MU_T, +1, p.bc)), a)


def _temporal_link_derivative_CR(U, w, v, p):
    """Z_0(x) with d(w^dag C_R v) = Tr[i T_a Z_0]: c = T^-1 P_+ w, e = T^-dag P_+ v,
    Z_0(t) = -s(t) sum_spin e(t) (U_0(t) c(t+1))^dag."""
    c = W.Tinv(U, W.spin(W.P_PLUS, w), p)
    e = W.Tdag_inv(U, W.spin(W.P_PLUS, v), p)
    U0 = W.link(U, W.MU_T)
    return -_outer(e, W.colour(U0, W.shift(c, W.MU_T, +1, p.bc)))


def force(U, phi_o, p, tol=1e-13):
    """F[t, z, y, x, mu, a] = dS / d eps for U_mu(x) -> exp(i eps T_a) U_mu(x), FP64."""
    par3 = W.parity3(p.L, p.T)
    ev, od = par3 == 0, par3 == 1
    X = normal_solve(U, phi_o, p, tol)
    Y = W.M_hat(U, X, p, par3)
    R = lambda f, m: W.restrict(f, m)
    dag5 = lambda f: W.spin(W.GAMMA5, f)
    # right chain v_k and left chain w_k of M-hat = 1 - gamma_f^-2 C_L^o D^oe C_R^e C_L^e D^eo C_R^o
    v0 = R(X, od)
    v1 = R(W.C_R(U, v0, p), od)
    v2 = R(W.D_s(U, v1), ev)
    v3 = R(W.C_L(U, v2, p), ev)
    v4 = R(W.C_R(U, v3, p), ev)
    w0 = R(Y, od)
    w1 = R(W.spin(W.P_PLUS, w0) + W.spin(W.P_MINUS, W.Tdag_inv(U, w0, p)), od)   # C_L^dag = P_+ + P_- T^-dag
    w2 = R(dag5(W.D_s(U, dag5(w1))), ev)                                          # D_s^dag = gamma_5 D_s gamma_5
    w3 = R(W.spin(W.P_MINUS, w2) + W.spin(W.P_PLUS, W.Tinv(U, w2, p)), ev)      # C_R^dag = P_- + P_+ T^-1
    w4 = R(W.spin(W.P_PLUS, w3) + W.spin(W.P_MINUS, W.Tdag_inv(U, w3, p)), ev)
    w5 = R(dag5(W.D_s(U, dag5(w4))), od)
    v5 = R(W.D_s(U, v4), od)
    Z = np.zeros(U.shape, dtype=np.complex128)
    # temporal factors: (w0, v5) C_L^o, (w2, v3) C_R^e, (w3, v2) C_L^e, (w5, v0) C_R^o
    Z[..., W.MU_T, :, :] += _temporal_link_derivative_CL(U, w0, v5, p)
    Z[..., W.MU_T, :, :] += _temporal_link_derivative_CR(U, w2, v3, p)
    Z[..., W.MU_T, :, :] += _temporal_link_derivative_CL(U, w3, v2, p)
    Z[..., W.MU_T, :, :] += _temporal_link_derivative_CR(U, w5, v0, p)
    # hopping factors: (w1, v4) D^oe and (w4, v1) D^eo
    for k in range(3):
        Z[..., k, :, :] += _hop_link_derivative(U, w1, v4, k) + _hop_link_derivative(U, w4, v1, k)
    # dS = -2 Re(Y^dag dM-hat X) and dM-hat = -gamma_f^-2 (sum of the six terms)
    Ta = generators()
    return 2.0 / p.gamma_f ** 2 * np.real(np.einsum("aij,...ji->...a", 1j * Ta, Z))


def perturb(U, mu, site, a, h):
    """U with U_mu(site) -> exp(i h T_a) U_mu(site); site = (t, z, y, x)."""
    Ta = generators()[a]
    w, v = np.linalg.eigh(Ta)
    E = (v * np.exp(1j * h * w)) @ v.conj().T
    Up = U.copy()
    t, z, y, x = site
    Up[t, z, y, x, mu] = E @ U[t, z, y, x, mu]
    return Up


def force_fd(U, phi_o, p, mu, site, a, h=1e-5, tol=1e-13):
    """Central finite difference (S(+h) - S(-h)) / 2h of the action for one link and generator."""
    return (action(perturb(U, mu, site, a, +h), phi_o, p, tol)
            - action(perturb(U, mu, site, a, -h), phi_o, p, tol)) / (2 * h)
