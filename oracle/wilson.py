"""Plain FP64 oracle for the anisotropic Wilson matrix and its temporal preconditioner.

TEST INFRASTRUCTURE ONLY. This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py``. The library's product path never imports it, and it
imports nothing from the library.

Everything here follows arXiv 0910.0992 (Joo, Edwards, Peardon), section by
section, in plain NumPy on whole-lattice arrays. Nothing is blocked, fused or
reordered beyond what the definitions state; every step is a direct transcription
of the equation it cites, written out with einsum (colour and spin products)
and np.roll (lattice shifts).

Conventions (readings of points the paper leaves open):

* Spinor fields have shape ``(..., T, L, L, L, 4, 3)`` = ``[t, z, y, x, spin, colour]``;
  gauge fields ``(T, L, L, L, 4, 3, 3)`` with ``mu = 0, 1, 2, 3`` for x, y, z, t.
  The paper's temporal link ``U_0`` is ``U[..., 3, :, :]`` here.
* Spin basis: Euclidean Dirac-Pauli (§II.C, "Dirac-Pauli spin basis"),
  ``gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]``, ``gamma_t = diag(1, 1, -1, -1)``,
  ``gamma_5 = gamma_x gamma_y gamma_z gamma_t``. Spectra and iteration counts do not
  depend on this choice; component values do.
* Temporal boundary: ``bc = s = +1`` periodic, ``-1`` antiperiodic. The wrap entry of
  the temporal hopping matrix is ``T[N_t-1, 0] = -s U_0(N_t-1)`` (§II.A; the printed
  position and sign of this entry are garbled, and this is the only reading that
  agrees with the bulk ``-U`` entries, with ``V W^dagger`` and with
  ``mu - D_t = C_L^-1 C_R^-1``). The hop of ``D_t`` across ``t = N_t-1 <-> 0``
  carries the same sign ``s``.
* Parameters: ``mu = 1 / (2 kappa_t)`` and ``gamma_f = kappa_t / kappa_s``, so that the
  paper's ``M`` is ``1/(2 kappa_t)`` times the hopping-parameter form
  ``1 - kappa_t sum (1 -+ gamma_t) U - kappa_s sum (1 -+ gamma_i) U``.
"""

import numpy as np

# ---------------------------------------------------------------------------
# Lattice axes (counted from the end so a leading batch axis is allowed)
# ---------------------------------------------------------------------------
AX_T, AX_Z, AX_Y, AX_X = -6, -5, -4, -3
MU_AXIS = (AX_X, AX_Y, AX_Z, AX_T)  # axis of direction mu = 0 (x), 1 (y), 2 (z), 3 (t)
MU_T = 3

# ---------------------------------------------------------------------------
# Spin algebra: Dirac-Pauli basis (§II.C and App. C)
# ---------------------------------------------------------------------------
_SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)
I4 = np.eye(4, dtype=np.complex128)

GAMMA = tuple(
    [np.block([[_Z2, -1j * _SIGMA[k]], [1j * _SIGMA[k], _Z2]]) for k in range(3)]
    + [np.block([[_I2, _Z2], [_Z2, -_I2]])]
)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]

# Temporal spin projectors P_{+-} = (1 +- gamma_0) / 2 (§II.A)
P_PLUS = 0.5 * (I4 + GAMMA[MU_T])
P_MINUS = 0.5 * (I4 - GAMMA[MU_T])


class Params:
    """Lattice size, boundary sign and the couplings (mu, gamma_f) of the paper's M (§II, Eq. for M)."""

    def __init__(self, L, T, kappa_s, kappa_t=None, xi=None, bc=-1):
        if kappa_t is None or kappa_t <= 0:
            kappa_t = xi * kappa_s
        self.L, self.T, self.bc = int(L), int(T), float(bc)
        self.kappa_s, self.kappa_t = float(kappa_s), float(kappa_t)
        self.mu = 1.0 / (2.0 * kappa_t)
        self.gamma_f = kappa_t / kappa_s

    @property
    def volume(self):
        return self.L ** 3 * self.T


# ---------------------------------------------------------------------------
# Elementary field operations
# ---------------------------------------------------------------------------
def spin(G, psi):
    """Apply a 4x4 spin matrix to every site: (G psi)_s = sum_s' G_{s s'} psi_s'."""
    return np.einsum("st,...tc->...sc", G, psi)


def colour(U, psi):
    """Apply a site-dependent 3x3 colour matrix U(x) to every spin (or column) component."""
    return np.einsum("...ab,...sb->...sa", U, psi)


def dag(U):
    """Hermitian conjugate of every 3x3 matrix of a field."""
    return np.conj(np.swapaxes(U, -1, -2))


def shift(f, mu, step, bc):
    """f(x + step * mu_hat) on the periodic lattice; hops across the time boundary pick up ``bc``.

    Works for spinor fields ``(..., T, L, L, L, 4, 3)`` and for link / matrix fields
    ``(T, L, L, L, 3, 3)``: in both the lattice axes are -6 .. -3.
    """
    ax = MU_AXIS[mu]
    out = np.roll(f, -step, axis=ax)
    if mu == MU_T and bc != 1.0:
        T = f.shape[ax]
        idx = [slice(None)] * f.ndim
        idx[f.ndim + ax] = T - 1 if step == +1 else 0
        out[tuple(idx)] *= bc
    return out


def link(U, mu):
    """The link field U_mu(x), shape (T, L, L, L, 3, 3)."""
    return U[..., mu, :, :]


# ---------------------------------------------------------------------------
# Hopping terms D_t, D_s and the Wilson matrix M (§II, Eqs. for M, D_t, D_s)
# ---------------------------------------------------------------------------
def hop(U, psi, mu, bc):
    """(1 - gamma_mu)/2 U_mu(x) psi(x + mu) + (1 + gamma_mu)/2 U_mu^dag(x - mu) psi(x - mu)."""
    Umu = link(U, mu)
    fwd = colour(Umu, shift(psi, mu, +1, bc))
    bwd = colour(dag(shift(Umu, mu, -1, 1.0)), shift(psi, mu, -1, bc))
    return spin(0.5 * (I4 - GAMMA[mu]), fwd) + spin(0.5 * (I4 + GAMMA[mu]), bwd)


def D_t(U, psi, bc):
    """Temporal hopping term D_t (§II, Eq. for D_t)."""
    return hop(U, psi, MU_T, bc)


def D_s(U, psi):
    """Spatial hopping term D_s = sum over i = x, y, z (§II, Eq. for D_s); spatially periodic."""
    return hop(U, psi, 0, 1.0) + hop(U, psi, 1, 1.0) + hop(U, psi, 2, 1.0)


def M(U, psi, p):
    """Wilson matrix M = mu - D_t - D_s / gamma_f (§II, Eq. for M with A = 0)."""
    return p.mu * psi - D_t(U, psi, p.bc) - D_s(U, psi) / p.gamma_f


def M_dag(U, psi, p):
    """M^dag = gamma_5 M gamma_5 (gamma_5-hermiticity of the Wilson matrix)."""
    return spin(GAMMA5, M(U, spin(GAMMA5, psi), p))


# ---------------------------------------------------------------------------
# Temporal matrix T and its inverse by Sherman-Morrison-Woodbury (§II.A)
# ---------------------------------------------------------------------------
def T_apply(U, chi, p):
    """(T chi)(t) = mu chi(t) - U_0(t) chi(t+1), with T[N_t-1, 0] = -s U_0(N_t-1) (§II.A, Eq. for T)."""
    U0 = link(U, MU_T)
    return p.mu * chi - colour(U0, shift(chi, MU_T, +1, p.bc))


def Tdag_apply(U, chi, p):
    """(T^dag chi)(t) = mu chi(t) - U_0^dag(t-1) chi(t-1), the adjoint of T_apply."""
    U0 = link(U, MU_T)
    return p.mu * chi - colour(dag(shift(U0, MU_T, -1, 1.0)), shift(chi, MU_T, -1, p.bc))


def _t_index(a, t):
    idx = [slice(None)] * a.ndim
    idx[a.ndim + AX_T] = t
    return tuple(idx)


def T0_backsub(U0, rhs, mu):
    """Solve T_0 chi = rhs by back-substitution from the open end (§II.A, T_0; App. B, C(B)).

    chi(N_t-1) = rhs(N_t-1)/mu, then chi(t) = (rhs(t) + U_0(t) chi(t+1))/mu for t = N_t-2 .. 0.
    (The paper's App. B writes the step with a minus sign; with T_0's -U entries the
    recurrence is the one used here.)
    """
    T = rhs.shape[AX_T]
    chi = np.zeros_like(rhs)
    chi[_t_index(chi, T - 1)] = rhs[_t_index(rhs, T - 1)] / mu
    for t in range(T - 2, -1, -1):
        nxt = chi[_t_index(chi, t + 1)]
        chi[_t_index(chi, t)] = (rhs[_t_index(rhs, t)] + colour(U0[t], nxt)) / mu
    return chi


def T0dag_forwardsub(U0, rhs, mu):
    """Solve T_0^dag chi = rhs by forward substitution from t = 0 (§II.A, the T^-dag paragraph).

    chi(0) = rhs(0)/mu, then chi(t) = (rhs(t) + U_0^dag(t-1) chi(t-1))/mu for t = 1 .. N_t-1.
    """
    T = rhs.shape[AX_T]
    chi = np.zeros_like(rhs)
    chi[_t_index(chi, 0)] = rhs[_t_index(rhs, 0)] / mu
    for t in range(1, T):
        prv = chi[_t_index(chi, t - 1)]
        chi[_t_index(chi, t)] = (rhs[_t_index(rhs, t)] + colour(dag(U0[t - 1]), prv)) / mu
    return chi


def _vw(U, p):
    """The SMW column blocks V and W of T = T_0 + V W^dag (§II.A, Eqs. for V and W).

    Stored as fields of 3 column vectors, shape (T, L, L, L, 3(column), 3(colour)):
    V_t = -s U_0(N_t-1) delta_{t, N_t-1} and W_t = delta_{t, 0} * identity.
    """
    T, L = p.T, p.L
    U0 = link(U, MU_T)
    V = np.zeros((T, L, L, L, 3, 3), dtype=np.complex128)
    V[T - 1] = np.swapaxes(-p.bc * U0[T - 1], -1, -2)  # column k of the matrix -> row k here
    W = np.zeros((T, L, L, L, 3, 3), dtype=np.complex128)
    W[0] = np.eye(3)
    return V, W


def _cols_to_matrix(c):
    """(..., 3(column), 3(colour)) column storage -> ordinary (..., 3, 3) matrix."""
    return np.swapaxes(c, -1, -2)


def smw_init(U, p):
    """Step 1 of the SMW procedure (§II.A): X = T_0^-1 V by back-substitution, Lambda = (I + W^dag X)^-1.

    Returns (X, Lam) with X in column storage (T, L, L, L, 3, 3) and Lam (L, L, L, 3, 3).
    """
    U0 = link(U, MU_T)
    V, W = _vw(U, p)
    X = T0_backsub(U0, V, p.mu)
    WdX = np.einsum("tzyxka,tzyxja->zyxkj", W.conj(), X)  # (W^dag X)_{k j} = sum_t W_t^dag X_t
    Lam = np.linalg.inv(np.eye(3) + WdX)
    return X, Lam


def Tinv(U, eta, p, init=None):
    """psi = T^-1 eta by SMW step 2 (§II.A): chi = T_0^-1 eta, q = Lambda W^dag chi, psi = chi - X q.

    ``eta`` may carry any number of spin (or other) vectors per site: shape (..., T, L, L, L, K, 3).
    """
    X, Lam = smw_init(U, p) if init is None else init
    U0 = link(U, MU_T)
    chi = T0_backsub(U0, eta, p.mu)
    chi0 = chi[_t_index(chi, 0)]                       # W^dag chi = chi on time slice 0
    q = np.einsum("zyxkj,...zyxsj->...zyxsk", Lam, chi0)
    Xm = _cols_to_matrix(X)                             # (T, L, L, L, 3, 3) ordinary matrices
    return chi - np.einsum("tzyxak,...zyxsk->...tzyxsa", Xm, q)


def smw_init_dag(U, p):
    """SMW initialisation for T^dag = T_0^dag + W V^dag (§II.A, T^-dag paragraph).

    Y = (T_0^dag)^-1 W by forward substitution and Lambda' = (I + V^dag Y)^-1.
    """
    U0 = link(U, MU_T)
    V, W = _vw(U, p)
    Y = T0dag_forwardsub(U0, W, p.mu)
    VdY = np.einsum("tzyxka,tzyxja->zyxkj", V.conj(), Y)
    Lam = np.linalg.inv(np.eye(3) + VdY)
    return Y, Lam


def Tdag_inv(U, eta, p, init=None):
    """psi = (T^dag)^-1 eta: chi = (T_0^dag)^-1 eta, q = Lambda' V^dag chi, psi = chi - Y q."""
    Y, Lam = smw_init_dag(U, p) if init is None else init
    U0 = link(U, MU_T)
    V, _ = _vw(U, p)
    chi = T0dag_forwardsub(U0, eta, p.mu)
    Vd_chi = np.einsum("tzyxka,...tzyxsa->...zyxsk", V.conj(), chi)  # V^dag chi
    q = np.einsum("zyxkj,...zyxsj->...zyxsk", Lam, Vd_chi)
    Ym = _cols_to_matrix(Y)
    return chi - np.einsum("tzyxak,...zyxsk->...tzyxsa", Ym, q)


# ---------------------------------------------------------------------------
# Left and right temporal preconditioners C_L, C_R (§II.A)
# ---------------------------------------------------------------------------
def C_L(U, psi, p):
    """C_L = P_+ + P_- T^-1 (§II.A)."""
    return spin(P_PLUS, psi) + spin(P_MINUS, Tinv(U, psi, p))


def C_R(U, psi, p):
    """C_R = P_- + P_+ (T^dag)^-1 (§II.A)."""
    return spin(P_MINUS, psi) + spin(P_PLUS, Tdag_inv(U, psi, p))


def C_L_inv(U, psi, p):
    """C_L^-1 = P_+ + P_- T (§II.A)."""
    return spin(P_PLUS, psi) + spin(P_MINUS, T_apply(U, psi, p))


def C_R_inv(U, psi, p):
    """C_R^-1 = P_- + P_+ T^dag (§II.A)."""
    return spin(P_MINUS, psi) + spin(P_PLUS, Tdag_apply(U, psi, p))


def M_tilde(U, psi, p):
    """Temporally preconditioned matrix M~ = C_L M C_R (§II.A)."""
    return C_L(U, M(U, C_R(U, psi, p), p), p)


def M_tilde_dag(U, psi, p):
    """M~^dag = gamma_5 M~ gamma_5, from C_L^{dag -1} = gamma_5 C_R^-1 gamma_5 (§II.A)."""
    return spin(GAMMA5, M_tilde(U, spin(GAMMA5, psi), p))


# ---------------------------------------------------------------------------
# Parities and the 3-D Schur (even-odd) combination (§II.B)
# ---------------------------------------------------------------------------
def parity3(L, T):
    """p_3(x) = (x_1 + x_2 + x_3) mod 2 on every site, shape (T, L, L, L) (§II.B)."""
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    return (x + y + z) % 2


def parity4(L, T):
    """p_4(x) = (x_0 + x_1 + x_2 + x_3) mod 2 on every site, shape (T, L, L, L) (§II.B)."""
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    return (x + y + z + t) % 2


def restrict(psi, mask):
    """Keep the sites where ``mask`` is true (the block restriction written f^e or f^o)."""
    return psi * mask[..., None, None]


def Dbar_s(U, psi, p, to_par, par3):
    """D-bar_s^{to, from} = C_L^{to} D_s^{to, from} C_R^{from} (§II.B, Eq. for D-bar_s^{eo})."""
    frm = 1 - to_par
    return restrict(C_L(U, restrict(D_s(U, restrict(C_R(U, restrict(psi, par3 == frm), p), par3 == frm)),
                                    par3 == to_par), p), par3 == to_par)


def M_hat(U, psi_o, p, par3=None):
    """Temporal + 3-D Schur operator on odd-p_3 sites: 1 - gamma_f^-2 D-bar^{oe} D-bar^{eo} (§II.B, Eq. TPrecFull)."""
    if par3 is None:
        par3 = parity3(p.L, p.T)
    x = restrict(psi_o, par3 == 1)
    return x - Dbar_s(U, Dbar_s(U, x, p, 0, par3), p, 1, par3) / p.gamma_f ** 2


def M_hat_dag(U, psi_o, p, par3=None):
    """M-hat^dag = gamma_5 M-hat gamma_5 (gamma_5-hermiticity kept by the preconditioner, §II.A)."""
    return spin(GAMMA5, M_hat(U, spin(GAMMA5, psi_o), p, par3))


def S_L(U, eta, p, par3=None):
    """Left block preconditioner S_L = [[C_L^e, 0], [gamma_f^-1 D-bar^{oe} C_L^e, C_L^o]] (§II.B)."""
    if par3 is None:
        par3 = parity3(p.L, p.T)

    ev, od = par3 == 0, par3 == 1
    cle = restrict(C_L(U, restrict(eta, ev), p), ev)
    clo = restrict(C_L(U, restrict(eta, od), p), od)
    return cle + Dbar_s(U, cle, p, 1, par3) / p.gamma_f + clo


def S_R(U, y, p, par3=None):
    """Right block preconditioner S_R = [[C_R^e, gamma_f^-1 C_R^e D-bar^{eo}], [0, C_R^o]] (§II.B)."""
    if par3 is None:
        par3 = parity3(p.L, p.T)
    ev, od = par3 == 0, par3 == 1
    ye, yo = restrict(y, ev), restrict(y, od)
    top = restrict(C_R(U, ye + Dbar_s(U, yo, p, 0, par3) / p.gamma_f, p), ev)
    bot = restrict(C_R(U, yo, p), od)
    return top + bot


# ---------------------------------------------------------------------------
# 4-D Schur (standard even-odd) comparator (§II.B, first display; App. B)
# ---------------------------------------------------------------------------
def D_w(U, psi, p):
    """4-D Wilson dslash D_w = D_s / gamma_f + D_t (§II.B)."""
    return D_s(U, psi) / p.gamma_f + D_t(U, psi, p.bc)


def M_hat4(U, psi_o, p, par4=None):
    """4-D Schur complement on odd-p_4 sites: mu - D_w^{oe} mu^-1 D_w^{eo} (§II.B; App. B, Wilson case)."""
    if par4 is None:
        par4 = parity4(p.L, p.T)
    ev, od = par4 == 0, par4 == 1
    x = restrict(psi_o, od)
    return p.mu * x - restrict(D_w(U, restrict(D_w(U, x, p), ev), p), od) / p.mu


def M_hat4_dag(U, psi_o, p, par4=None):
    return spin(GAMMA5, M_hat4(U, spin(GAMMA5, psi_o), p, par4))
