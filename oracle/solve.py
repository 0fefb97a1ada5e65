"""FP64 CG on the normal equations for the four operators of the comparison (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/wilson.py``).

The paper measures condition numbers (§III) and names conjugate gradients as
its Krylov method (§III.B); the normal-equation form is not stated, so every
method here uses CGNR: CG on A^dag A x = A^dag b, the fair common choice for
comparing preconditioners. A solve is accepted when the FP64 true residual of
the original system, ||eta - M psi||_2 / ||eta||_2, is at most ``tol``.
"""

import numpy as np

from . import wilson as W

METHODS = ("unprec", "eo4d", "temporal", "temporal_schur")


def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def _norm2(a):
    return float(np.real(_dot(a, a)))


def cgnr(A, Adag, b, x0=None, tol=1e-10, maxiter=100000):
    """CG on A^dag A x = A^dag b; stops when ||b - A x|| / ||b|| <= tol.

    Returns (x, iterations, relative residual of the last iterate).
    """
    bnorm = np.sqrt(_norm2(b))
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    s = Adag(r)
    pdir = s.copy()
    gamma = _norm2(s)
    it = 0
    rel = np.sqrt(_norm2(r)) / bnorm
    while rel > tol and it < maxiter:
        q = A(pdir)
        alpha = gamma / _norm2(q)
        x = x + alpha * pdir
        r = r - alpha * q
        s = Adag(r)
        gamma_new = _norm2(s)
        it += 1
        rel = np.sqrt(_norm2(r)) / bnorm
        pdir = s + (gamma_new / gamma) * pdir
        gamma = gamma_new
    return x, it, rel


def true_residual(U, psi, eta, p):
    """||eta - M psi||_2 / ||eta||_2 over all sites, spins and colours, in FP64."""
    return np.sqrt(_norm2(eta - W.M(U, psi, p)) / _norm2(eta))


def _system(U, eta, p, method):
    """(A, A^dag, b, reconstruct) for one method: the solution is reconstruct(A^-1 b)."""
    if method == "unprec":
        return (lambda v: W.M(U, v, p)), (lambda v: W.M_dag(U, v, p)), eta, (lambda y: y)
    if method == "temporal":
        b = W.C_L(U, eta, p)
        return (lambda v: W.M_tilde(U, v, p)), (lambda v: W.M_tilde_dag(U, v, p)), b, (lambda y: W.C_R(U, y, p))
    if method == "temporal_schur":
        par3 = W.parity3(p.L, p.T)
        bp = W.S_L(U, eta, p, par3)
        ye = W.restrict(bp, par3 == 0)
        bo = W.restrict(bp, par3 == 1)
        A = lambda v: W.M_hat(U, v, p, par3)
        Ad = lambda v: W.M_hat_dag(U, v, p, par3)
        return A, Ad, bo, (lambda yo: W.S_R(U, ye + yo, p, par3))
    if method == "eo4d":
        par4 = W.parity4(p.L, p.T)
        ev, od = par4 == 0, par4 == 1
        eta_e = W.restrict(eta, ev)
        bo = W.restrict(eta, od) + W.restrict(W.D_w(U, eta_e, p), od) / p.mu
        A = lambda v: W.M_hat4(U, v, p, par4)
        Ad = lambda v: W.M_hat4_dag(U, v, p, par4)

        def recon(po):
            pe = W.restrict(eta_e + W.D_w(U, po, p), ev) / p.mu
            return pe + po

        return A, Ad, bo, recon
    raise ValueError(f"unknown method {method!r}")


def solve(U, eta, p, method="temporal_schur", tol=1e-10, maxiter=100000):
    """Solve M psi = eta with CGNR on the chosen preconditioned system.

    The inner CG tolerance starts at ``tol`` and is tightened (restarting from
    the current iterate) until the FP64 true residual is at most ``tol``.
    Returns (psi, total CG iterations, true relative residual).
    """
    A, Ad, b, recon = _system(U, eta, p, method)
    inner = tol
    y, total, rel = None, 0, np.inf
    for _ in range(8):
        y, it, _ = cgnr(A, Ad, b, x0=y, tol=inner, maxiter=maxiter - total)
        total += it
        psi = recon(y)
        rel = true_residual(U, psi, eta, p)
        if rel <= tol or total >= maxiter:
            break
        inner *= 0.5 * tol / rel
    return psi, total, rel


def compact(psi, mask):
    """Gather the sites where ``mask`` is true, in lexicographic (t, z, y, x) order: (..., n, 4, 3)."""
    return psi[..., mask, :, :]


def expand(c, mask):
    """Inverse of ``compact``: scatter (..., n, 4, 3) back onto a zero lattice field."""
    T, L = mask.shape[0], mask.shape[1]
    out = np.zeros(c.shape[:-3] + (T, L, L, L, 4, 3), dtype=np.complex128)
    out[..., mask, :, :] = c
    return out
