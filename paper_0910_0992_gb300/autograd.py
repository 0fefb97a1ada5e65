"""torch.autograd binding of the pseudofermion force (wf_force).

PseudofermionAction.apply(theta, wilson, U0, phi) returns
    S = phi^dag (M-hat^dag M-hat)^-1 phi   at the links  U = exp(i theta_a T_a) U0,
with theta of shape (T, L, L, L, 4, 8) (one su(3) coordinate vector per link, T_a the
Gell-Mann matrices halved) and phi an odd field. Its gradient with respect to theta is the
force F = dS/d eps for U -> exp(i eps T_a) U at U(theta), computed by the library's adjoint
(wf_force); at theta = 0, where a molecular-dynamics force is evaluated, it is exactly dS/dtheta.
The forward pass keeps nothing of the solve: the backward pass runs the solve again, so
memory stays at one force field.

TemporalDeterminant.apply(theta, wilson, U0) returns log det(mu - D_t) at U(theta) with the
same gradient convention (wf_temporal_logdet). det M = det(M-hat) det(mu - D_t), so a
two-flavour action in terms of M-hat is
    PseudofermionAction.apply(theta, w, U0, phi) - 2 * TemporalDeterminant.apply(theta, w, U0).

Building U from theta (a 3x3 matrix exponential per link) is input preparation done with
torch; every step of the action and the force runs in libwf.
"""

import torch

from . import _lib

_T = None


def generators(device):
    lam = torch.zeros((8, 3, 3), dtype=torch.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1], lam[1, 1, 0] = -1j, 1j
    lam[2, 0, 0], lam[2, 1, 1] = 1, -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2], lam[4, 2, 0] = -1j, 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2], lam[6, 2, 1] = -1j, 1j
    lam[7] = torch.diag(torch.tensor([1, 1, -2], dtype=torch.complex128)) / 3 ** 0.5
    return (lam / 2).to(device)


def links_at(theta, U0):
    """U = exp(i theta_a T_a) U0 per link."""
    if not torch.any(theta != 0):
        return U0
    Ta = generators(theta.device)
    H = torch.einsum("...a,aij->...ij", theta.to(torch.complex128), Ta)
    return torch.linalg.matrix_exp(1j * H) @ U0


class PseudofermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, wilson, U0, phi, precision=_lib.WF_FP64, tol=1e-12):
        U = links_at(theta.detach(), U0).contiguous()
        wilson.load_gauge(U)
        S, _ = _lib.wf_force(wilson.h, phi, None, precision, tol)
        ctx.wilson, ctx.U, ctx.phi, ctx.precision, ctx.tol = wilson, U, phi, precision, tol
        return torch.tensor(S, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, grad_S):
        ctx.wilson.load_gauge(ctx.U)
        F = torch.empty(ctx.U.shape[:-2] + (8,), dtype=torch.float64, device=ctx.U.device)
        _lib.wf_force(ctx.wilson.h, ctx.phi, F, ctx.precision, ctx.tol)
        return grad_S * F, None, None, None, None, None


class TemporalDeterminant(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, wilson, U0):
        U = links_at(theta.detach(), U0).contiguous()
        wilson.load_gauge(U)
        ctx.wilson, ctx.U = wilson, U
        return torch.tensor(_lib.wf_temporal_logdet(wilson.h), dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, grad_S):
        ctx.wilson.load_gauge(ctx.U)
        F = torch.empty(ctx.U.shape[:-2] + (8,), dtype=torch.float64, device=ctx.U.device)
        _lib.wf_temporal_logdet(ctx.wilson.h, F)
        return grad_S * F, None, None
