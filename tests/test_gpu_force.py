"""GPU parity of the pseudofermion force (wf_force) and its autograd binding.

* FP64 force against the oracle's FP64 adjoint (relative 1e-10), both frames;
  FP32-inner solve against the same (relative 1e-6).
* The force workloads (8^3 x 32 and 16^3 x 64, xi = 3): central finite differences of the
  library's own action on 20 random links near a point-supported pseudofermion (h = 1e-5), FP64,
  and FP32-inner against FP64 over the whole lattice.
* PseudofermionAction: its theta-gradient at theta = 0 equals the force, and a directional
  finite difference of the action through the autograd Function agrees with it.
"""

import numpy as np
import pytest

import synthetic as S
from oracle import force as OF
from oracle import solve as SV
from oracle import wilson as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0910_0992_gb300 as wf  # noqa: E402
from paper_0910_0992_gb300.autograd import PseudofermionAction, generators  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _odd_phi(L, T, seed):
    par3 = W.parity3(L, T)
    full = S.gaussian_source(L, T, seed)
    return SV.compact(full, par3 == 1), W.restrict(full, par3 == 1)


@pytest.mark.parametrize("axial", [True, False])
@pytest.mark.parametrize("L,T,bc", [(4, 8, -1), (2, 6, 1)])
def test_force_matches_oracle(L, T, bc, axial):
    p = W.Params(L, T, 0.07, xi=3.0, bc=bc)
    U = S.random_gauge(L, T, 0.35, 31)
    phi_c, phi_full = _odd_phi(L, T, 32)
    ref = OF.force(U, phi_full, p)
    w = wf.Wilson(L, T, 0.07, kappa_t=0.21, bc=bc, axial=axial)
    w.load_gauge(U)
    F = torch.empty((T, L, L, L, 4, 8), dtype=torch.float64, device="cuda")
    S64, it = wf.wf_force(w.h, torch.from_numpy(phi_c).cuda(), F, wf.WF_FP64, 1e-13)
    assert _rel(F.cpu().numpy(), ref) < 1e-10
    assert abs(S64 - OF.action(U, phi_full, p)) < 1e-11 * abs(S64)
    F32 = np.empty((T, L, L, L, 4, 8))  # host output, FP32 iterations with FP64 reliable updates
    wf.wf_force(w.h, torch.from_numpy(phi_c).cuda(), F32, wf.WF_FP32, 1e-12)
    assert _rel(F32, ref) < 1e-6
    w.close()


def _perturbed(U, mu, site, a, h):
    return OF.perturb(U, mu, site, a, h)


@pytest.mark.parametrize("workload", ["force_8c32_xi3", "force_16c64_xi3"])
def test_force_finite_differences_on_force_workloads(workload):
    """20 links near a point-supported pseudofermion on each force workload (8^3 x 32 and
    16^3 x 64, xi = 3): S stays small, so a central difference resolves dS/dU to ~1e-9 (for a
    field spread over the whole lattice S grows with the volume and the FP64 floor eps * S / h
    of the difference swamps single-link forces). The difference uses only the library's action
    (a CG solve), not its force kernels, so it checks them at sizes the oracle cannot reach in a
    test run; the FP32-inner force must agree with the FP64 one over the whole lattice."""
    prm, U, _ = S.workload(workload, with_sources=False)
    L, T = prm["L"], prm["T"]
    rng = np.random.default_rng(5)
    src = (7, 3, 2, 4)  # (t, z, y, x): x + y + z = 9, odd
    full = np.zeros((T, L, L, L, 4, 3), dtype=np.complex128)
    full[src] = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    phi_c = SV.compact(full, W.parity3(L, T) == 1)
    phi_d = torch.from_numpy(phi_c).cuda()
    w = wf.Wilson(L, T, prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"])
    w.load_gauge(U)
    F = torch.empty((T, L, L, L, 4, 8), dtype=torch.float64, device="cuda")
    wf.wf_force(w.h, phi_d, F, wf.WF_FP64, 1e-13)
    F32 = torch.empty_like(F)
    wf.wf_force(w.h, phi_d, F32, wf.WF_FP32, 1e-12)
    F = F.cpu().numpy()
    assert _rel(F32.cpu().numpy(), F) < 1e-6
    h = 1e-5
    for _ in range(20):
        mu = int(rng.integers(0, 4))
        site = ((src[0] + int(rng.integers(-3, 4))) % T,) + tuple((src[1 + k] + int(rng.integers(-1, 2))) % L
                                                                   for k in range(3))
        a = int(rng.integers(0, 8))
        sp = []
        for sgn in (+1, -1):
            w.load_gauge(_perturbed(U, mu, site, a, sgn * h))
            sp.append(wf.wf_force(w.h, phi_d, None, wf.WF_FP64, 1e-14)[0])
        fd = (sp[0] - sp[1]) / (2 * h)
        err = abs(F[site + (mu, a)] - fd)
        # FP64 floor of the difference: eps * S / h ~ 1e-9 for S ~ 1e2
        assert err < 2e-8 + 1e-6 * abs(fd), (mu, site, a, F[site + (mu, a)], fd)
    w.close()


def test_autograd_gradient_is_the_force():
    L, T = 4, 8
    p = W.Params(L, T, 0.075, xi=3.0, bc=-1)
    U = S.random_gauge(L, T, 0.3, 51)
    phi_c, phi_full = _odd_phi(L, T, 52)
    w = wf.Wilson(L, T, 0.075, kappa_t=0.225, bc=-1)
    U0 = torch.from_numpy(U).cuda()
    phi = torch.from_numpy(phi_c).cuda()
    theta = torch.zeros((T, L, L, L, 4, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    S0 = PseudofermionAction.apply(theta, w, U0, phi)
    S0.backward()
    ref = OF.force(U, phi_full, p)
    assert _rel(theta.grad.cpu().numpy(), ref) < 1e-10
    # directional derivative along a random theta direction, through the Function itself
    d = torch.from_numpy(np.random.default_rng(3).standard_normal(theta.shape)).cuda()
    h = 1e-5
    with torch.no_grad():
        sp = PseudofermionAction.apply(h * d, w, U0, phi).item()
        sm = PseudofermionAction.apply(-h * d, w, U0, phi).item()
    fd = (sp - sm) / (2 * h)
    assert abs(fd - float((theta.grad * d).sum())) < 1e-6 * abs(fd) + 1e-7
    w.close()
