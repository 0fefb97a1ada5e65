"""GPU parity of the temporal-preconditioner determinant (wf_temporal_logdet) and its force.

* log det(mu - D_t) and its force against the oracle on the parity lattices (several warps,
  padded time lines, both boundary conditions) in both frames, device and host outputs.
  The value is 4 L^3 * 3 N_t log mu plus a gauge-dependent part that can be many orders
  smaller (mu^-N_t); the two are compared separately: the whole value to 1e-13 relative and
  the gauge-dependent part to 1e-10 relative above the rounding of the whole (1e-14 of it). The force is
  compared as a relative 2-norm (1e-11).
* TemporalDeterminant: its theta-gradient at theta = 0 is the force, and a directional
  finite difference of the value through the Function agrees with it.
"""

import numpy as np
import pytest

import synthetic as S
from oracle import determinant as DT
from oracle import wilson as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0910_0992_gb300 as wf  # noqa: E402
from paper_0910_0992_gb300.autograd import TemporalDeterminant  # noqa: E402

from test_gpu_parity import CASES  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _check_value(got, U, p):
    ref = DT.logdet_temporal(U, p)
    const = 4 * p.L ** 3 * 3 * p.T * np.log(p.mu)
    assert abs(got - ref) <= 1e-13 * abs(ref)
    assert abs((got - const) - (ref - const)) <= 1e-10 * abs(ref - const) + 1e-14 * abs(const)


@pytest.mark.parametrize("axial", [True, False], ids=["axial", "general"])
@pytest.mark.parametrize("L,T,ks,xi,bc,eps,seed", CASES, ids=[f"L{c[0]}T{c[1]}bc{c[4]}" for c in CASES])
def test_temporal_logdet_matches_oracle(L, T, ks, xi, bc, eps, seed, axial):
    p = W.Params(L, T, ks, xi=xi, bc=bc)
    U = S.random_gauge(L, T, eps, seed)
    w = wf.Wilson(L, T, ks, kappa_t=xi * ks, bc=bc, axial=axial)
    w.load_gauge(U)
    F = torch.empty((T, L, L, L, 4, 8), dtype=torch.float64, device="cuda")
    _check_value(w.temporal_logdet(F), U, p)
    ref = DT.force_logdet_temporal(U, p)
    Fh = F.cpu().numpy()
    assert _rel(Fh, ref) < 1e-11
    assert np.all(Fh[..., :3, :] == 0.0)
    Fhost = np.full((T, L, L, L, 4, 8), np.nan)  # host output (staged)
    _check_value(w.temporal_logdet(Fhost), U, p)
    assert np.array_equal(Fhost, Fh)
    assert wf.wf_temporal_logdet(w.h) == w.temporal_logdet()  # value alone, deterministic
    w.close()


def test_temporal_determinant_autograd():
    L, T = 4, 8
    p = W.Params(L, T, 0.12, kappa_t=0.36, bc=-1)   # mu^-N_t ~ 0.07: a sizeable gauge-dependent part
    U = S.random_gauge(L, T, 0.4, 61)
    w = wf.Wilson(L, T, 0.12, kappa_t=0.36, bc=-1)
    U0 = torch.from_numpy(U).cuda()
    theta = torch.zeros((T, L, L, L, 4, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    v = TemporalDeterminant.apply(theta, w, U0)
    v.backward()
    _check_value(float(v), U, p)
    ref = DT.force_logdet_temporal(U, p)
    assert _rel(theta.grad.cpu().numpy(), ref) < 1e-11
    d = torch.from_numpy(np.random.default_rng(7).standard_normal(theta.shape)).cuda()
    h = 1e-5
    with torch.no_grad():
        vp = TemporalDeterminant.apply(h * d, w, U0).item()
        vm = TemporalDeterminant.apply(-h * d, w, U0).item()
    fd = (vp - vm) / (2 * h)
    # FP64 floor of the difference: eps * |value| / h ~ 2e-8 for a value ~ 1e2
    assert abs(fd - float((theta.grad * d).sum())) < 1e-6 * abs(fd) + 1e-7
    w.close()


def test_temporal_logdet_needs_a_gauge_field():
    w = wf.Wilson(4, 8, 0.1, kappa_t=0.3, bc=-1)
    with pytest.raises(wf.WFError):
        w.temporal_logdet()
    w.close()
