"""GPU parity of the clover operator with partial temporal preconditioning and 3-D ILU.

Against ``oracle/clover.py`` on lattices with several warps, padded time lines, both boundary
conditions and both frames: the clover term A (FP64, 1e-12), M-tilde_ILU and its adjoint
(FP64 1e-12, FP32 1e-6), the reduction to diag(1, M-hat) without a clover term, the 4-D Schur
clover comparator and its adjoint (same tolerances), solves of M_SW by both methods to an FP64
true residual <= 1e-10 (checked again with the oracle's M_SW), and the errors of the clover state
(Wilson-only methods and the force refuse while a clover term is loaded).
"""

import numpy as np
import pytest

import synthetic as S
from oracle import clover as CL
from oracle import solve as SV
from oracle import wilson as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0910_0992_gb300 as wf  # noqa: E402

CASES = [
    # L, T, kappa_s, xi, bc, eps, seed, c_s, c_t
    (4, 16, 0.10, 3.0, -1, 0.3, 11, 1.2, 0.8),
    (2, 6, 0.07, 3.0, -1, 0.4, 12, 0.9, 1.1),
    (4, 7, 0.08, 2.5, 1, 0.3, 13, 1.0, 1.0),
    (4, 128, 0.074, 3.5, -1, 0.2, 14, 0.45, 0.75),
    (8, 32, 0.07, 3.0, 1, 0.25, 15, 0.5, 0.9),
]


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", params=[(c, ax) for c in CASES for ax in (True, False)],
                ids=lambda ca: f"L{ca[0][0]}T{ca[0][1]}bc{ca[0][4]}-{'axial' if ca[1] else 'general'}")
def case(request):
    (L, T, ks, xi, bc, eps, seed, c_s, c_t), axial = request.param
    p = W.Params(L, T, ks, xi=xi, bc=bc)
    U = S.random_gauge(L, T, eps, seed)
    Acl = CL.clover_term(U, c_s, c_t)
    eta = S.gaussian_source(L, T, seed + 100, nrhs=2)
    w = wf.Wilson(L, T, ks, kappa_t=xi * ks, bc=bc, axial=axial)
    w.load_gauge_clover(U, c_s, c_t)
    yield p, U, Acl, eta, w
    w.close()


def test_clover_term(case):
    p, U, Acl, eta, w = case
    assert _rel(w.apply_clover(_dev(eta)).cpu().numpy(), CL.apply_A(Acl, eta)) < 1e-12


def test_ilu_operator(case):
    p, U, Acl, eta, w = case
    par3 = W.parity3(p.L, p.T)
    x = _dev(eta)
    ref = CL.M_ilu(U, Acl, eta, p, par3)
    assert _rel(w.apply_ilu(x).cpu().numpy(), ref) < 1e-12
    refd = CL.M_ilu_dag(U, Acl, eta, p, par3)
    assert _rel(w.apply_ilu(x, dagger=True).cpu().numpy(), refd) < 1e-12
    assert _rel(w.apply_ilu(x, f32=True).cpu().numpy(), ref) < 1e-6
    host = np.empty_like(eta)  # host input and output (staged)
    wf.wf_apply_ilu(w.h, np.ascontiguousarray(eta), host, 0, 2)
    assert _rel(host, ref) < 1e-12


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_ilu_solve(case, precision):
    p, U, Acl, eta, w = case
    x, iters, res, status = w.solve(_dev(eta), tol=1e-10, method=wf.WF_TEMPORAL_ILU, precision=precision)
    assert status == wf.WF_OK
    assert max(res) <= 1e-10 and min(iters) > 0
    xh = x.cpu().numpy()
    for k in range(eta.shape[0]):
        assert CL.true_residual(U, Acl, xh[k], eta[k], p) <= 2e-10


def test_eo4d_clover_operator(case):
    p, U, Acl, eta, w = case
    if p.T % 2:
        pytest.skip("the 4-D even-odd operator needs an even T")
    par4 = W.parity4(p.L, p.T)
    od = par4 == 1
    xo = np.ascontiguousarray(np.stack([SV.compact(eta[k], od) for k in range(eta.shape[0])]))
    ref = np.stack([SV.compact(CL.M_hat4_sw(U, Acl, SV.expand(xo[k], od), p, par4), od) for k in range(2)])
    refd = np.stack([SV.compact(CL.M_hat4_sw_dag(U, Acl, SV.expand(xo[k], od), p, par4), od) for k in range(2)])
    assert _rel(w.apply_eo4d(_dev(xo)).cpu().numpy(), ref) < 1e-12
    assert _rel(w.apply_eo4d(_dev(xo), dagger=True).cpu().numpy(), refd) < 1e-12
    assert _rel(w.apply_eo4d(_dev(xo), f32=True).cpu().numpy(), ref) < 1e-6


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_eo4d_clover_solve(case, precision):
    p, U, Acl, eta, w = case
    if p.T % 2:
        pytest.skip("the 4-D even-odd method needs an even T")
    x, iters, res, status = w.solve(_dev(eta), tol=1e-10, method=wf.WF_EO4D, precision=precision)
    assert status == wf.WF_OK
    assert max(res) <= 1e-10 and min(iters) > 0
    xh = x.cpu().numpy()
    for k in range(eta.shape[0]):
        assert CL.true_residual(U, Acl, xh[k], eta[k], p) <= 2e-10


def test_ilu_without_clover_is_schur():
    L, T = 4, 16
    p = W.Params(L, T, 0.1, xi=3.0, bc=-1)
    U = S.random_gauge(L, T, 0.3, 21)
    eta = S.gaussian_source(L, T, 22)
    w = wf.Wilson(L, T, 0.1, kappa_t=0.3, bc=-1)
    w.load_gauge(U)
    par3 = W.parity3(L, T)
    ref = W.restrict(eta, par3 == 0) + W.M_hat(U, eta, p, par3)
    assert _rel(w.apply_ilu(_dev(eta)).cpu().numpy(), ref) < 1e-12
    x, iters, res, status = w.solve(_dev(eta), tol=1e-10, method=wf.WF_TEMPORAL_ILU)
    assert status == wf.WF_OK and max(res) <= 1e-10
    w.close()


def test_clover_state_errors():
    L, T = 4, 8
    U = S.random_gauge(L, T, 0.3, 23)
    eta = _dev(S.gaussian_source(L, T, 24))
    w = wf.Wilson(L, T, 0.1, kappa_t=0.3, bc=-1)
    w.load_gauge(U)
    with pytest.raises(wf.WFError):
        w.apply_clover(eta)  # no clover term
    w.load_gauge_clover(U, 1.0, 1.0)
    with pytest.raises(wf.WFError):
        w.solve(eta, method=wf.WF_TEMPORAL_SCHUR)  # solves the Wilson matrix
    with pytest.raises(wf.WFError):
        w.solve(eta, method=wf.WF_TEMPORAL_ILU, x0=torch.zeros_like(eta))
    phi = torch.zeros(L ** 3 * T // 2 * 12, dtype=torch.complex128, device="cuda")
    with pytest.raises(wf.WFError):
        wf.wf_force(w.h, phi, None)
    with pytest.raises(wf.WFError):
        wf.wf_load_gauge_clover(w.h, U, float("nan"), 1.0)
    w.load_gauge(U)  # a plain load removes the clover term
    with pytest.raises(wf.WFError):
        w.apply_clover(eta)
    w.close()
