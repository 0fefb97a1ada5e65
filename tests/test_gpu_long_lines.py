"""Time extents above 128 sites (the line kernels' long-line variant, up to 8 sites per lane, N_t
<= 256) against the FP64 oracle: M, T^-1, C_L / C_R and M-hat applies (1e-12 FP64, 1e-6 FP32) in
both frames, solves by temporal + Schur (FP64, FP32 defect correction, FP32 with reliable updates)
and 4-D even-odd to the oracle-checked 1e-10 true residual, and the requests that need the
128-slot kernels refused with WF_EINVAL. The layouts: N_t = 160 (5 sites per lane), 200 (7, with
padding slots), 256 (8), and 129 (5, the first long line)."""

import numpy as np
import pytest

import synthetic as S
from oracle import solve as SV
from oracle import wilson as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0910_0992_gb300 as wf  # noqa: E402

TRUE_RESID = 1e-10 + 1e-13  # the rounding room of two FP64 evaluations of one residual
# L, T, kappa_s, xi, bc, eps, seed
CASES = [(2, 160, 0.07, 3.5, -1, 0.3, 21), (4, 200, 0.065, 4.5, 1, 0.25, 22), (2, 256, 0.06, 6.0, -1, 0.3, 23),
         (2, 129, 0.07, 3.0, 1, 0.3, 24)]


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module", params=[(c, ax) for c in CASES for ax in (True, False)],
                ids=lambda ca: f"L{ca[0][0]}T{ca[0][1]}-{'axial' if ca[1] else 'general'}")
def case(request):
    (L, T, ks, xi, bc, eps, seed), axial = request.param
    p = W.Params(L, T, ks, xi=xi, bc=bc)
    U = S.random_gauge(L, T, eps, seed)
    eta = S.gaussian_source(L, T, seed + 100, nrhs=2)
    w = wf.Wilson(L, T, ks, kappa_t=xi * ks, bc=bc, axial=axial)
    w.load_gauge(U)
    yield p, U, eta, w
    w.close()


def test_applies(case):
    p, U, eta, w = case
    x = _dev(eta)
    assert _rel(_host(w.apply_M(x)), W.M(U, eta, p)) < 1e-12
    assert _rel(_host(w.apply_M(x, dagger=True)), W.M_dag(U, eta, p)) < 1e-12
    assert _rel(_host(w.apply_M(x, f32=True)), W.M(U, eta, p)) < 1e-6
    assert _rel(_host(w.apply_Tinv(x)), W.Tinv(U, eta, p)) < 1e-12
    assert _rel(_host(w.apply_Tinv(x, dagger=True)), W.Tdag_inv(U, eta, p)) < 1e-12
    assert _rel(_host(w.apply_Tinv(x, f32=True)), W.Tinv(U, eta, p)) < 1e-6
    assert _rel(_host(w.apply_C(x, 0)), W.C_L(U, eta, p)) < 1e-12
    assert _rel(_host(w.apply_C(x, 1)), W.C_R(U, eta, p)) < 1e-12


def test_apply_schur(case):
    p, U, eta, w = case
    par3 = W.parity3(p.L, p.T)
    odd = par3 == 1
    xo = SV.compact(eta, odd)
    full = SV.expand(xo, odd)
    ref = SV.compact(W.M_hat(U, full, p, par3), odd)
    refd = SV.compact(W.M_hat_dag(U, full, p, par3), odd)
    x = _dev(xo)
    assert _rel(_host(w.apply_schur(x)), ref) < 1e-12
    assert _rel(_host(w.apply_schur(x, dagger=True)), refd) < 1e-12
    assert _rel(_host(w.apply_schur(x, f32=True)), ref) < 1e-6
    assert _rel(_host(w.apply_schur(x, dagger=True, f32=True)), refd) < 1e-6


@pytest.mark.parametrize("scheme", ["fp64", "fp32_dc", "fp32_ru", "eo4d"])
def test_solves(case, scheme, monkeypatch):
    p, U, eta, w = case
    method, precision = wf.WF_TEMPORAL_SCHUR, wf.WF_FP32
    if scheme == "fp64":
        precision = wf.WF_FP64
    elif scheme == "fp32_ru":
        monkeypatch.setenv("WF_DC", "0")
    elif scheme == "eo4d":
        if p.T % 2:
            pytest.skip("the 4-D checkerboard needs an even T")
        method = wf.WF_EO4D
    x, iters, res, status = w.solve(_dev(eta), tol=1e-10, method=method, precision=precision)
    assert status == wf.WF_OK and max(res) <= 1e-10
    psi = _host(x)
    for k in range(eta.shape[0]):
        assert SV.true_residual(U, psi[k], eta[k], p) <= TRUE_RESID


def test_long_lines_refuse_fp16_storage():
    L, T = 2, 160
    w = wf.Wilson(L, T, 0.07, kappa_t=0.245, bc=-1)
    try:
        w.load_gauge(S.random_gauge(L, T, 0.3, 25))
        eta = S.gaussian_source(L, T, 26, nrhs=1)
        with pytest.raises(wf.WFError) as e:
            w.solve(_dev(eta), tol=1e-10, precision=wf.WF_FP16MIX)
        assert e.value.code == wf.WF_EINVAL
        x, iters, res, status = w.solve(_dev(eta), tol=1e-10, precision=wf.WF_FP32)
        assert status == wf.WF_OK and res[0] <= 1e-10
    finally:
        w.close()
