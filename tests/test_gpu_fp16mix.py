"""FP16-stored spinors with FP32 arithmetic (WF_FP16MIX and wf_apply_schur_f16) against the
FP64 oracle.

Apply tolerance, derived from the storage: every stored value is a source's field divided by its
RMS and rounded to FP16 (unit roundoff 2^-11 = 4.9e-4, RMS rounding error about 2.8e-4 of a
component). The input, K-a's output, K-b's output and the result are each rounded once, and the
operator's norm is O(1), so the relative 2-norm error is about sqrt(4) * 2.8e-4 * O(1) ~ 1e-3;
the tests allow 3e-3 and also require the error to exceed 1e-6, which FP32 storage would not
reach (so the FP16 path is the one that ran). Solves must meet the FP64 true residual 1e-10 of
the full M (checked again with the oracle's M), in at most 1.5 times the FP32 iterations + 5, in
both FP32 schemes (defect correction and, with WF_DC=0, reliable updates).
"""

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
# L, T, kappa_s, xi, bc, eps, seed: 128-slot lines, a padded 128-slot line, the 96- and 48-slot layouts
LATTICES = [(4, 128, 0.074, 3.5, -1, 0.2, 5), (6, 100, 0.07, 3.5, 1, 0.25, 6), (4, 96, 0.06, 4.5, 1, 0.25, 8),
            (4, 48, 0.075, 3.0, -1, 0.25, 7)]


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("lat", LATTICES, ids=lambda c: f"L{c[0]}T{c[1]}")
def test_fp16_apply_parity(lat):
    L, T, ks, xi, bc, eps, seed = lat
    p = W.Params(L, T, ks, xi=xi, bc=bc)
    U = S.random_gauge(L, T, eps, seed)
    eta = S.gaussian_source(L, T, seed + 100, nrhs=3)
    eta[2] *= 1e7  # a source far outside the FP16 range: stored divided by its RMS
    par3 = W.parity3(L, T)
    xo = SV.compact(eta, par3 == 1)
    full = SV.expand(xo, par3 == 1)
    w = wf.Wilson(L, T, ks, kappa_t=xi * ks, bc=bc)
    try:
        w.load_gauge(U)
        for dagger in (0, 1):
            ref = SV.compact((W.M_hat_dag if dagger else W.M_hat)(U, full, p, par3), par3 == 1)
            out = torch.empty_like(_dev(xo))
            wf.wf_apply_schur_f16(w.h, _dev(xo), out, dagger, 3)
            out = out.cpu().numpy()
            for k in range(3):
                err = _rel(out[k], ref[k])
                assert 1e-6 < err < 3e-3, (dagger, k, err)
    finally:
        w.close()


@pytest.mark.parametrize("scheme", ["dc", "ru"])
@pytest.mark.parametrize("lat", LATTICES, ids=lambda c: f"L{c[0]}T{c[1]}")
def test_fp16mix_solve(lat, scheme, monkeypatch):
    """FP16 storage inside defect-correction passes (default), or with FP64 reliable updates and
    FP64 S_L / S_R (WF_DC=0); the FP32 solve of the same scheme sets the iteration bar."""
    if scheme == "ru":
        monkeypatch.setenv("WF_DC", "0")
    L, T, ks, xi, bc, eps, seed = lat
    p = W.Params(L, T, ks, xi=xi, bc=bc)
    U = S.random_gauge(L, T, eps, seed)
    eta = S.gaussian_source(L, T, seed + 200, nrhs=3)
    eta[1] = 0.0
    eta[1].reshape(-1)[0] = 1.0  # a point source next to the Gaussian ones
    eta[2] *= 1e-6               # and one of another scale
    w = wf.Wilson(L, T, ks, kappa_t=xi * ks, bc=bc)
    try:
        w.load_gauge(U)
        _, it32, _, st32 = w.solve(_dev(eta), tol=1e-10, precision=wf.WF_FP32)
        assert st32 == wf.WF_OK
        x, iters, res, status = w.solve(_dev(eta), tol=1e-10, precision=wf.WF_FP16MIX)
        assert status == wf.WF_OK and max(res) <= 1e-10
        xs = x.cpu().numpy()
        for k in range(3):
            assert SV.true_residual(U, xs[k], eta[k], p) <= TRUE_RESID
            assert iters[k] <= 1.5 * it32[k] + 5, (iters, it32)
    finally:
        w.close()


def test_fp16mix_scope():
    """FP16 storage serves the temporal + Schur method in the axial frame; other requests are refused."""
    L, T = 4, 16
    U = S.random_gauge(L, T, 0.3, 9)
    eta = S.gaussian_source(L, T, 10)
    w = wf.Wilson(L, T, 0.075, kappa_t=0.26, bc=-1)
    g = wf.Wilson(L, T, 0.075, kappa_t=0.26, bc=-1, axial=False)
    try:
        w.load_gauge(U)
        g.load_gauge(U)
        for method in (wf.WF_EO4D, wf.WF_UNPREC, wf.WF_TEMPORAL):
            with pytest.raises(wf.WFError) as e:
                w.solve(_dev(eta[None]), tol=1e-10, method=method, precision=wf.WF_FP16MIX)
            assert e.value.code == wf.WF_EINVAL
        with pytest.raises(wf.WFError) as e:
            g.solve(_dev(eta[None]), tol=1e-10, precision=wf.WF_FP16MIX)
        assert e.value.code == wf.WF_EINVAL
        x, iters, res, status = w.solve(_dev(eta[None]), tol=1e-10, precision=wf.WF_FP16MIX)
        assert status == wf.WF_OK and res[0] <= 1e-10
    finally:
        w.close()
        g.close()
