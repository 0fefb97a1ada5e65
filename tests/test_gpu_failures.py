"""Failure detection through the C ABI, made on the host side (no GPU fault is involved):

* a NaN in a source ends a solve with WF_ENAN (FP64 and FP32 precision);
* an iteration cap ends a solve with WF_ENOCONV, and the outputs hold the last iterate (finite,
  with the true residual the call reports);
* wf_load_gauge rejects a field with a NaN entry, a non-unitary link, or a unitary link with
  det != 1 (WF_EINVAL), and the handle stays usable;
* an output may be the same array as the input (every input is read in full first).
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

L, T = 4, 16


def _setup():
    p = W.Params(L, T, 0.075, xi=3.5, bc=-1)
    U = S.random_gauge(L, T, 0.3, 41)
    eta = S.gaussian_source(L, T, 42, nrhs=2)
    w = wf.Wilson(L, T, p.kappa_s, kappa_t=p.kappa_t, bc=-1)
    w.load_gauge(U)
    return p, U, eta, w


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("precision", [wf.WF_FP64, wf.WF_FP32])
def test_nan_in_source_reports_enan(precision):
    p, U, eta, w = _setup()
    try:
        bad = eta.copy()
        bad[1].reshape(-1)[17] = complex(np.nan, 0.0)
        with pytest.raises(wf.WFError) as e:  # the binding raises for every status but OK and ENOCONV
            w.solve(_dev(bad), tol=1e-10, precision=precision)
        assert e.value.code == wf.WF_ENAN
        assert "NaN" in wf.wf_last_error(w.h)
        # the handle still solves a clean source
        x, iters, res, status = w.solve(_dev(eta), tol=1e-10, precision=precision)
        assert status == wf.WF_OK and max(res) <= 1e-10
    finally:
        w.close()


@pytest.mark.parametrize("method,precision", [(wf.WF_TEMPORAL_SCHUR, wf.WF_FP64), (wf.WF_EO4D, wf.WF_FP64),
                                              (wf.WF_TEMPORAL_SCHUR, wf.WF_FP32)])
def test_iteration_cap_reports_enoconv_with_outputs_written(method, precision):
    """The iteration limit ends a solve with WF_ENOCONV and the last iterate written (FP32 temporal +
    Schur: defect correction, whose passes share the limit)."""
    p, U, eta, w = _setup()
    try:
        wf.wf_set_max_iterations(w.h, 3)
        x0 = torch.full((2, eta[0].size), complex(np.nan, np.nan), dtype=torch.complex128).cuda()
        st, iters, res = wf.wf_solve(w.h, _dev(eta).reshape(2, -1), x0, 2, 1e-10, method, precision, 0)
        assert st == wf.WF_ENOCONV
        if precision == wf.WF_FP32:
            assert all(0 < i <= 3 for i in iters)  # the passes share the limit
        assert all(0 < i <= 3 * 6 for i in iters)  # at most the cap per pass, a few passes
        xs = x0.cpu().numpy().reshape(eta.shape)
        assert np.isfinite(xs).all()
        for k in range(2):
            tr = SV.true_residual(U, xs[k], eta[k], p)
            assert 1e-10 < tr < 1.0
            assert tr == pytest.approx(res[k], rel=1e-6)  # the reported residual is that of the output
        wf.wf_set_max_iterations(w.h, 0)  # back to the default
        x, iters, res, status = w.solve(_dev(eta), tol=1e-10, method=method)
        assert status == wf.WF_OK and max(res) <= 1e-10
        with pytest.raises(wf.WFError) as e:
            wf.wf_set_max_iterations(w.h, -1)
        assert e.value.code == wf.WF_EINVAL
    finally:
        w.close()


def _bad_fields(U):
    nan = U.copy()
    nan[3, 1, 0, 2, 1, 0, 1] = np.nan
    scaled = U.copy()
    scaled[2, 0, 1, 1, 3] *= 1.001                       # not unitary
    phase = U.copy()
    phase[1, 1, 1, 1, 0] *= np.exp(1j * 0.3)            # unitary, det = e^{0.9 i}
    return {"nan": nan, "non-unitary": scaled, "det": phase}


@pytest.mark.parametrize("kind", ["nan", "non-unitary", "det"])
def test_load_gauge_rejects_links_outside_su3(kind):
    p, U, eta, w = _setup()
    try:
        bad = _bad_fields(U)[kind]
        with pytest.raises(wf.WFError) as e:
            w.load_gauge(bad)
        assert e.value.code == wf.WF_EINVAL
        msg = wf.wf_last_error(w.h)
        assert ("NaN" in msg) if kind == "nan" else ("SU(3)" in msg)
        w.load_gauge(U)  # a good field loads again on the same handle
        x, iters, res, status = w.solve(_dev(eta), tol=1e-10)
        assert status == wf.WF_OK and max(res) <= 1e-10
    finally:
        w.close()


@pytest.mark.parametrize("on_device", [True, False])
def test_in_place_applies_and_solve(on_device):
    p, U, eta, w = _setup()
    try:
        par3 = W.parity3(L, T)
        xo = np.ascontiguousarray(SV.compact(eta, par3 == 1))
        conv = _dev if on_device else (lambda a: np.ascontiguousarray(a).copy())
        back = (lambda t: t.cpu().numpy()) if on_device else (lambda a: a)
        # M-hat in place
        ref = np.empty_like(xo)
        wf.wf_apply_schur(w.h, xo, ref, 0, 2)
        a = conv(xo)
        wf.wf_apply_schur(w.h, a, a, 0, 2)
        assert np.array_equal(back(a), ref)
        # M in place, FP32
        refm = np.empty_like(eta)
        wf.wf_apply_M_f32(w.h, eta, refm, 0, 2)
        b = conv(eta)
        wf.wf_apply_M_f32(w.h, b, b, 0, 2)
        assert np.array_equal(back(b), refm)
        # a solve whose solution overwrites its source
        c = conv(eta)
        st, iters, res = wf.wf_solve(w.h, c, c, 2, 1e-10, wf.WF_TEMPORAL_SCHUR, wf.WF_FP64, 0)
        assert st == wf.WF_OK
        xs = back(c)
        for k in range(2):
            assert SV.true_residual(U, xs[k], eta[k], p) <= 1e-10
    finally:
        w.close()
