"""The opt-in TMA-fed hop kernels (WF_TMA=1): parity, and the bounded-wait failure path.

The failure path is exercised without any GPU fault: the host asks the kernel to skip one
bulk copy (WF_TEST_DROP_COPY), so one mbarrier wait can never complete; the wait runs out
after its iteration limit, the kernel sets its error word, drains and returns, and the call
must report WF_ETIMEOUT with the context still usable.
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


def _setup():
    L, T = 4, 128
    p = W.Params(L, T, 0.074, xi=3.5, bc=-1)
    U = S.random_gauge(L, T, 0.2, 5)
    eta = S.gaussian_source(L, T, 105, nrhs=2)
    par3 = W.parity3(L, T)
    xo = SV.compact(eta, par3 == 1)
    ref = SV.compact(W.M_hat(U, SV.expand(xo, par3 == 1), p, par3), par3 == 1)
    return p, U, eta, xo, ref


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_tma_kernels_parity(monkeypatch):
    monkeypatch.setenv("WF_TMA", "1")
    p, U, eta, xo, ref = _setup()
    w = wf.Wilson(p.L, p.T, p.kappa_s, kappa_t=p.kappa_t, bc=-1)
    w.load_gauge(U)
    out = w.apply_schur(_dev(xo), f32=True).cpu().numpy()
    assert _rel(out, ref) < 1e-6
    x, iters, res, status = w.solve(_dev(eta), tol=1e-10, precision=wf.WF_FP32)
    assert status == wf.WF_OK and max(res) <= 1e-10
    w.close()


def test_expired_wait_reports_timeout_and_context_survives(monkeypatch):
    monkeypatch.setenv("WF_TMA", "1")
    p, U, eta, xo, ref = _setup()
    w = wf.Wilson(p.L, p.T, p.kappa_s, kappa_t=p.kappa_t, bc=-1)
    w.load_gauge(U)
    x = _dev(xo)
    monkeypatch.setenv("WF_TEST_DROP_COPY", "3")
    with pytest.raises(wf.WFError) as e:
        w.apply_schur(x, f32=True)
    assert e.value.code == wf.WF_ETIMEOUT
    monkeypatch.delenv("WF_TEST_DROP_COPY")
    out = w.apply_schur(x, f32=True).cpu().numpy()   # same handle, same context
    assert _rel(out, ref) < 1e-6
    w.close()
