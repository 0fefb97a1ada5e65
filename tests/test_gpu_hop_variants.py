"""The bulk-copy-fed hop kernels of M-hat (K-b, K-c fed by cp.async.bulk into shared-memory
stages): parity of every configuration against the FP64 oracle, FP32 solves through them, and the
bounded-wait failure path.

A configuration is fixed per handle with WF_HOP=pipe,<sources per unit>,<stages>,<tile rows>,
which the library reads at a handle's first FP32 Schur apply for a given source count. The
lattices have 128-slot time lines (the kernels' domain): a full one (T = 128) and a padded one
(T = 100); source counts 1, 2, 3 and 6 give units whose sources are all live and half-empty last
groups.
Tolerance: 1e-6 relative (FP32 applies), as in the other parity tests.

The failure path is driven without any GPU fault: the host asks the producer warp to skip the
copies of one job, so one mbarrier phase never completes; the consumers' bounded waits run out,
the kernel sets its error word, drains and returns, and the call reports WF_ETIMEOUT with the
context still usable.
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

CONFIGS = ["pipe,1,2", "pipe,1,3", "pipe,1,4", "pipe,2,2", "pipe,2,3"]
LATTICES = [(4, 128, -1, 5), (6, 100, 1, 6)]         # L, T, bc, seed


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _problem(L, T, bc, seed, nrhs):
    p = W.Params(L, T, 0.074, xi=3.5, bc=bc)
    U = S.random_gauge(L, T, 0.2, seed)
    eta = S.gaussian_source(L, T, seed + 100, nrhs=nrhs)
    par3 = W.parity3(L, T)
    xo = SV.compact(eta, par3 == 1)
    return p, U, eta, xo, par3


def _oracle_mhat(U, xo, p, par3, dagger):
    v = SV.expand(xo, par3 == 1)
    out = W.M_hat_dag(U, v, p, par3) if dagger else W.M_hat(U, v, p, par3)
    return SV.compact(out, par3 == 1)


def _expect(cfg):
    _, g, ns = cfg.split(",")
    return 3, (int(g), int(ns))


@pytest.mark.parametrize("lat", LATTICES, ids=lambda c: f"L{c[0]}T{c[1]}")
@pytest.mark.parametrize("cfg", CONFIGS)
def test_hop_variant_apply_parity(monkeypatch, lat, cfg):
    L, T, bc, seed = lat
    monkeypatch.setenv("WF_HOP", f"{cfg},2")
    p, U, eta, xo, par3 = _problem(L, T, bc, seed, 6)
    w = wf.Wilson(L, T, p.kappa_s, kappa_t=p.kappa_t, bc=bc)
    variant, pipe_cfg = _expect(cfg)
    try:
        w.load_gauge(U)
        for nrhs in (1, 2, 3, 6):
            for dagger in (0, 1):
                ref = _oracle_mhat(U, xo[:nrhs], p, par3, dagger)
                out = w.apply_schur(_dev(xo[:nrhs]), dagger=bool(dagger), f32=True).cpu().numpy()
                assert _rel(out, ref) < 1e-6, (nrhs, dagger)
            assert wf.wf_hop_config(w.h, nrhs)[0] == variant
            assert wf.wf_hop_pipe_config(w.h, nrhs) == pipe_cfg
    finally:
        w.close()


@pytest.mark.parametrize("scheme", ["dc", "ru"])
@pytest.mark.parametrize("cfg", ["pipe,1,3", "pipe,2,2"])
def test_hop_variant_fp32_solve(monkeypatch, cfg, scheme):
    """Three sources through the FP32 CG (defect correction, or reliable updates with WF_DC=0);
    sources stop at different iterations, so the kernels also run units whose sources are partly
    stopped."""
    monkeypatch.setenv("WF_HOP", f"{cfg},2")
    if scheme == "ru":
        monkeypatch.setenv("WF_DC", "0")
    L, T, bc, seed = LATTICES[0]
    p, U, eta, xo, par3 = _problem(L, T, bc, seed, 3)
    eta[1] = 0.0
    eta[1].reshape(-1)[0] = 1.0  # a point source converges at another iteration than the Gaussian ones
    w = wf.Wilson(L, T, p.kappa_s, kappa_t=p.kappa_t, bc=bc)
    try:
        w.load_gauge(U)
        x, iters, res, status = w.solve(_dev(eta), tol=1e-10, precision=wf.WF_FP32)
        assert status == wf.WF_OK and max(res) <= 1e-10
        xs = x.cpu().numpy()
        for k in range(3):
            assert SV.true_residual(U, xs[k], eta[k], p) <= 1e-10 * (1 + 1e-3)
        assert wf.wf_hop_config(w.h, 3)[0] == _expect(cfg)[0]
    finally:
        w.close()


def test_pipe_expired_wait_reports_timeout_and_context_survives(monkeypatch):
    monkeypatch.setenv("WF_HOP", "pipe,1,3,2")
    L, T, bc, seed = LATTICES[0]
    p, U, eta, xo, par3 = _problem(L, T, bc, seed, 2)
    ref = _oracle_mhat(U, xo, p, par3, 0)
    w = wf.Wilson(L, T, p.kappa_s, kappa_t=p.kappa_t, bc=bc)
    try:
        w.load_gauge(U)
        x = _dev(xo)
        out = w.apply_schur(x, f32=True).cpu().numpy()   # tuned (fixed) before the drop
        assert _rel(out, ref) < 1e-6
        monkeypatch.setenv("WF_TEST_DROP_COPY", "4")
        with pytest.raises(wf.WFError) as e:
            w.apply_schur(x, f32=True)
        assert e.value.code == wf.WF_ETIMEOUT
        monkeypatch.delenv("WF_TEST_DROP_COPY")
        out = w.apply_schur(x, f32=True).cpu().numpy()   # same handle, same context
        assert _rel(out, ref) < 1e-6
    finally:
        w.close()
