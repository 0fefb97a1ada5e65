"""Parity at the benchmark's full size, in the launch configuration bench.py times.

24^3 x 128, xi = 3.5: twelve right-hand sides per launch with the autotuned FP32 hop kernels.
The oracle computes sampled outputs: one source of a batched M-hat apply against the oracle's
full-lattice M-hat (FP32 tolerance, 1e-6 relative), and the solve of the twelve point sources
checked by the oracle's M on two sampled sources (FP64 true residual <= 1e-10 plus 1e-13 for the
rounding difference between the two FP64 evaluations of the same residual);
and log det(mu - D_t) with its force on the whole lattice (1e-13 / 1e-11 relative).
Each oracle evaluation at this size takes tens of seconds on the host.
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

NAME = "wilson_24c128_xi3.5"


@pytest.fixture(scope="module")
def full():
    prm, U, eta = S.workload(NAME)
    p = W.Params(prm["L"], prm["T"], prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"])
    w = wf.Wilson(prm["L"], prm["T"], prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"])
    stream = torch.cuda.Stream()
    w.set_stream(stream.cuda_stream)
    w.load_gauge(U)
    yield p, U, eta, w
    w.close()


def test_full_size_batched_schur_apply_sampled(full):
    p, U, _, w = full
    nrhs = 12
    par3 = W.parity3(p.L, p.T)
    odd = par3 == 1
    src = S.gaussian_source(p.L, p.T, 1234, nrhs=nrhs)
    xo = np.ascontiguousarray(np.stack([SV.compact(src[k], odd) for k in range(nrhs)]))
    xd = torch.from_numpy(xo).cuda()
    w.apply_schur(xd, f32=True)  # the first 12-source apply runs the autotuner
    out = w.apply_schur(xd, f32=True).cpu().numpy()  # the tuned configuration bench.py times
    assert wf.wf_hop_config(w.h, nrhs) is not None
    k = 7
    ref = SV.compact(W.M_hat(U, SV.expand(xo[k], odd), p, par3), odd)
    err = np.linalg.norm(out[k] - ref) / np.linalg.norm(ref)
    assert err < 1e-6, err


def test_full_size_point_source_solve_sampled(full):
    p, U, eta, w = full
    x, iters, res, status = w.solve(torch.from_numpy(eta).cuda(), tol=1e-10, precision=wf.WF_FP32)
    assert status == wf.WF_OK and max(res) <= 1e-10
    psi = x.cpu().numpy()
    for k in (0, 11):
        assert SV.true_residual(U, psi[k], eta[k], p) <= 1e-10 + 1e-13


def test_full_size_temporal_logdet(full):
    """log det(mu - D_t) and its force on the whole 24^3 x 128 lattice (axial frame)."""
    from oracle import determinant as DT
    p, U, _, w = full
    F = torch.empty((p.T, p.L, p.L, p.L, 4, 8), dtype=torch.float64, device="cuda")
    got = w.temporal_logdet(F)
    ref = DT.logdet_temporal(U, p)
    assert abs(got - ref) <= 1e-13 * abs(ref)
    Fr = DT.force_logdet_temporal(U, p)
    Fg = F.cpu().numpy()
    assert np.linalg.norm((Fg - Fr).ravel()) <= 1e-11 * np.linalg.norm(Fr.ravel())
