"""GPU parity: every C-ABI apply and solve against the FP64 oracle (needs a GB300).

Tolerances (relative 2-norm over the whole output): 1e-12 for FP64 applies and
1e-6 for FP32 applies; solves must reach an FP64 true residual ||eta - M psi|| /
||eta|| <= 1e-10, checked again here with the oracle's own M.

Lattices span several warps and lines per warp, padded time lines (T not a
multiple of the lane segment) and both boundary conditions.
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

CASES = [
    # L, T, kappa_s, xi, bc, eps, seed
    (4, 16, 0.12, 3.0, -1, 0.3, 1),      # the 4^3 x 16 workload's parameters
    (2, 6, 0.07, 3.0, -1, 0.4, 2),       # 3 sites per lane, 2 lanes per line
    (4, 7, 0.08, 2.5, 1, 0.3, 3),        # odd T: padded slot, periodic
    (6, 12, 0.075, 3.5, -1, 0.3, 4),     # L = 6
    (4, 128, 0.074, 3.5, -1, 0.2, 5),    # 4 sites per lane, full warp per line
    (8, 32, 0.07, 3.0, 1, 0.25, 6),      # many warps
    (4, 48, 0.075, 3.0, -1, 0.25, 7),    # the xi-sweep's 48-slot layout: 3 sites per lane, 16 lanes, 2 lines per warp
    (4, 96, 0.06, 4.5, 1, 0.25, 8),      # the xi-sweep's 96-slot layout: 3 sites per lane, full warp per line
]

# The oracle recomputes ||eta - M psi|| / ||eta|| with its own M for a solution the library
# accepted at <= 1e-10. The two FP64 evaluations of the same residual differ only by rounding:
# each site's eta - M psi is formed from O(||eta||)-sized terms with errors of a few eps_64, so
# the relative difference is ~1e-15; TRUE_RESID allows 1e-13 of it.
TRUE_RESID = 1e-10 + 1e-13


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    return t.cpu().numpy()


FRAMES = [True, False]  # axial frame (default), caller's gauge


@pytest.fixture(scope="module", params=[(c, ax) for c in CASES for ax in FRAMES],
                ids=lambda ca: f"L{ca[0][0]}T{ca[0][1]}bc{ca[0][4]}-{'axial' if ca[1] else 'general'}")
def case(request):
    (L, T, ks, xi, bc, eps, seed), axial = request.param
    p = W.Params(L, T, ks, xi=xi, bc=bc)
    U = S.random_gauge(L, T, eps, seed)
    eta = S.gaussian_source(L, T, seed + 100, nrhs=2)
    w = wf.Wilson(L, T, ks, kappa_t=xi * ks, bc=bc, axial=axial)
    w.load_gauge(U)
    yield p, U, eta, w
    w.close()


def test_apply_M(case):
    p, U, eta, w = case
    x = _dev(eta)
    ref = W.M(U, eta, p)
    assert _rel(_host(w.apply_M(x)), ref) < 1e-12
    refd = W.M_dag(U, eta, p)
    assert _rel(_host(w.apply_M(x, dagger=True)), refd) < 1e-12
    assert _rel(_host(w.apply_M(x, f32=True)), ref) < 1e-6


def test_apply_Tinv(case):
    p, U, eta, w = case
    x = _dev(eta)
    assert _rel(_host(w.apply_Tinv(x)), W.Tinv(U, eta, p)) < 1e-12
    assert _rel(_host(w.apply_Tinv(x, dagger=True)), W.Tdag_inv(U, eta, p)) < 1e-12
    assert _rel(_host(w.apply_Tinv(x, f32=True)), W.Tinv(U, eta, p)) < 1e-6


def test_apply_C(case):
    p, U, eta, w = case
    x = _dev(eta)
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


def test_host_pointers_match_device(case):
    p, U, eta, w = case
    par3 = W.parity3(p.L, p.T)
    xo = np.ascontiguousarray(SV.compact(eta, par3 == 1))
    a = w.apply_schur(xo)               # NumPy in, NumPy out: host staging in the library
    b = _host(w.apply_schur(_dev(xo)))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [wf.WF_FP64, wf.WF_FP32, "fp32_reliable_updates"])
def test_solve_temporal_schur(case, precision, monkeypatch):
    """FP64 CG; FP32 by defect correction (the default); FP32 with reliable updates (WF_DC=0)."""
    p, U, eta, w = case
    if precision == "fp32_reliable_updates":
        monkeypatch.setenv("WF_DC", "0")
        precision = wf.WF_FP32
    x, iters, res, status = w.solve(_dev(eta), tol=1e-10, precision=precision)
    assert status == wf.WF_OK
    assert all(r <= 1e-10 for r in res)
    assert all(i > 0 for i in iters)
    psi = _host(x)
    for k in range(eta.shape[0]):
        assert SV.true_residual(U, psi[k], eta[k], p) <= TRUE_RESID


def test_solve_matches_oracle_solution():
    """4^3 x 16 workload: the GPU solution equals the oracle's (unique solution, bound by kappa * tol)."""
    prm, U, eta = S.workload("wilson_4c16_xi3")
    p = W.Params(prm["L"], prm["T"], prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"])
    w = wf.Wilson(prm["L"], prm["T"], prm["kappa_s"], kappa_t=prm["kappa_t"], bc=prm["bc"])
    w.load_gauge(U)
    psi_ref, it_ref, _ = SV.solve(U, eta[0], p, "temporal_schur", tol=1e-12)
    x, iters, res, status = w.solve(_dev(eta), tol=1e-10, precision=wf.WF_FP32)
    assert status == wf.WF_OK and res[0] <= 1e-10
    assert _rel(_host(x)[0], psi_ref) < 1e-7
    w.close()


@pytest.mark.parametrize("axial", FRAMES)
def test_singular_preconditioner_is_reported(axial):
    """mu = 1 (kappa_t = 1/2), periodic, unit links: T has a zero mode, so Lambda does not exist."""
    L, T = 2, 4
    w = wf.Wilson(L, T, 0.25, kappa_t=0.5, bc=1, axial=axial)
    with pytest.raises(wf.WFError) as e:
        w.load_gauge(S.unit_gauge(L, T))
    assert e.value.code == wf.WF_ESINGULAR
    w.close()


def test_apply_eo4d(case):
    """The 4-D even-odd comparator M-hat_4 (§II.B, 4D-Schur) against the oracle, odd 4-D sites."""
    p, U, eta, w = case
    if p.T % 2:
        pytest.skip("the 4-D checkerboard needs an even T")
    par4 = W.parity4(p.L, p.T)
    odd = par4 == 1
    xo = SV.compact(eta, odd)
    full = SV.expand(xo, odd)
    ref = SV.compact(W.M_hat4(U, full, p, par4), odd)
    refd = SV.compact(W.M_hat4_dag(U, full, p, par4), odd)
    x = _dev(xo)
    assert _rel(_host(w.apply_eo4d(x)), ref) < 1e-12
    assert _rel(_host(w.apply_eo4d(x, dagger=True)), refd) < 1e-12
    assert _rel(_host(w.apply_eo4d(x, f32=True)), ref) < 1e-6


@pytest.mark.parametrize("method", [wf.WF_EO4D, wf.WF_UNPREC, wf.WF_TEMPORAL])
@pytest.mark.parametrize("precision", [wf.WF_FP64, wf.WF_FP32])
def test_solve_comparators(case, method, precision):
    """Every comparator method reaches the unique solution: FP64 true residual <= 1e-10, checked
    with the oracle's M."""
    p, U, eta, w = case
    if method == wf.WF_EO4D and p.T % 2:
        pytest.skip("the 4-D checkerboard needs an even T")
    x, iters, res, status = w.solve(_dev(eta), tol=1e-10, method=method, precision=precision)
    assert status == wf.WF_OK
    assert all(r <= 1e-10 for r in res)
    psi = _host(x)
    for k in range(eta.shape[0]):
        assert SV.true_residual(U, psi[k], eta[k], p) <= TRUE_RESID


def test_fp64_iterations_match_oracle():
    """FP64 CGNR on the GPU takes the oracle's iteration count for each method (same algorithm)."""
    L, T = 4, 8
    p = W.Params(L, T, 0.075, xi=3.5, bc=-1)
    U = S.random_gauge(L, T, 0.3, 21)
    eta = S.gaussian_source(L, T, 22)
    w = wf.Wilson(L, T, 0.075, kappa_t=3.5 * 0.075, bc=-1)
    w.load_gauge(U)
    for method, name in [(wf.WF_UNPREC, "unprec"), (wf.WF_EO4D, "eo4d"), (wf.WF_TEMPORAL, "temporal"),
                         (wf.WF_TEMPORAL_SCHUR, "temporal_schur")]:
        _, it_ref, _ = SV.solve(U, eta, p, name, tol=1e-10)
        _, iters, res, status = w.solve(_dev(eta[None]), tol=1e-10, method=method, precision=wf.WF_FP64)
        assert status == wf.WF_OK
        assert abs(iters[0] - it_ref) <= max(2, it_ref // 20), (name, iters[0], it_ref)
    w.close()


@pytest.mark.parametrize("L,T", [(4, 16), (4, 128), (4, 7)])
@pytest.mark.parametrize("method", [wf.WF_TEMPORAL_SCHUR, wf.WF_EO4D, wf.WF_TEMPORAL])
def test_solve_with_double_float_steps(monkeypatch, L, T, method):
    """WF_DF64=1 at handle creation: the FP64 steps of an FP32 solve with reliable updates
    (reliable updates, S_L, S_R, the comparators' reconstructions; WF_DC=0 for the temporal +
    Schur method) run in double-float; the FP64 true residual still decides."""
    if method == wf.WF_EO4D and T % 2:
        pytest.skip("the 4-D checkerboard needs an even T")
    monkeypatch.setenv("WF_DF64", "1")
    monkeypatch.setenv("WF_DC", "0")
    p = W.Params(L, T, 0.074, xi=3.5, bc=-1)
    U = S.random_gauge(L, T, 0.25, 41)
    eta = S.gaussian_source(L, T, 42, nrhs=2)
    w = wf.Wilson(L, T, 0.074, kappa_t=3.5 * 0.074, bc=-1)
    w.load_gauge(U)
    x, iters, res, status = w.solve(_dev(eta), tol=1e-10, method=method, precision=wf.WF_FP32)
    assert status == wf.WF_OK and all(r <= 1e-10 for r in res)
    psi = _host(x)
    for k in range(eta.shape[0]):
        assert SV.true_residual(U, psi[k], eta[k], p) <= TRUE_RESID
    w.close()


@pytest.mark.parametrize("L,T", [(4, 128), (8, 32), (6, 12)])
def test_autotuned_hop_kernels(monkeypatch, L, T):
    """The first FP32 Schur apply tunes the hop kernels (family, tile rows, and for the bulk-fed
    kernels sources per unit and stages); the result of every
    later apply, and of the tuning call itself, matches the oracle. WF_AUTOTUNE=0: no tuning."""
    p = W.Params(L, T, 0.07, xi=3.0, bc=-1)
    U = S.random_gauge(L, T, 0.3, 61)
    eta = S.gaussian_source(L, T, 62, nrhs=3)
    par3 = W.parity3(L, T)
    xo = np.ascontiguousarray(SV.compact(eta, par3 == 1))
    ref = SV.compact(W.M_hat(U, SV.expand(xo, par3 == 1), p, par3), par3 == 1)
    for tune in ("1", "0"):
        monkeypatch.setenv("WF_AUTOTUNE", tune)
        w = wf.Wilson(L, T, 0.07, kappa_t=0.21, bc=-1)
        w.load_gauge(U)
        assert wf.wf_hop_config(w.h, 3) is None
        for _ in range(2):
            assert _rel(_host(w.apply_schur(_dev(xo), f32=True)), ref) < 1e-6
        cfg = wf.wf_hop_config(w.h, 3)
        if tune == "1":
            assert cfg is not None and cfg[0] in (1, 2, 3) and L % cfg[1] == 0 and cfg[2] > 0
            gs, ns = wf.wf_hop_pipe_config(w.h, 3)
            # bulk-fed kernels only serve 128-slot lines; their group size and stages are reported
            assert (cfg[0] == 3) == (gs > 0) and (cfg[0] != 3 or (T > 96 and gs in (1, 2) and 2 <= ns <= 4))
        else:
            assert cfg is None
        w.close()


@pytest.mark.parametrize("method", [wf.WF_TEMPORAL_SCHUR, wf.WF_EO4D])
def test_solve_many_ragged_lattices(method):
    """wf_solve_many: three lattices of different sizes in one call, each on its own stream and host
    thread; every solution meets the FP64 true residual and the iteration counts of the same solves
    made one at a time (within one iteration: the norms' summation order differs)."""
    shapes = [(4, 16, 0.074), (6, 12, 0.07), (4, 8, 0.075)]
    hs, ws, rhs, xs, refs, prms = [], [], [], [], [], []
    for i, (L, T, ks) in enumerate(shapes):
        p = W.Params(L, T, ks, xi=3.5, bc=-1)
        U = S.random_gauge(L, T, 0.25, 70 + i)
        eta = S.gaussian_source(L, T, 80 + i, nrhs=2)
        w = wf.Wilson(L, T, ks, kappa_t=3.5 * ks, bc=-1)
        w.load_gauge(U)
        _, it1, _, st1 = w.solve(_dev(eta), tol=1e-10, method=method, precision=wf.WF_FP32)
        assert st1 == wf.WF_OK
        ws.append(w); hs.append(w.h); rhs.append(_dev(eta)); xs.append(torch.empty_like(rhs[-1]))
        refs.append((U, eta, it1)); prms.append(p)
    st, per = wf.wf_solve_many(hs, rhs, xs, [2, 2, 2], 1e-10, method, wf.WF_FP32)
    assert st == wf.WF_OK
    for (U, eta, it1), p, x, (sti, its, res) in zip(refs, prms, xs, per):
        assert sti == wf.WF_OK and max(res) <= 1e-10
        assert all(abs(a - b) <= 1 for a, b in zip(its, it1))
        psi = _host(x)
        for k in range(eta.shape[0]):
            assert SV.true_residual(U, psi[k], eta[k], p) <= TRUE_RESID
    for w in ws:
        w.close()


def test_solve_many_rejects_a_shared_handle():
    L, T = 4, 8
    w = wf.Wilson(L, T, 0.075, kappa_t=0.26, bc=-1)
    w.load_gauge(S.random_gauge(L, T, 0.2, 90))
    eta = _dev(S.gaussian_source(L, T, 91, nrhs=1))
    x = torch.empty_like(eta)
    st, _ = wf.wf_solve_many([w.h, w.h], [eta, eta], [x, x], [1, 1], 1e-10, wf.WF_TEMPORAL_SCHUR, wf.WF_FP32)
    assert st == wf.WF_EINVAL
    w.close()


def test_solve_with_pinned_host_arrays():
    """Page-locked host arrays for rhs and x (staged by the library): the solution equals the one
    from device arrays bit for bit, also with an initial guess and for a ragged call."""
    L, T = 4, 16
    p = W.Params(L, T, 0.075, xi=3.5, bc=-1)
    U = S.random_gauge(L, T, 0.25, 51)
    eta = S.gaussian_source(L, T, 52, nrhs=2)
    w = wf.Wilson(L, T, 0.075, kappa_t=3.5 * 0.075, bc=-1)
    try:
        w.load_gauge(U)
        xd = torch.empty_like(_dev(eta))
        st, it_d, _ = wf.wf_solve(w.h, _dev(eta), xd, 2, 1e-10, wf.WF_TEMPORAL_SCHUR, wf.WF_FP32, 0)
        assert st == wf.WF_OK
        rh = torch.from_numpy(np.ascontiguousarray(eta)).pin_memory()
        xh = torch.zeros_like(rh).pin_memory()
        st, it_h, res = wf.wf_solve(w.h, rh, xh, 2, 1e-10, wf.WF_TEMPORAL_SCHUR, wf.WF_FP32, 0)
        assert st == wf.WF_OK and it_h == it_d
        assert np.array_equal(xh.numpy(), _host(xd))
        for k in range(2):
            assert SV.true_residual(U, xh.numpy()[k], eta[k], p) <= TRUE_RESID
        # from the solution as initial guess (read in place) the solve stays at tol
        st, it0, res0 = wf.wf_solve(w.h, rh, xh, 2, 1e-10, wf.WF_TEMPORAL_SCHUR, wf.WF_FP32, wf.WF_X0)
        assert st == wf.WF_OK and max(res0) <= 1e-10
        # a ragged call with pinned arrays
        xh2 = torch.zeros_like(rh).pin_memory()
        st, per = wf.wf_solve_many([w.h], [rh], [xh2], [2], 1e-10, wf.WF_TEMPORAL_SCHUR, wf.WF_FP32)
        assert st == wf.WF_OK and np.array_equal(xh2.numpy(), _host(xd))
    finally:
        w.close()
