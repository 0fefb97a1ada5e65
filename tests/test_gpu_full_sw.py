"""GPU parity of full SW temporal preconditioning (§II.A, SW paragraphs; appendix "Full
Preconditioning with Clover") against ``oracle/clover.py``.

Q^-1 = (A + mu - D_t)^-1 (FP64 1e-12, FP32 1e-5) and M-hat_full with its adjoint (same
tolerances) on lattices with several warps, padded and odd time lines, a 160-site line (five
sites per lane), both boundary conditions and both frames, with two and five sources; without a
clover term Q^-1 equals the Wilson C_R C_L; the kept factors follow every reload of the field; solves of M_SW in FP64 and by FP32 defect correction
to the oracle-checked 1e-10 true residual, in the oracle's iteration count (FP64); host arrays;
and the errors (precision, arguments, iteration limit, NaN source).
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

TRUE_RESID = 1e-10 + 1e-13  # the rounding room of two FP64 evaluations of one residual
CASES = [
    # L, T, kappa_s, xi, bc, eps, seed, c_s, c_t
    (2, 8, 0.08, 3.0, -1, 0.5, 41, 1.1, 0.9),
    (4, 12, 0.07, 3.5, 1, 0.3, 42, 1.2, 0.8),
    (4, 7, 0.08, 2.5, -1, 0.3, 43, 1.0, 1.0),
    (4, 128, 0.074, 3.5, -1, 0.2, 44, 0.45, 0.75),
    (2, 160, 0.07, 3.5, 1, 0.3, 45, 0.8, 0.9),
]
SOLVE_CASES = {(2, 8), (4, 12), (4, 7)}
_ORACLE = {}


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _oracle(key, fn):
    """The oracle's results depend on the case only, not on the library's frame: computed once."""
    if key not in _ORACLE:
        _ORACLE[key] = fn()
    return _ORACLE[key]


@pytest.fixture(scope="module", params=[(c, ax) for c in CASES for ax in (True, False)],
                ids=lambda ca: f"L{ca[0][0]}T{ca[0][1]}bc{ca[0][4]}-{'axial' if ca[1] else 'general'}")
def case(request):
    (L, T, ks, xi, bc, eps, seed, c_s, c_t), axial = request.param
    p = W.Params(L, T, ks, xi=xi, bc=bc)
    U = S.random_gauge(L, T, eps, seed)
    Acl = _oracle((L, T, "A"), lambda: CL.clover_term(U, c_s, c_t))
    eta = S.gaussian_source(L, T, seed + 100, nrhs=2)
    w = wf.Wilson(L, T, ks, kappa_t=xi * ks, bc=bc, axial=axial)
    w.load_gauge_clover(U, c_s, c_t)
    yield (L, T), p, U, Acl, eta, w
    w.close()


def test_qinv(case):
    key, p, U, Acl, eta, w = case
    ref = _oracle(key + ("Qinv",), lambda: CL.Q_inverse(U, Acl, eta, p))
    x = _dev(eta)
    assert _rel(w.apply_Qinv(x).cpu().numpy(), ref) < 1e-12
    assert _rel(w.apply_Qinv(x, f32=True).cpu().numpy(), ref) < 1e-5


def test_qinv_many_sources(case):
    """Five sources: groups of one CTA on different lines and sources; their FP32 solve."""
    key, p, U, Acl, eta, w = case
    if key not in ((4, 12), (2, 160)):
        pytest.skip("two layouts suffice")
    eta5 = S.gaussian_source(p.L, p.T, 149, nrhs=5)
    ref = _oracle(key + ("Qinv5",), lambda: CL.Q_inverse(U, Acl, eta5, p))
    x = _dev(eta5)
    assert _rel(w.apply_Qinv(x).cpu().numpy(), ref) < 1e-12
    assert _rel(w.apply_Qinv(x, f32=True).cpu().numpy(), ref) < 1e-5
    x5, iters, res, status = w.solve_full_sw(x, tol=1e-10, precision=wf.WF_FP32)
    assert status == wf.WF_OK and max(res) <= 1e-10
    psi = x5.cpu().numpy()
    assert max(CL.true_residual(U, Acl, psi[k], eta5[k], p) for k in range(5)) <= TRUE_RESID


def test_schur_full(case):
    key, p, U, Acl, eta, w = case
    par3 = W.parity3(p.L, p.T)
    odd = par3 == 1
    xo = SV.compact(eta, odd)
    full = SV.expand(xo, odd)
    ref = _oracle(key + ("Mhat",), lambda: SV.compact(CL.M_hat_full_sw(U, Acl, full, p, par3), odd))
    refd = _oracle(key + ("Mhat_dag",), lambda: SV.compact(CL.M_hat_full_sw_dag(U, Acl, full, p, par3), odd))
    x = _dev(xo)
    assert _rel(w.apply_schur_full_sw(x).cpu().numpy(), ref) < 1e-12
    assert _rel(w.apply_schur_full_sw(x, dagger=True).cpu().numpy(), refd) < 1e-12
    assert _rel(w.apply_schur_full_sw(x, f32=True).cpu().numpy(), ref) < 1e-5
    assert _rel(w.apply_schur_full_sw(x, dagger=True, f32=True).cpu().numpy(), refd) < 1e-5


@pytest.mark.parametrize("precision", [wf.WF_FP64, wf.WF_FP32], ids=["fp64", "fp32_dc"])
def test_solve(case, precision):
    key, p, U, Acl, eta, w = case
    if key not in SOLVE_CASES:
        pytest.skip("solves on the small lattices (the oracle's reference solve is slow at N_t >= 128)")
    x, iters, res, status = w.solve_full_sw(_dev(eta), tol=1e-10, precision=precision)
    assert status == wf.WF_OK and max(res) <= 1e-10
    psi = x.cpu().numpy()
    for k in range(eta.shape[0]):
        assert CL.true_residual(U, Acl, psi[k], eta[k], p) <= TRUE_RESID
    it_ref = _oracle(key + ("solve_iters",), lambda: CL.solve_full_sw(U, Acl, eta[0], p, tol=1e-10)[1])
    if precision == wf.WF_FP64:
        assert abs(iters[0] - it_ref) <= max(3, 0.15 * it_ref), (iters, it_ref)
    else:
        assert iters[0] <= 2 * it_ref + 10, (iters, it_ref)


def test_host_arrays(case):
    key, p, U, Acl, eta, w = case
    if key != (2, 8):
        pytest.skip("one case suffices")
    ref = _oracle(key + ("Qinv",), lambda: CL.Q_inverse(U, Acl, eta, p))
    out = np.empty_like(eta)
    wf.wf_apply_Qinv(w.h, np.ascontiguousarray(eta), out, 2)
    assert _rel(out, ref) < 1e-12
    x = np.zeros_like(eta)
    st, iters, res = wf.wf_solve_full_sw(w.h, np.ascontiguousarray(eta), x, 2, 1e-10, wf.WF_FP64)
    assert st == wf.WF_OK and max(res) <= 1e-10
    assert CL.true_residual(U, Acl, x[1], eta[1], p) <= TRUE_RESID


@pytest.mark.parametrize("axial", [True, False], ids=["axial", "general"])
def test_without_clover_term_q_is_the_wilson_block(axial):
    """A = 0: Q^-1 = (mu - D_t)^-1 = C_R C_L (§II.A), against the oracle and the library's C_R C_L."""
    L, T, ks, xi, bc = 4, 12, 0.07, 3.5, -1
    p = W.Params(L, T, ks, xi=xi, bc=bc)
    U = S.random_gauge(L, T, 0.3, 46)
    eta = S.gaussian_source(L, T, 146, nrhs=1)
    w = wf.Wilson(L, T, ks, kappa_t=xi * ks, bc=bc, axial=axial)
    try:
        w.load_gauge(U)
        x = _dev(eta)
        got = w.apply_Qinv(x).cpu().numpy()
        zero = np.zeros(U.shape[:4] + (4, 3, 4, 3), dtype=np.complex128)
        assert _rel(got, CL.Q_inverse(U, zero, eta, p)) < 1e-12
        assert _rel(got, w.apply_C(w.apply_C(x, 0), 1).cpu().numpy()) < 1e-12
    finally:
        w.close()


@pytest.mark.parametrize("axial", [True, False], ids=["axial", "general"])
def test_factors_follow_the_loaded_field(axial):
    """The factors are reused while the field is unchanged and formed again after every reload:
    another gauge field, other clover coefficients, no clover term, and the first field again."""
    L, T, ks, xi, bc = 4, 12, 0.07, 3.5, -1
    p = W.Params(L, T, ks, xi=xi, bc=bc)
    U1, U2 = S.random_gauge(L, T, 0.3, 50), S.random_gauge(L, T, 0.3, 51)
    eta = S.gaussian_source(L, T, 150, nrhs=1)
    zero = np.zeros(U1.shape[:4] + (4, 3, 4, 3), dtype=np.complex128)
    w = wf.Wilson(L, T, ks, kappa_t=xi * ks, bc=bc, axial=axial)
    try:
        x = _dev(eta)
        for U, cs, ct in ((U1, 1.0, 0.9), (U1, 1.0, 0.9), (U2, 1.0, 0.9), (U2, 0.6, 1.2), (U2, None, None),
                          (U1, 1.0, 0.9)):
            if cs is None:
                w.load_gauge(U)
                Acl = zero
            else:
                w.load_gauge_clover(U, cs, ct)
                Acl = CL.clover_term(U, cs, ct)
            ref = CL.Q_inverse(U, Acl, eta, p)
            for f32, tol in ((False, 1e-12), (True, 1e-5), (False, 1e-12)):
                assert _rel(w.apply_Qinv(x, f32=f32).cpu().numpy(), ref) < tol
    finally:
        w.close()


def test_errors():
    L, T, ks, xi, bc = 2, 8, 0.08, 3.0, -1
    w = wf.Wilson(L, T, ks, kappa_t=xi * ks, bc=bc)
    try:
        eta = S.gaussian_source(L, T, 47, nrhs=1)
        with pytest.raises(wf.WFError) as e:  # no gauge field
            w.apply_Qinv(_dev(eta))
        assert e.value.code == wf.WF_EINVAL
        U = S.random_gauge(L, T, 0.5, 48)
        w.load_gauge_clover(U, 1.0, 1.0)
        for prec in (wf.WF_FP16MIX, 7):
            with pytest.raises(wf.WFError) as e:
                w.solve_full_sw(_dev(eta), precision=prec)
            assert e.value.code == wf.WF_EINVAL
        with pytest.raises(wf.WFError) as e:
            w.solve_full_sw(_dev(eta), tol=0.0)
        assert e.value.code == wf.WF_EINVAL
        x = torch.zeros_like(_dev(eta))
        assert wf.lib.wf_apply_Qinv(w.h, x.data_ptr(), x.data_ptr(), 0) == wf.WF_EINVAL  # nrhs 0
        # the iteration limit: outputs written, WF_ENOCONV
        wf.wf_set_max_iterations(w.h, 3)
        x, iters, res, status = w.solve_full_sw(_dev(eta), tol=1e-10)
        assert status == wf.WF_ENOCONV and iters[0] <= 3 and res[0] > 1e-10
        assert torch.isfinite(torch.view_as_real(x)).all() and float(x.abs().max()) > 0
        wf.wf_set_max_iterations(w.h, 100000)
        bad = eta.copy()
        bad[0, 1, 0, 0, 1, 2, 0] = np.nan
        with pytest.raises(wf.WFError) as e:
            w.solve_full_sw(_dev(bad), tol=1e-10)
        assert e.value.code == wf.WF_ENAN
        x, iters, res, status = w.solve_full_sw(_dev(eta), tol=1e-10)  # the handle still works
        assert status == wf.WF_OK and res[0] <= 1e-10
    finally:
        w.close()
