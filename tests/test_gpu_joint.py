"""Ragged batches solved jointly (wf_solve_many with WF_JOINT=1, FP32 temporal + Schur, axial
frame): the CG iterations of every lattice run as one solve over the concatenated odd fields, with
K-a, K-b and K-c launched once per iteration over all lattices' sources.

Checks against the FP64 oracle: every solution meets the true residual 1e-10 (recomputed with the
oracle's M), each source takes the iterations of its separate solve to within one (the joint norms
add the same terms in another grouping), the hop kernels ran on the first handle only (one launch
over all lattices), batches of more than eight lattices, the iteration limit, host arrays, an
initial guess, and the per-lattice fallback (WF_JOINT=0, or handles with different limits).
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

# L, T, kappa_s, xi, bc, eps, seed, sources: 128-, 96-, 48-slot lines and a padded one, mixed
# anisotropies and boundary conditions
MIXED = [(4, 128, 0.074, 3.5, -1, 0.2, 11, 3), (4, 96, 0.06, 4.5, 1, 0.25, 12, 2),
         (6, 48, 0.075, 3.0, -1, 0.25, 13, 2), (4, 100, 0.07, 1.0, 1, 0.25, 14, 1)]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(autouse=True)
def _joint(monkeypatch):
    monkeypatch.setenv("WF_JOINT", "1")  # the joint path is opt-in


def _setup(lats):
    out = []
    for L, T, ks, xi, bc, eps, seed, m in lats:
        p = W.Params(L, T, ks, xi=xi, bc=bc)
        U = S.random_gauge(L, T, eps, seed)
        eta = S.gaussian_source(L, T, seed + 50, nrhs=m)
        w = wf.Wilson(L, T, ks, kappa_t=xi * ks, bc=bc)
        w.load_gauge(U)
        out.append((w, p, U, eta))
    return out


def _check(lats, xs, per, ref_iters=None):
    for i, ((w, p, U, eta), x, (st, its, res)) in enumerate(zip(lats, xs, per)):
        assert st == wf.WF_OK and max(res) <= 1e-10, (i, st, res)
        psi = x.cpu().numpy() if hasattr(x, "cpu") else x
        for k in range(eta.shape[0]):
            assert SV.true_residual(U, psi[k], eta[k], p) <= TRUE_RESID
        if ref_iters is not None:
            assert all(abs(a - b) <= 1 for a, b in zip(its, ref_iters[i])), (i, its, ref_iters[i])


def test_joint_mixed_sizes_against_separate_solves():
    lats = _setup(MIXED)
    try:
        sep = []
        for w, p, U, eta in lats:
            _, it, _, st = w.solve(_dev(eta), tol=1e-10, precision=wf.WF_FP32)
            assert st == wf.WF_OK
            sep.append(it)
        rhs = [_dev(q[3]) for q in lats]
        xs = [torch.empty_like(r) for r in rhs]
        for q in lats:
            wf.wf_profile(q[0].h, 1)
        st, per = wf.wf_solve_many([q[0].h for q in lats], rhs, xs, [q[3].shape[0] for q in lats], 1e-10,
                                   wf.WF_TEMPORAL_SCHUR, wf.WF_FP32)
        assert st == wf.WF_OK
        _check(lats, xs, per, sep)
        # the FP32 hop kernels ran as joint launches on the first handle, never on the others
        prof = [wf.wf_profile_get(q[0].h) for q in lats]
        for q in lats:
            wf.wf_profile(q[0].h, 0)
        nb, _ = prof[0]["schur_b_hop_tsolve_f32"]
        nc, _ = prof[0]["schur_c_hop_tinv_axpy_f32"]
        na, _ = prof[0]["schur_a_tdag_f32"]
        assert nb == nc == na > 0
        assert nb >= 2 * max(max(it) for it in sep)  # two applies per iteration, one launch each
        for pr in prof[1:]:
            assert pr.get("schur_b_hop_tsolve_f32", (0, 0))[0] == 0
            assert pr.get("prep_hop_f32", (0, 0))[0] > 0  # S_L and the true residual stay per lattice
            assert pr.get("apply_M_f64", (0, 0))[0] > 0
    finally:
        for q in lats:
            q[0].close()


def test_joint_more_lattices_than_one_launch_holds():
    """Ten lattices: the joint kernels split into launches of at most eight lattices."""
    lats = _setup([(4, 8 + 4 * (i % 5), 0.07 + 0.001 * i, 2.0 + 0.5 * (i % 3), -1 if i % 2 else 1, 0.25,
                    30 + i, 1 + i % 2) for i in range(10)])
    try:
        rhs = [_dev(q[3]) for q in lats]
        xs = [torch.empty_like(r) for r in rhs]
        for q in lats[:2]:
            wf.wf_profile(q[0].h, 1)
        st, per = wf.wf_solve_many([q[0].h for q in lats], rhs, xs, [q[3].shape[0] for q in lats], 1e-10,
                                   wf.WF_TEMPORAL_SCHUR, wf.WF_FP32)
        prof = [wf.wf_profile_get(q[0].h) for q in lats[:2]]
        for q in lats[:2]:
            wf.wf_profile(q[0].h, 0)
        assert st == wf.WF_OK
        _check(lats, xs, per)
        nb, _ = prof[0]["schur_b_hop_tsolve_f32"]
        assert nb > 0  # applies (each two launches here: 8 + 2 lattices)
        assert prof[1].get("schur_b_hop_tsolve_f32", (0, 0))[0] == 0
    finally:
        for q in lats:
            q[0].close()


def test_joint_host_arrays_and_initial_guess():
    lats = _setup(MIXED[:3])
    try:
        hs = [q[0].h for q in lats]
        rhs = [np.ascontiguousarray(q[3]) for q in lats]
        xs = [np.empty_like(r) for r in rhs]
        st, per = wf.wf_solve_many(hs, rhs, xs, [r.shape[0] for r in rhs], 1e-10, wf.WF_TEMPORAL_SCHUR, wf.WF_FP32)
        assert st == wf.WF_OK
        _check(lats, xs, per)
        # an initial guess (the odd part of the solutions) costs no more iterations than none
        st, per2 = wf.wf_solve_many(hs, rhs, xs, [r.shape[0] for r in rhs], 1e-10, wf.WF_TEMPORAL_SCHUR,
                                    wf.WF_FP32, wf.WF_X0)
        assert st == wf.WF_OK
        _check(lats, xs, per2)
        for (_, its, _), (_, its0, _) in zip(per2, per):
            assert all(a <= b + 1 for a, b in zip(its, its0)), (its, its0)
    finally:
        for q in lats:
            q[0].close()


def test_joint_iteration_limit():
    lats = _setup(MIXED[:3])
    try:
        for q in lats:
            wf.wf_set_max_iterations(q[0].h, 3)
        rhs = [_dev(q[3]) for q in lats]
        xs = [torch.empty_like(r) for r in rhs]
        st, per = wf.wf_solve_many([q[0].h for q in lats], rhs, xs, [q[3].shape[0] for q in lats], 1e-10,
                                   wf.WF_TEMPORAL_SCHUR, wf.WF_FP32)
        assert st == wf.WF_ENOCONV
        for (w, p, U, eta), x, (sti, its, res) in zip(lats, xs, per):
            assert sti == wf.WF_ENOCONV
            assert all(0 < i <= 3 * 6 for i in its)
            psi = x.cpu().numpy()
            assert np.isfinite(psi).all()
            for k in range(eta.shape[0]):
                tr = SV.true_residual(U, psi[k], eta[k], p)
                assert 1e-10 < tr < 1.0
                assert tr == pytest.approx(res[k], rel=1e-6)
    finally:
        for q in lats:
            q[0].close()


@pytest.mark.parametrize("how", ["env", "limits"])
def test_per_lattice_fallback(how, monkeypatch):
    """Without WF_JOINT=1 (the default), or with handles of different iteration limits, one solve
    per lattice (each on its own stream and host thread); the results meet the same bar."""
    lats = _setup(MIXED[1:4])
    try:
        if how == "env":
            monkeypatch.delenv("WF_JOINT")
        else:
            wf.wf_set_max_iterations(lats[0][0].h, 5000)
        rhs = [_dev(q[3]) for q in lats]
        xs = [torch.empty_like(r) for r in rhs]
        for q in lats:
            wf.wf_profile(q[0].h, 1)
        st, per = wf.wf_solve_many([q[0].h for q in lats], rhs, xs, [q[3].shape[0] for q in lats], 1e-10,
                                   wf.WF_TEMPORAL_SCHUR, wf.WF_FP32)
        prof = [wf.wf_profile_get(q[0].h) for q in lats]
        for q in lats:
            wf.wf_profile(q[0].h, 0)
        assert st == wf.WF_OK
        _check(lats, xs, per)
        for pr in prof:  # every handle ran its own hop kernels
            assert pr["schur_b_hop_tsolve_f32"][0] > 0
    finally:
        for q in lats:
            q[0].close()


def test_solve_rejects_too_many_sources():
    L, T = 2, 4
    w = wf.Wilson(L, T, 0.075, kappa_t=0.26, bc=-1)
    try:
        w.load_gauge(S.random_gauge(L, T, 0.2, 95))
        m = wf.WF_MAX_SOLVE_RHS + 1
        eta = torch.zeros((m, L * L * L * T * 12), dtype=torch.complex128).cuda()
        x = torch.empty_like(eta)
        with pytest.raises(wf.WFError) as e:
            wf.wf_solve(w.h, eta, x, m, 1e-10, wf.WF_TEMPORAL_SCHUR, wf.WF_FP32, 0)
        assert e.value.code == wf.WF_EINVAL
    finally:
        w.close()


@pytest.mark.parametrize("precision", [wf.WF_FP32, wf.WF_FP64])
def test_solve_at_the_source_limit(precision):
    """WF_MAX_SOLVE_RHS sources in one solve (a 2^3 x 4 lattice): every source converges, sampled
    sources meet the oracle's true residual, and the CG bookkeeping of the last source is right."""
    L, T = 2, 4
    p = W.Params(L, T, 0.075, xi=3.0, bc=-1)
    U = S.random_gauge(L, T, 0.3, 97)
    m = wf.WF_MAX_SOLVE_RHS
    eta = S.gaussian_source(L, T, 98, nrhs=m)
    eta[m - 1] *= 1e-3  # the last source at another scale
    w = wf.Wilson(L, T, 0.075, kappa_t=0.225, bc=-1)
    try:
        w.load_gauge(U)
        x, iters, res, status = w.solve(_dev(eta), tol=1e-10, precision=precision)
        assert status == wf.WF_OK and len(iters) == m and max(res) <= 1e-10 and min(iters) > 0
        psi = x.cpu().numpy()
        for k in (0, 1, m // 2, m - 2, m - 1):
            assert SV.true_residual(U, psi[k], eta[k], p) <= TRUE_RESID
    finally:
        w.close()
