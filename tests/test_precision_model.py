"""The precision model behind the mixed-precision solve (CPU only, oracle operators).

Reliable-update CGNR on M-hat with every vector and operator result rounded to a storage
precision, the residual recomputed in FP64 whenever the iterated one fell by delta since the last
recomputation. FP32 storage with delta = 1e-5 (the library's scheme) reaches a 1e-10 residual with
two FP64 recomputations; FP16 storage with one FP32 scale per site (the option the library does
not build) needs delta ~ 1e-2 and five of them at the same iteration count. Each recomputation
costs two FP64 M-hat applies, which on GB300 (FP64 rate ~1/64 of FP32) outweighs what halving the
spinor traffic of the FP32 applies saves.
"""

import numpy as np

import synthetic as S
from oracle import wilson as W


def _store(v, kind):
    if kind == "fp32":
        return (v.real.astype(np.float32) + 1j * v.imag.astype(np.float32)).astype(np.complex128)
    re, im = v.real, v.imag  # fp16 with one FP32 scale per site (the largest of its 24 reals)
    m = np.maximum(np.abs(re).max(axis=(-1, -2), keepdims=True), np.abs(im).max(axis=(-1, -2), keepdims=True))
    m = np.where(m == 0, 1.0, m).astype(np.float32).astype(np.float64)
    q = lambda a: (a / m).astype(np.float16).astype(np.float64) * m
    return q(re) + 1j * q(im)


def _reliable_cgnr(p, U, par3, b, kind, delta, tol=1e-10, maxit=2000):
    A = lambda v: W.M_hat(U, v, p, par3)
    Ad = lambda v: W.M_hat_dag(U, v, p, par3)
    lo = lambda v: _store(v, kind)
    rhs = Ad(b)
    target = tol * np.linalg.norm(rhs)
    x = np.zeros_like(b)
    xi = np.zeros_like(b)
    r = lo(rhs)
    pv = r.copy()
    rr = np.vdot(r, r).real
    rmax = np.sqrt(rr)
    it = updates = 0
    while it < maxit:
        q = lo(Ad(lo(A(lo(pv)))))
        alpha = rr / np.vdot(pv, q).real
        xi = lo(xi + alpha * pv)
        r = lo(r - alpha * q)
        rrn = np.vdot(r, r).real
        it += 1
        if np.sqrt(rrn) < delta * rmax or np.sqrt(rrn) <= target:
            x, xi = x + xi, np.zeros_like(b)
            r64 = rhs - Ad(A(x))
            updates += 1
            t = np.linalg.norm(r64)
            if t <= target:
                break
            r, rmax = lo(r64), t
            rrn = np.vdot(r, r).real
        pv = lo(r + (rrn / rr) * pv)
        rr = rrn
    return it, updates, np.linalg.norm(rhs - Ad(A(x))) / np.linalg.norm(rhs)


def test_fp16_storage_needs_more_fp64_recomputations_than_fp32():
    L, T, xi = 4, 16, 3.5
    p = W.Params(L, T, 0.95 / (2 * (xi + 3)), xi=xi, bc=-1)
    U = S.random_gauge(L, T, 0.25, 3)
    par3 = W.parity3(L, T)
    b = W.restrict(S.gaussian_source(L, T, 4), par3 == 1)
    it32, ru32, res32 = _reliable_cgnr(p, U, par3, b, "fp32", 1e-5)
    it16, ru16, res16 = _reliable_cgnr(p, U, par3, b, "fp16", 1e-2)
    assert res32 <= 1e-10 and res16 <= 1e-10
    assert ru32 <= 2
    assert ru16 >= ru32 + 2
    assert abs(it16 - it32) <= 2
