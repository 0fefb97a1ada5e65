"""Seeded generators for gauge fields, sources and gauge transformations.

Every generator takes an explicit integer seed and uses NumPy's PCG64, so
the same call gives the same field on any machine. Random numbers are drawn
in C order of the output array: for the gauge field that is site
lexicographic with x fastest, then the direction mu = x, y, z, t, then the
eight Gaussian coefficients of H.
"""

import numpy as np


def gell_mann():
    """The eight Gell-Mann matrices lambda_a (Hermitian, traceless, tr(l_a l_b) = 2 delta_ab)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return lam


def _reunitarise(u):
    """Project a stack of 3x3 matrices to the nearest SU(3) element (polar part, det fixed to 1)."""
    w, _, vh = np.linalg.svd(u)
    q = w @ vh
    det = np.linalg.det(q)
    phase = np.exp(-1j * np.angle(det) / 3.0)
    return q * phase[..., None, None]


def _det3(u):
    return (u[..., 0, 0] * (u[..., 1, 1] * u[..., 2, 2] - u[..., 1, 2] * u[..., 2, 1])
            - u[..., 0, 1] * (u[..., 1, 0] * u[..., 2, 2] - u[..., 1, 2] * u[..., 2, 0])
            + u[..., 0, 2] * (u[..., 1, 0] * u[..., 2, 1] - u[..., 1, 1] * u[..., 2, 0]))


def random_su3(shape, eps, rng):
    """exp(i eps H) with H = sum_a h_a lambda_a / 2, h_a ~ N(0, 1), one per entry of ``shape``.

    The exponential is taken through the eigen-decomposition of H; one Newton step
    of the polar iteration, u <- u (3 - u^dag u) / 2, and a cube-root phase fix of
    the determinant then hold u in SU(3) to rounding.
    """
    h = rng.standard_normal(size=tuple(shape) + (8,))
    lam = gell_mann().reshape(8, 9)
    H = (h @ lam).reshape(tuple(shape) + (3, 3)) * 0.5
    w, v = np.linalg.eigh(H)
    u = (v * np.exp(1j * eps * w)[..., None, :]) @ np.swapaxes(v.conj(), -1, -2)
    u = 0.5 * u @ (3.0 * np.eye(3) - np.swapaxes(u.conj(), -1, -2) @ u)
    return u * np.exp(-1j * np.angle(_det3(u)) / 3.0)[..., None, None]


def random_gauge(L, T, eps, seed):
    """Random SU(3) gauge field U[t, z, y, x, mu, row, col] with U = exp(i eps H)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return random_su3((T, L, L, L, 4), eps, rng)


def unit_gauge(L, T):
    """The free field: every link is the 3x3 unit matrix."""
    U = np.zeros((T, L, L, L, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def random_gauge_transform(L, T, seed):
    """Haar-random SU(3) matrix g(x) on every site (QR of a complex Gaussian matrix)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = (rng.standard_normal((T, L, L, L, 3, 3)) + 1j * rng.standard_normal((T, L, L, L, 3, 3))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    return _reunitarise(q)


def gaussian_source(L, T, seed, nrhs=None):
    """Complex Gaussian source: Re and Im ~ N(0, 1/2) on every spin-colour component."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (T, L, L, L, 4, 3) if nrhs is None else (nrhs, T, L, L, L, 4, 3)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) * np.sqrt(0.5)


def point_sources(L, T):
    """The 12 spin-colour point sources at site 0: source k = 3*spin + colour has a 1 there."""
    eta = np.zeros((12, T, L, L, L, 4, 3), dtype=np.complex128)
    for s in range(4):
        for c in range(3):
            eta[3 * s + c, 0, 0, 0, 0, s, c] = 1.0
    return eta


def kappa_critical_free(xi):
    """Free-field critical spatial hopping parameter at kappa_t = xi * kappa_s: 1 / (2 (xi + 3))."""
    return 1.0 / (2.0 * (xi + 3.0))


def _wl(name, L, T, xi, kappa_s, kappa_t, bc, eps, seed, sources, nsrc):
    return dict(name=name, L=L, T=T, xi=xi, kappa_s=kappa_s, kappa_t=kappa_t, bc=bc,
                eps=eps, seed=seed, sources=sources, nsrc=nsrc)


# The workloads of the benchmark plan. kappa_t = xi * kappa_s unless given;
# below the free critical point kappa_s = f * kappa_critical_free(xi).
WORKLOADS = {
    "wilson_4c16_xi3": _wl("wilson_4c16_xi3", 4, 16, 3.0, 0.12, 0.36, -1, 0.3, 1, "gaussian", 1),
    "wilson_16c128_xi3.5": _wl("wilson_16c128_xi3.5", 16, 128, 3.5, 0.9 * kappa_critical_free(3.5),
                               3.5 * 0.9 * kappa_critical_free(3.5), -1, 0.25, 2, "gaussian", 1),
    "wilson_24c128_xi3.5": _wl("wilson_24c128_xi3.5", 24, 128, 3.5, 0.97 * kappa_critical_free(3.5),
                               3.5 * 0.97 * kappa_critical_free(3.5), -1, 0.2, 3, "point", 12),
    "force_8c32_xi3": _wl("force_8c32_xi3", 8, 32, 3.0, 0.075, 0.225, -1, 0.25, 4, "gaussian", 1),
    "force_16c64_xi3": _wl("force_16c64_xi3", 16, 64, 3.0, 0.075, 0.225, -1, 0.25, 4, "gaussian", 1),
}
for _i, _xi in enumerate((1.0, 3.0, 4.5, 6.0)):
    for _L, _T in ((12, 48), (16, 96), (16, 128)):
        _ks = 0.9 * kappa_critical_free(_xi)
        WORKLOADS[f"sweep_xi{_xi:g}_{_L}c{_T}"] = _wl(f"sweep_xi{_xi:g}_{_L}c{_T}", _L, _T, _xi, _ks, _xi * _ks,
                                                       -1, 0.25, 5 + _i, "gaussian", 4)


def workload(name, with_sources=True):
    """Build (params, U, eta) for a named workload; eta has a leading source axis."""
    p = WORKLOADS[name]
    U = random_gauge(p["L"], p["T"], p["eps"], p["seed"])
    eta = None
    if with_sources:
        if p["sources"] == "point":
            eta = point_sources(p["L"], p["T"])
        else:
            eta = gaussian_source(p["L"], p["T"], p["seed"] + 1000, nrhs=p["nsrc"])
    return p, U, eta
