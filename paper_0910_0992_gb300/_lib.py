"""ctypes binding of libwf.so: one Python function per C entry point (include/wf.h)."""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "libwf.so")

WF_OK, WF_EINVAL, WF_ENOMEM, WF_ECUDA, WF_ESINGULAR, WF_ENOCONV, WF_ENAN, WF_ETIMEOUT = range(8)
WF_UNPREC, WF_EO4D, WF_TEMPORAL, WF_TEMPORAL_SCHUR, WF_TEMPORAL_ILU = range(5)
WF_FP64, WF_FP32, WF_FP16MIX = 0, 1, 2
WF_X0 = 1
WF_MAX_SOLVE_RHS = 1024  # right-hand sides of one solve (all lattices of a joint wf_solve_many)

_STATUS = {0: "WF_OK", 1: "WF_EINVAL", 2: "WF_ENOMEM", 3: "WF_ECUDA", 4: "WF_ESINGULAR",
           5: "WF_ENOCONV", 6: "WF_ENAN", 7: "WF_ETIMEOUT"}

if not os.path.exists(lib_path):
    raise ImportError(f"libwf.so is not built ({lib_path}); run paper_0910_0992_gb300.build_lib.build()")
lib = ctypes.CDLL(lib_path)

_vp, _ip, _dp, _i, _d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double

_SIGS = {
    "wf_create": (_i, [_i, _i, _d, _d, _d, _i, ctypes.POINTER(_vp)]),
    "wf_destroy": (_i, [_vp]),
    "wf_set_stream": (_i, [_vp, _vp]),
    "wf_last_error": (ctypes.c_char_p, [_vp]),
    "wf_set_gauge_frame": (_i, [_vp, _i]),
    "wf_field_elems": (ctypes.c_longlong, [_vp]),
    "wf_half_elems": (ctypes.c_longlong, [_vp]),
    "wf_load_gauge": (_i, [_vp, _vp]),
    "wf_apply_M": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_apply_M_f32": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_apply_Tinv": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_apply_Tinv_f32": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_apply_C": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_apply_schur": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_apply_schur_f32": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_apply_schur_f16": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_apply_schur_noalloc": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_apply_eo4d": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_apply_eo4d_f32": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_solve": (_i, [_vp, _vp, _vp, _i, _d, _i, _i, _i, _ip, _dp]),
    "wf_force": (_i, [_vp, _vp, _vp, _i, _d, _dp, _ip]),
    "wf_temporal_logdet": (_i, [_vp, _dp, _vp]),
    "wf_load_gauge_clover": (_i, [_vp, _vp, _d, _d]),
    "wf_apply_clover": (_i, [_vp, _vp, _vp, _i]),
    "wf_apply_ilu": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_apply_ilu_f32": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_apply_Qinv": (_i, [_vp, _vp, _vp, _i]),
    "wf_apply_Qinv_f32": (_i, [_vp, _vp, _vp, _i]),
    "wf_apply_schur_full_sw": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_apply_schur_full_sw_f32": (_i, [_vp, _vp, _vp, _i, _i]),
    "wf_solve_full_sw": (_i, [_vp, _vp, _vp, _i, _d, _i, _ip, _dp]),
    "wf_solve_many": (_i, [_i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _ip, _d, _i, _i, _i,
                           ctypes.POINTER(_ip), ctypes.POINTER(_dp), _ip]),
    "wf_launch_count": (ctypes.c_longlong, [_vp]),
    "wf_check_tables": (_i, [_i, _i, _i, _i, _i]),
    "wf_hop_config": (_i, [_vp, _i, _ip, _ip, ctypes.POINTER(ctypes.c_float)]),
    "wf_hop_pipe_config": (_i, [_vp, _i, _ip, _ip]),
    "wf_set_max_iterations": (_i, [_vp, _i]),
    "wf_profile": (_i, [_vp, _i]),
    "wf_profile_get": (_i, [_vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_longlong), _dp, _i]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def exported_symbols():
    """Names of the C entry points this binding declares (all must resolve in libwf.so)."""
    return sorted(_SIGS)


class WFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


def _check(h, code):
    if code != WF_OK:
        raise WFError(code, (lib.wf_last_error(h) or b"").decode())
    return code


def _ptr(a):
    """Address of a complex128 C-contiguous torch tensor / NumPy array (or a raw int address)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):  # torch.Tensor
        import torch
        if a.dtype != torch.complex128 or not a.is_contiguous():
            raise TypeError("expected a contiguous complex128 tensor")
        return a.data_ptr()
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.complex128 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous complex128 array")
    return a.ctypes.data


# ---------------------------------------------------------------- raw entry points
def wf_create(L, T, xi, kappa_s, kappa_t, bc):
    h = _vp()
    code = lib.wf_create(int(L), int(T), float(xi), float(kappa_s), float(kappa_t), int(bc), ctypes.byref(h))
    if code != WF_OK:
        raise WFError(code, "wf_create rejected its arguments or could not allocate")
    return h


def wf_destroy(h):
    return lib.wf_destroy(h)


def wf_set_stream(h, stream):
    return _check(h, lib.wf_set_stream(h, stream))


def wf_last_error(h):
    return (lib.wf_last_error(h) or b"").decode()


def wf_set_gauge_frame(h, axial):
    return _check(h, lib.wf_set_gauge_frame(h, int(axial)))


def wf_field_elems(h):
    return lib.wf_field_elems(h)


def wf_half_elems(h):
    return lib.wf_half_elems(h)


def wf_load_gauge(h, U):
    return _check(h, lib.wf_load_gauge(h, _ptr(U)))


def wf_load_gauge_clover(h, U, c_s, c_t):
    return _check(h, lib.wf_load_gauge_clover(h, _ptr(U), float(c_s), float(c_t)))


def wf_apply_clover(h, inp, out, nrhs=1):
    return _check(h, lib.wf_apply_clover(h, _ptr(inp), _ptr(out), int(nrhs)))


def _apply(fn):
    def call(h, inp, out, flag, nrhs=1):
        return _check(h, fn(h, _ptr(inp), _ptr(out), int(flag), int(nrhs)))
    return call


wf_apply_M = _apply(lib.wf_apply_M)
wf_apply_ilu = _apply(lib.wf_apply_ilu)
wf_apply_ilu_f32 = _apply(lib.wf_apply_ilu_f32)
wf_apply_M_f32 = _apply(lib.wf_apply_M_f32)
wf_apply_Tinv = _apply(lib.wf_apply_Tinv)
wf_apply_Tinv_f32 = _apply(lib.wf_apply_Tinv_f32)
wf_apply_C = _apply(lib.wf_apply_C)
wf_apply_schur = _apply(lib.wf_apply_schur)
wf_apply_schur_f32 = _apply(lib.wf_apply_schur_f32)
wf_apply_schur_f16 = _apply(lib.wf_apply_schur_f16)
wf_apply_schur_noalloc = _apply(lib.wf_apply_schur_noalloc)
wf_apply_eo4d = _apply(lib.wf_apply_eo4d)
wf_apply_eo4d_f32 = _apply(lib.wf_apply_eo4d_f32)
wf_apply_schur_full_sw = _apply(lib.wf_apply_schur_full_sw)
wf_apply_schur_full_sw_f32 = _apply(lib.wf_apply_schur_full_sw_f32)


def wf_apply_Qinv(h, inp, out, nrhs=1):
    return _check(h, lib.wf_apply_Qinv(h, _ptr(inp), _ptr(out), int(nrhs)))


def wf_apply_Qinv_f32(h, inp, out, nrhs=1):
    return _check(h, lib.wf_apply_Qinv_f32(h, _ptr(inp), _ptr(out), int(nrhs)))


def wf_solve_full_sw(h, rhs, x, nrhs, tol, precision=WF_FP64):
    """Returns (status, iterations[nrhs], true_residual[nrhs]); raises on errors other than WF_ENOCONV."""
    iters = (ctypes.c_int * nrhs)()
    res = (ctypes.c_double * nrhs)()
    code = lib.wf_solve_full_sw(h, _ptr(rhs), _ptr(x), int(nrhs), float(tol), int(precision), iters, res)
    if code not in (WF_OK, WF_ENOCONV):
        _check(h, code)
    return code, list(iters), list(res)


def wf_solve(h, rhs, x, nrhs, tol, method, precision, flags=0):
    """Returns (status, iterations[nrhs], true_residual[nrhs]); raises on errors other than WF_ENOCONV."""
    iters = (ctypes.c_int * nrhs)()
    res = (ctypes.c_double * nrhs)()
    code = lib.wf_solve(h, _ptr(rhs), _ptr(x), int(nrhs), float(tol), int(method), int(precision), int(flags),
                        iters, res)
    if code not in (WF_OK, WF_ENOCONV):
        _check(h, code)
    return code, list(iters), list(res)


def wf_solve_many(hs, rhs, x, nrhs, tol, method, precision, flags=0):
    """Independent solves on several handles (lattices) at once; returns (status, per-handle
    (status, iterations, true residuals))."""
    n = len(hs)
    if not (len(rhs) == len(x) == len(nrhs) == n):
        raise ValueError("hs, rhs, x and nrhs must have the same length")
    Hs = (_vp * n)(*[ctypes.c_void_p(h.value if isinstance(h, ctypes.c_void_p) else h) for h in hs])
    R = (_vp * n)(*[_ptr(a) for a in rhs])
    X = (_vp * n)(*[_ptr(a) for a in x])
    N = (ctypes.c_int * n)(*[int(k) for k in nrhs])
    its = [(ctypes.c_int * int(k))() for k in nrhs]
    res = [(ctypes.c_double * int(k))() for k in nrhs]
    I = (_ip * n)(*[ctypes.cast(a, _ip) for a in its])
    D = (_dp * n)(*[ctypes.cast(a, _dp) for a in res])
    S = (ctypes.c_int * n)()
    st = lib.wf_solve_many(n, Hs, R, X, N, float(tol), int(method), int(precision), int(flags), I, D, S)
    return st, [(S[i], list(its[i]), list(res[i])) for i in range(n)]


def wf_force(h, phi_odd, F, precision=WF_FP64, tol=1e-12):
    """Fills F (shape (..., 4, 8) float64) with dS/dU (F None: action only); returns (S, CG iterations)."""
    import numpy as np
    if F is None:
        fp = None
    elif hasattr(F, "data_ptr"):
        import torch
        if F.dtype != torch.float64 or not F.is_contiguous():
            raise TypeError("F must be a contiguous float64 tensor")
        fp = F.data_ptr()
    else:
        if not isinstance(F, np.ndarray) or F.dtype != np.float64 or not F.flags["C_CONTIGUOUS"]:
            raise TypeError("F must be a C-contiguous float64 array")
        fp = F.ctypes.data
    S = ctypes.c_double()
    it = ctypes.c_int()
    _check(h, lib.wf_force(h, _ptr(phi_odd), fp, int(precision), float(tol), ctypes.byref(S), ctypes.byref(it)))
    return S.value, it.value


def wf_temporal_logdet(h, F=None):
    """log det(mu - D_t) of the loaded gauge field; fills F (shape (..., 4, 8) float64) with its force if given."""
    import numpy as np
    if F is None:
        fp = None
    elif hasattr(F, "data_ptr"):
        import torch
        if F.dtype != torch.float64 or not F.is_contiguous():
            raise TypeError("F must be a contiguous float64 tensor")
        fp = F.data_ptr()
    else:
        if not isinstance(F, np.ndarray) or F.dtype != np.float64 or not F.flags["C_CONTIGUOUS"]:
            raise TypeError("F must be a C-contiguous float64 array")
        fp = F.ctypes.data
    v = ctypes.c_double()
    _check(h, lib.wf_temporal_logdet(h, ctypes.byref(v), fp))
    return v.value


def wf_launch_count(h):
    return lib.wf_launch_count(h)


def wf_check_tables(L, T, nrhs, tile_rows=0, plant=0):
    """Host-only check of the kernels' index tables for a geometry; returns the status code."""
    return lib.wf_check_tables(int(L), int(T), int(nrhs), int(tile_rows), int(plant))


def wf_hop_config(h, nrhs):
    """The autotuned FP32 hop-kernel configuration for nrhs: (variant, tile_rows, ms), or None."""
    v, r, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    if lib.wf_hop_config(h, int(nrhs), ctypes.byref(v), ctypes.byref(r), ctypes.byref(ms)) != WF_OK:
        return None
    return v.value, r.value, ms.value


def wf_set_max_iterations(h, maxiter):
    return _check(h, lib.wf_set_max_iterations(h, int(maxiter)))


def wf_hop_pipe_config(h, nrhs):
    """Sources per unit and stages of the bulk-fed hop kernels for nrhs ((0, 0) for the others), or None."""
    g, n = ctypes.c_int(), ctypes.c_int()
    if lib.wf_hop_pipe_config(h, int(nrhs), ctypes.byref(g), ctypes.byref(n)) != WF_OK:
        return None
    return g.value, n.value


def wf_profile(h, on):
    return _check(h, lib.wf_profile(h, int(on)))


def wf_profile_get(h, cap=64):
    """{kernel name: (launches, total milliseconds)} recorded since wf_profile(h, 1)."""
    names = (ctypes.c_char_p * cap)()
    cnt = (ctypes.c_longlong * cap)()
    ms = (ctypes.c_double * cap)()
    n = lib.wf_profile_get(h, names, cnt, ms, cap)
    if n < 0:
        raise WFError(-n, wf_last_error(h))
    return {names[i].decode(): (cnt[i], ms[i]) for i in range(min(n, cap))}


# ---------------------------------------------------------------- convenience wrapper
class Wilson:
    """A handle with its parameters; methods allocate outputs like their inputs (torch or NumPy)."""

    def __init__(self, L, T, kappa_s, kappa_t=0.0, xi=0.0, bc=-1, axial=True):
        self.L, self.T, self.bc = int(L), int(T), int(bc)
        self.h = wf_create(L, T, xi, kappa_s, kappa_t, bc)
        wf_set_gauge_frame(self.h, 1 if axial else 0)

    def close(self):
        if self.h is not None:
            wf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _like(a):
        if hasattr(a, "data_ptr"):
            import torch
            return torch.empty_like(a)
        import numpy as np
        return np.empty_like(a)

    def set_stream(self, stream):
        wf_set_stream(self.h, stream)

    def load_gauge(self, U):
        wf_load_gauge(self.h, U)

    def load_gauge_clover(self, U, c_s, c_t):
        wf_load_gauge_clover(self.h, U, c_s, c_t)

    def apply_clover(self, x):
        out = self._like(x)
        wf_apply_clover(self.h, x, out, self._nrhs(x, wf_field_elems(self.h)))
        return out

    def apply_ilu(self, x, dagger=False, f32=False):
        out = self._like(x)
        (wf_apply_ilu_f32 if f32 else wf_apply_ilu)(self.h, x, out, dagger, self._nrhs(x, wf_field_elems(self.h)))
        return out

    def _nrhs(self, a, per):
        n = 1
        for s in a.shape:
            n *= int(s)
        if n % per:
            raise ValueError("array size is not a multiple of one field")
        return n // per

    def apply_M(self, x, dagger=False, f32=False):
        out = self._like(x)
        (wf_apply_M_f32 if f32 else wf_apply_M)(self.h, x, out, dagger, self._nrhs(x, wf_field_elems(self.h)))
        return out

    def apply_Tinv(self, x, dagger=False, f32=False):
        out = self._like(x)
        (wf_apply_Tinv_f32 if f32 else wf_apply_Tinv)(self.h, x, out, dagger, self._nrhs(x, wf_field_elems(self.h)))
        return out

    def apply_C(self, x, which):
        out = self._like(x)
        wf_apply_C(self.h, x, out, which, self._nrhs(x, wf_field_elems(self.h)))
        return out

    def apply_schur(self, x_odd, dagger=False, f32=False):
        out = self._like(x_odd)
        (wf_apply_schur_f32 if f32 else wf_apply_schur)(self.h, x_odd, out, dagger,
                                                         self._nrhs(x_odd, wf_half_elems(self.h)))
        return out

    def apply_eo4d(self, x_odd4, dagger=False, f32=False):
        out = self._like(x_odd4)
        (wf_apply_eo4d_f32 if f32 else wf_apply_eo4d)(self.h, x_odd4, out, dagger,
                                                       self._nrhs(x_odd4, wf_half_elems(self.h)))
        return out

    def apply_Qinv(self, x, f32=False):
        """(A + mu - D_t)^-1 on full fields (clover term of load_gauge_clover; A = 0 without one)."""
        out = self._like(x)
        (wf_apply_Qinv_f32 if f32 else wf_apply_Qinv)(self.h, x, out, self._nrhs(x, wf_field_elems(self.h)))
        return out

    def apply_schur_full_sw(self, x_odd, dagger=False, f32=False):
        out = self._like(x_odd)
        (wf_apply_schur_full_sw_f32 if f32 else wf_apply_schur_full_sw)(self.h, x_odd, out, dagger,
                                                                         self._nrhs(x_odd, wf_half_elems(self.h)))
        return out

    def solve_full_sw(self, rhs, tol=1e-10, precision=WF_FP64):
        x = self._like(rhs)
        status, iters, res = wf_solve_full_sw(self.h, rhs, x, self._nrhs(rhs, wf_field_elems(self.h)), tol, precision)
        return x, iters, res, status

    def temporal_logdet(self, F=None):
        """log det(mu - D_t) of the loaded gauge field (F, if given, receives its force)."""
        return wf_temporal_logdet(self.h, F)

    def solve(self, rhs, tol=1e-10, method=WF_TEMPORAL_SCHUR, precision=WF_FP64, x0=None):
        x = self._like(rhs) if x0 is None else x0
        flags = WF_X0 if x0 is not None else 0
        nrhs = self._nrhs(rhs, wf_field_elems(self.h))
        status, iters, res = wf_solve(self.h, rhs, x, nrhs, tol, method, precision, flags)
        return x, iters, res, status
