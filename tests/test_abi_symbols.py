"""The C-ABI library loads without a GPU and exports every entry point include/wf.h declares."""

import ctypes
import os
import re


def _declared(root):
    names = set()
    for fn in os.listdir(os.path.join(root, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(root, "include", fn)) as fh:
                text = fh.read()
            names |= set(re.findall(r"^\s*(?:int|long long|const char\s*\*)\s*\*?\s*(wf_\w+)\s*\(", text, re.M))
    return names


def test_library_exports_every_declared_symbol(root_dir):
    import paper_0910_0992_gb300 as wf

    declared = _declared(root_dir)
    assert len(declared) >= 18
    lib = ctypes.CDLL(wf.lib_path)
    for name in sorted(declared):
        assert hasattr(lib, name), name
    # the Python binding declares exactly the same entry points
    assert set(wf.exported_symbols()) == declared


def test_create_rejects_bad_geometry_without_gpu():
    """Argument validation happens before any device work."""
    import paper_0910_0992_gb300 as wf

    h = ctypes.c_void_p()
    for L, T, ks, bc in [(3, 8, 0.1, -1), (4, 1, 0.1, -1), (4, 300, 0.1, -1), (4, 8, -0.1, -1), (4, 8, 0.1, 0)]:
        assert wf.lib.wf_create(L, T, 3.0, ks, 0.0, bc, ctypes.byref(h)) == wf.WF_EINVAL


def test_full_sw_entry_points_reject_a_null_handle_without_gpu():
    """The full SW entry points check their handle before any device work."""
    import paper_0910_0992_gb300 as wf

    it = ctypes.c_int()
    res = ctypes.c_double()
    assert wf.lib.wf_apply_Qinv(None, None, None, 1) == wf.WF_EINVAL
    assert wf.lib.wf_apply_Qinv_f32(None, None, None, 1) == wf.WF_EINVAL
    assert wf.lib.wf_apply_schur_full_sw(None, None, None, 0, 1) == wf.WF_EINVAL
    assert wf.lib.wf_apply_schur_full_sw_f32(None, None, None, 1, 1) == wf.WF_EINVAL
    assert wf.lib.wf_solve_full_sw(None, None, None, 1, 1e-10, wf.WF_FP32, ctypes.byref(it),
                                   ctypes.byref(res)) == wf.WF_EINVAL
