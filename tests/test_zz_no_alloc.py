"""wf_apply_schur_noalloc: the M-hat apply that takes its work memory from a fixed device array.

It exists for callers that cannot let the library allocate device memory at apply time
(pools that have reserved the device, latency-critical loops, fixed memory budgets). This
file is collected last on purpose (pytest orders test files by name), so a run that stops at
the first failure has already run every other test when it gets here.

The new entry point must give what wf_apply_schur gives, within the FP64 tolerance of the
other parity tests (1e-12 relative), on consecutive calls that reuse the same array, and
reject what it cannot serve without allocating.
"""

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0910_0992_gb300 as wf  # noqa: E402


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def _handle(L, T, seed):
    w = wf.Wilson(L, T, 0.075, kappa_t=0.26, bc=-1)
    w.load_gauge(S.random_gauge(L, T, 0.3, seed))
    return w


def _odd(L, T, nrhs, seed):
    n = nrhs * L ** 3 * T // 2 * 12
    return torch.from_numpy(S.gaussian_source(L, T, seed, nrhs=nrhs).reshape(-1)[:n].copy()).cuda()


@pytest.mark.parametrize("dagger", [0, 1])
def test_noalloc_matches_apply_schur_on_consecutive_calls(dagger):
    # 4^3 x 16 (no padded time slots), then 4^3 x 7 (padded slots): the second lattice runs on
    # an array that still holds the first one's data
    for L, T, nrhs, seed in [(4, 16, 2, 1), (4, 16, 1, 2), (4, 7, 2, 3), (4, 7, 2, 4)]:
        w = _handle(L, T, seed)
        for call in range(2):
            x = _odd(L, T, nrhs, 100 * seed + call)
            ref = torch.empty_like(x)
            wf.wf_apply_schur(w.h, x, ref, dagger, nrhs)
            out = torch.full_like(x, complex(np.nan, np.nan))
            wf.wf_apply_schur_noalloc(w.h, x, out, dagger, nrhs)
            assert _rel(out, ref) < 1e-12, (L, T, nrhs, call)
        w.close()


def test_noalloc_rejects_what_it_cannot_serve():
    w = _handle(4, 16, 5)
    big = 64  # 64 x 1024 sites needs more than the fixed array
    x = _odd(4, 16, 1, 6).repeat(big)
    out = torch.empty_like(x)
    with pytest.raises(wf.WFError) as e:
        wf.wf_apply_schur_noalloc(w.h, x, out, 0, big)
    assert e.value.code == wf.WF_EINVAL and "maximum" in str(e.value)
    xh = _odd(4, 16, 1, 7).cpu().numpy()
    with pytest.raises(wf.WFError) as e:
        wf.wf_apply_schur_noalloc(w.h, xh, np.empty_like(xh), 0, 1)
    assert e.value.code == wf.WF_EINVAL
    # a rejected call leaves the handle usable
    x = _odd(4, 16, 1, 8)
    ref, out = torch.empty_like(x), torch.empty_like(x)
    wf.wf_apply_schur(w.h, x, ref, 0, 1)
    wf.wf_apply_schur_noalloc(w.h, x, out, 0, 1)
    assert _rel(out, ref) < 1e-12
    w.close()


@pytest.mark.parametrize("nrhs", [1, 2])
def test_noalloc_call_allocates_no_device_memory(nrhs):
    # One call on a separate handle first, so that the kernels' code and the fixed array are
    # loaded on the device (lazy module loading would otherwise show up as used memory). Then,
    # on a fresh handle, the device's free memory must be the same before and after the first
    # call: the call takes nothing from the device beyond what the handle already holds.
    L, T = 4, 16
    warm = _handle(L, T, 11)
    xw = _odd(L, T, nrhs, 12)
    wf.wf_apply_schur_noalloc(warm.h, xw, torch.empty_like(xw), 0, nrhs)
    warm.close()
    w = _handle(L, T, 13)
    x = _odd(L, T, nrhs, 14)
    out = torch.empty_like(x)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    wf.wf_apply_schur_noalloc(w.h, x, out, 0, nrhs)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    ref = torch.empty_like(x)
    wf.wf_apply_schur(w.h, x, ref, 0, nrhs)
    assert _rel(out, ref) < 1e-12
    w.close()
