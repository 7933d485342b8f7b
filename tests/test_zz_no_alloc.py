"""The allocation-free gather (t3f_gather_noalloc) against the workspace version.

For callers that cannot allocate device memory (a plugin living inside another framework's
memory pool or under a hard memory cap, or code that must not trigger the implicit device
synchronisation of cudaMalloc/cudaFree), the library offers t3f_gather_noalloc, whose
scratch is a fixed device array inside the library. The tests call it through the C ABI
and compare values and loss with t3f_gather given a freshly allocated workspace:
  * two calls in a row, the small one first, so that the second (larger) launch reads loss
    partials from slots the first call left behind and must overwrite every one of them;
  * an out-of-range index, which the kernel clamps and records in the array's error word;
    t3f_gather_noalloc_status reads it back, and the next clean call clears it again.
The file sits on its own and pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synth as S
from tests._util import TOL, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _call_noalloc(t3f, X, idx, y):
    lib = t3f.load()
    N = idx.shape[1]
    vals = torch.empty(N, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    st = lib.t3f_gather_noalloc(ctypes.byref(X.desc()), ctypes.c_void_p(idx.data_ptr()), N,
                                ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                ctypes.c_void_p(loss.data_ptr()), _stream())
    assert st == 0, lib.t3f_status_string(st).decode()
    return vals, loss


def _case(lib, seed, N):
    rng = np.random.default_rng(seed)
    n = [10] * 10
    X = [np.asarray(c, np.float32) for c in S.random_tt(rng, 1, n, S.tt_ranks(10, 8), 8 ** -0.5)]
    idx = torch.tensor(S.random_indices(rng, N, n), device="cuda")
    y = torch.tensor(rng.normal(size=N).astype(np.float32), device="cuda")
    return lib.TT.from_cores(X, device="cuda"), idx, y


def test_gather_noalloc_matches_workspace_version_twice(lib):
    c = lib.load()
    # small launch first (few CTAs write loss partials), then a large one (many more CTAs)
    for seed, N in ((302, 4_099), (301, 250_003)):
        Xd, idx, y = _case(lib, seed, N)
        v_ref, l_ref = lib.gather(Xd, idx, y, want_vals=True, want_loss=True)
        v_na, l_na = _call_noalloc(lib, Xd, idx, y)
        torch.cuda.synchronize()
        assert rel_err(v_na.cpu().numpy(), v_ref.cpu().numpy()) <= TOL["fp32"]
        assert abs(l_na.item() - l_ref.item()) <= TOL["fp32"] * abs(l_ref.item())
        assert c.t3f_gather_noalloc_status(_stream()) == 0


def test_gather_noalloc_reports_out_of_range_index(lib):
    c = lib.load()
    Xd, idx, y = _case(lib, 303, 1000)
    bad = idx.clone()
    bad[3, 17] = 10  # n_3 = 10: one past the end; the kernel clamps it and records the error
    _call_noalloc(lib, Xd, bad, y)
    assert c.t3f_gather_noalloc_status(_stream()) == -1  # T3F_ERR_ARG
    # a clean call clears the error word again, with the same values as the workspace version
    v_na, l_na = _call_noalloc(lib, Xd, idx, y)
    assert c.t3f_gather_noalloc_status(_stream()) == 0
    v_ref, l_ref = lib.gather(Xd, idx, y, want_vals=True, want_loss=True)
    torch.cuda.synchronize()
    assert rel_err(v_na.cpu().numpy(), v_ref.cpu().numpy()) <= TOL["fp32"]
    assert abs(l_na.item() - l_ref.item()) <= TOL["fp32"] * abs(l_ref.item())


def test_gather_noalloc_rejects_bad_descriptor(lib):
    c = lib.load()
    X = lib.TT.from_cores([np.ones((2, 1, 3, 1), np.float32)], device="cuda")  # batch 2
    st = c.t3f_gather_noalloc(ctypes.byref(X.desc()), None, 0, None, None, None, None)
    assert st == -2
