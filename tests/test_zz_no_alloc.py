"""The allocation-free norm entry point (collected last on purpose).

qs_norm_noalloc serves callers that may not allocate device memory, e.g. a host program
that has handed the whole GPU to its own buffers.  It keeps its partial sums in a fixed
device array instead of allocating; this test calls it through the C ABI twice in a row on
the same state and compares each result with qs_norm's, within the tolerance the other
read-out tests use, and checks that oversized and null arguments are rejected.
"""
import ctypes

import pytest

from workloads import circuits as wc

pytestmark = pytest.mark.gpu

qs = pytest.importorskip("paper_2010_09746_gb300")
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_norm_noalloc_matches_qs_norm(dtype, tol):
    L = qs._lib.load()
    n = 18
    st = qs.State(n, dtype)
    st.run(wc.random_mixed_circuit(n, 80, seed=3, kmax=3), mode="tile")
    ref = st.norm()
    assert abs(ref - 1.0) < tol
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    code = qs.QS_C128 if dtype == "c128" else qs.QS_C64
    for _ in range(2):
        out.fill_(-1.0)
        torch.cuda.synchronize()
        rc = L.qs_norm_noalloc(ctypes.c_void_p(st.device_ptr()), n, code, ctypes.c_void_p(out.data_ptr()), None)
        assert rc == 0, L.qs_last_error()
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= tol
        assert got == ref   # same kernels, same fixed reduction order


def test_norm_noalloc_rejects_bad_arguments():
    L = qs._lib.load()
    st = qs.State(4, "c128")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    ptr = ctypes.c_void_p(st.device_ptr())
    optr = ctypes.c_void_p(out.data_ptr())
    assert L.qs_norm_noalloc(ptr, 37, qs.QS_C128, optr, None) == 1
    assert b"2^36" in L.qs_last_error()
    assert L.qs_norm_noalloc(ptr, 0, qs.QS_C128, optr, None) == 1
    assert L.qs_norm_noalloc(None, 4, qs.QS_C128, optr, None) == 1
    assert L.qs_norm_noalloc(ptr, 4, qs.QS_C128, None, None) == 1
    assert L.qs_norm_noalloc(ptr, 4, 7, optr, None) == 1
