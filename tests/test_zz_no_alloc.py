"""The allocation-free slogdet entry point (lru_slogdet_batched_noalloc).

It serves callers that cannot let a library allocate device memory (a runtime
that owns most of the GPU in its own pool, code that must avoid cudaFree's
device-wide synchronisation, work recorded for replay).  Its results must
equal those of lru_slogdet_batched, which allocates its workspace, within the
tolerance of the other slogdet tests, on two calls in a row (the shared
workspace keeps the previous call's contents).  This file sorts last so that a
run stopping at the first failure has run every other test first.
"""
import ctypes
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_05255_gb300 import lrugb
    lib = ctypes.CDLL(lrugb.LIB_PATH)
    for name in ("lru_slogdet_batched", "lru_slogdet_batched_noalloc"):
        f = getattr(lib, name)
        f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32] + [ctypes.c_void_p] * 4
        f.restype = ctypes.c_int
    return torch, lib


def _call(torch, f, dtype_code, A):
    W, n = A.shape[0], A.shape[-1]
    logabs = torch.empty(W, dtype=torch.float64, device="cuda")
    sign = torch.empty(W, dtype=A.dtype, device="cuda")
    code = f(dtype_code, W, n, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(logabs.data_ptr()),
             ctypes.c_void_p(sign.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return code, logabs.cpu().numpy(), sign.cpu().numpy()


@pytest.mark.parametrize("cplx", [False, True])
def test_noalloc_matches_allocating_entry_point_twice(cplx):
    torch, lib = _lib()
    g = np.random.Generator(np.random.PCG64(2024))
    dtype_code = 1 if cplx else 0
    # two calls in a row with different sizes: the second must not see the first's contents
    for W, n in ((300, 96), (7, 513)):
        A = g.standard_normal((W, n, n)) + (1j * g.standard_normal((W, n, n)) if cplx else 0)
        At = torch.tensor(A, device="cuda")
        c0, l0, s0 = _call(torch, lib.lru_slogdet_batched, dtype_code, At)
        c1, l1, s1 = _call(torch, lib.lru_slogdet_batched_noalloc, dtype_code, At)
        assert c0 == 0 and c1 == 0
        assert np.allclose(l1, l0, rtol=1e-12, atol=0)
        assert np.allclose(s1, s0, rtol=0, atol=1e-12)


def test_noalloc_rejects_sizes_beyond_its_workspace():
    torch, lib = _lib()
    A = torch.zeros(1, 4, 4, dtype=torch.float64, device="cuda")
    dummy = torch.empty(1, dtype=torch.float64, device="cuda")
    code = lib.lru_slogdet_batched_noalloc(0, 1, 4096, ctypes.c_void_p(A.data_ptr()),
                                           ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                                           None)
    assert code == 1   # LRU_ERR_ARG: a 4096 x 4096 matrix does not fit the 64 MiB workspace
