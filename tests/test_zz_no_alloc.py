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


# dtype code, numpy dtype, relative tolerance on log|det| against the oracle
DTYPES = {"f64": (0, np.float64, 1e-12), "c128": (1, np.complex128, 1e-12),
          "f32": (2, np.float32, 1e-4), "c64": (3, np.complex64, 1e-4)}


@pytest.mark.parametrize("dt", list(DTYPES))
def test_noalloc_matches_allocating_entry_point_twice(dt):
    from oracle import lru_oracle as O
    torch, lib = _lib()
    code_dt, npdt, rtol = DTYPES[dt]
    cplx = np.iscomplexobj(np.zeros(1, npdt))
    g = np.random.Generator(np.random.PCG64(2024))
    # two calls in a row with different sizes: the second must not see the
    # first's contents; A = 3 I + N(0, 1/n) keeps the single-precision cases
    # well conditioned
    for W, n in ((300, 96), (7, 513)):
        A = g.standard_normal((W, n, n)) + (1j * g.standard_normal((W, n, n)) if cplx else 0)
        A = (A / np.sqrt(n) + 3 * np.eye(n)).astype(npdt)
        At = torch.tensor(A, device="cuda")
        c0, l0, s0 = _call(torch, lib.lru_slogdet_batched, code_dt, At)
        c1, l1, s1 = _call(torch, lib.lru_slogdet_batched_noalloc, code_dt, At)
        assert c0 == 0 and c1 == 0
        assert np.allclose(l1, l0, rtol=rtol, atol=0)
        assert np.allclose(s1, s0, rtol=0, atol=rtol)
        for w in (0, W - 1):
            s_ref, l_ref = O.slogdet(A[w].astype(np.complex128 if cplx else np.float64))
            assert abs(l1[w] - l_ref) <= rtol * max(1.0, abs(l_ref)), (dt, n, w)
            assert abs(s1[w] - s_ref) <= 10 * rtol, (dt, n, w)


def test_noalloc_one_slot_at_the_workspace_limit():
    # n = 2048 in complex128 is 64 MiB per matrix: the whole workspace holds one
    # slot, which the two walkers share in turn
    from oracle import lru_oracle as O
    torch, lib = _lib()
    g = np.random.Generator(np.random.PCG64(2025))
    W, n = 2, 2048
    A = (g.standard_normal((W, n, n)) + 1j * g.standard_normal((W, n, n))) / np.sqrt(n) + 3 * np.eye(n)
    At = torch.tensor(A, device="cuda")
    c0, l0, s0 = _call(torch, lib.lru_slogdet_batched, 1, At)
    c1, l1, s1 = _call(torch, lib.lru_slogdet_batched_noalloc, 1, At)
    assert c0 == 0 and c1 == 0
    assert np.allclose(l1, l0, rtol=1e-12, atol=0) and np.allclose(s1, s0, rtol=0, atol=1e-12)
    s_ref, l_ref = O.slogdet(A[1])
    assert abs(l1[1] - l_ref) <= 1e-11 * abs(l_ref) and abs(s1[1] - s_ref) <= 1e-10


def test_noalloc_rejects_sizes_beyond_its_workspace():
    torch, lib = _lib()
    A = torch.zeros(1, 4, 4, dtype=torch.float64, device="cuda")
    dummy = torch.empty(1, dtype=torch.float64, device="cuda")
    code = lib.lru_slogdet_batched_noalloc(0, 1, 4096, ctypes.c_void_p(A.data_ptr()),
                                           ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                                           None)
    assert code == 1   # LRU_ERR_ARG: a 4096 x 4096 matrix does not fit the 64 MiB workspace
