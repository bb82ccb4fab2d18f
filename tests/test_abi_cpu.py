"""The C-ABI library loads and exports every symbol include/lrugb.h declares.

No GPU needed: only host-side entry points are called (status strings,
version, argument validation that fails before any CUDA call).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lrugb.h")
LIB = os.path.join(ROOT, "paper_2602_05255_gb300", "liblrugb.so")


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:lru_status|const char\*)\s+(lru_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = declared()
    for must in ["lru_create", "lru_init_det", "lru_init_pf", "lru_propose_det", "lru_propose_pf",
                 "lru_accept", "lru_flush_delayed", "lru_refresh_from_scratch", "lru_get_inverse",
                 "lru_get_logvalue", "lru_save_state", "lru_load_state"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_covers_header():
    import importlib.util
    spec = importlib.util.spec_from_file_location("lrugb_sig", os.path.join(ROOT, "paper_2602_05255_gb300", "lrugb.py"))
    src = open(spec.origin).read()
    for name in declared():
        assert name in src, name


def test_host_only_entry_points(lib):
    lib.lru_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.lru_version()
    lib.lru_status_string.restype = ctypes.c_char_p
    assert lib.lru_status_string(0) == b"ok"
    assert b"argument" in lib.lru_status_string(1)


class Cfg(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dtype", ctypes.c_int32), ("walkers", ctypes.c_int64),
                ("n", ctypes.c_int32), ("n_per_walker", ctypes.c_void_p), ("k", ctypes.c_int32),
                ("k_per_walker", ctypes.c_void_p), ("delay", ctypes.c_int32), ("flush", ctypes.c_int32),
                ("device", ctypes.c_int32), ("arith", ctypes.c_int32), ("tile_chunks", ctypes.c_int32),
                ("refresh", ctypes.c_int32)]


@pytest.mark.parametrize("field,value,code", [
    ("kind", 7, 1), ("dtype", 9, 1), ("walkers", 0, 1), ("k", 0, 1), ("k", 17, 1),
    ("delay", -1, 1), ("flush", 11, 1), ("delay", 65, 1), ("arith", 3, 1), ("tile_chunks", -1, 1),
    ("refresh", 3, 1), ("refresh", -1, 1), ("refresh", 2, 8),
])
def test_create_rejects_bad_config_before_cuda(lib, field, value, code):
    cfg = Cfg(kind=0, dtype=0, walkers=4, n=16, n_per_walker=None, k=1, k_per_walker=None, delay=0,
              flush=0, device=0)
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    assert lib.lru_create(ctypes.byref(cfg), ctypes.byref(h)) == code
    assert not h.value


def test_tensor_flush_needs_delayed_f64(lib):
    cfg = Cfg(kind=0, dtype=1, walkers=4, n=16, n_per_walker=None, k=1, k_per_walker=None, delay=4,
              flush=1, device=0)
    h = ctypes.c_void_p()
    assert lib.lru_create(ctypes.byref(cfg), ctypes.byref(h)) == 8     # UNSUPPORTED, complex
    cfg.dtype, cfg.delay = 0, 0
    assert lib.lru_create(ctypes.byref(cfg), ctypes.byref(h)) == 8     # UNSUPPORTED, plain


def test_split_flush_and_tensor_refresh_shapes(lib):
    # the exact split-product flush: delayed F64 handles, uniform n % 128 == 0,
    # n <= 2048, K * k <= 64 (Pfaffian K * 2k); the tensor-core refresh: F64
    # determinants, same n rule
    base = dict(kind=0, dtype=0, walkers=4, n=256, n_per_walker=None, k=1, k_per_walker=None, delay=8,
                flush=6, device=0)
    h = ctypes.c_void_p()
    for field, value in [("n", 200), ("n", 4096), ("dtype", 1), ("delay", 0), ("delay", 65)]:
        cfg = Cfg(**base)
        setattr(cfg, field, value)
        code = lib.lru_create(ctypes.byref(cfg), ctypes.byref(h))
        assert code in (1, 8) and not h.value, (field, value, code)   # invalid, or not supported
    cfg = Cfg(**{**base, "kind": 1, "delay": 33})                      # Pfaffian: 33 x 2 slot columns > 64
    assert lib.lru_create(ctypes.byref(cfg), ctypes.byref(h)) == 1 and not h.value
    for field, value in [("n", 200), ("dtype", 1), ("kind", 1)]:
        cfg = Cfg(**{**base, "flush": 0, "delay": 0})
        cfg.refresh = 2
        setattr(cfg, field, value)
        assert lib.lru_create(ctypes.byref(cfg), ctypes.byref(h)) == 8 and not h.value, (field, value)


def test_null_arguments(lib):
    assert lib.lru_create(None, None) == 1
    assert lib.lru_destroy(None) == 1
    assert lib.lru_accept(None, None) == 1


@pytest.mark.parametrize("name", ["lru_slogdet_batched", "lru_slogpf_batched", "lru_slogdet_batched_noalloc"])
def test_batched_entry_points_reject_walker_counts_beyond_int32(lib, name):
    # the kernels index walkers with 32-bit ints: 2^31 walkers is an argument
    # error, found before any CUDA call (no pointer is dereferenced)
    f = getattr(lib, name)
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32] + [ctypes.c_void_p] * 4
    f.restype = ctypes.c_int
    for W in (2 ** 31, 2 ** 40, 0, -1):
        assert f(0, W, 4, 16, 16, 16, None) == 1, W
