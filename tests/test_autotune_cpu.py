"""Host-side logic of the autotuner: the paper's delay heuristic (Sec. 2.3:
T ~ n/10k for determinants; Sec. 3.3: n/20k for Pfaffians; T < n/k) and the
candidate set around it."""
import pytest


def at():
    try:
        from paper_2602_05255_gb300 import autotune
    except ImportError as e:
        pytest.skip(str(e))
    return autotune


def test_heuristic_delay():
    A = at()
    assert A.heuristic_delay("det", 128, 1) == 13
    assert A.heuristic_delay("pf", 128, 1) == 6
    assert A.heuristic_delay("det", 1024, 1) == 102
    assert A.heuristic_delay("det", 16, 8) == 2          # clipped at 2
    assert A.heuristic_delay("pf", 10, 1) == 2


def test_candidates_respect_slot_capacity():
    A = at()
    c = A.candidates("det", 1024, 1)
    assert c == sorted(c) and all(2 <= x <= 64 for x in c)
    c2 = A.candidates("pf", 256, 2)          # 2k = 4 columns per step: K <= 16
    assert all(4 * x <= 64 for x in c2) and 4 in c2


def test_flush_candidates_keep_fp64_class_kernels():
    torch = pytest.importorskip("torch")
    A = at()
    L = A.L
    # FP64 tiles always; split product where n % 128 == 0; double-float for F64
    assert A.flush_candidates("det", 256, 1, torch.float64) == [L.FLUSH_NATIVE, L.FLUSH_SPLIT, L.FLUSH_DF]
    assert A.flush_candidates("det", 200, 1, torch.float64) == [L.FLUSH_NATIVE, L.FLUSH_DF]
    assert A.flush_candidates("pf", 256, 1, torch.complex128) == [L.FLUSH_NATIVE]
