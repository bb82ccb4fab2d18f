"""Failure detection without a GPU fault: a bounded device wait on a flag
that no kernel sets gives up, the host reads LRU_ERR_TIMEOUT from the sticky
device error, and the same handle keeps working afterwards."""
import numpy as np
import pytest

from gpu_common import O, lrugb, tdev, torch

pytestmark = pytest.mark.gpu

ERR_TIMEOUT = 7


def test_bounded_wait_times_out_and_context_survives():
    L = lrugb()
    W, n = 2, 16
    g = np.random.Generator(np.random.PCG64(951))
    A = g.standard_normal((W, n, n)) + 3 * np.eye(n)
    st = L.LowRankState("det", W, n, k=1, dtype=torch.float64)
    st.init(tdev(A))
    st.wait_selftest(1 << 12)                   # ~0.3 ms of polling, then gives up
    with pytest.raises(L.LRUError) as e:
        st.check_device_error()
    assert e.value.code == ERR_TIMEOUT
    st.check_device_error()                     # the error was read and cleared
    # the handle and the context still compute: one update against the oracle
    Vd = g.standard_normal((W, 1, n)) * 0.1
    rows = np.array([[3], [5]], np.int32)
    r, status = st.propose_det(L.Operand(idx=tdev(rows), onehot_mask=1), L.Operand(dense=tdev(Vd)))
    st.accept()
    r = r.cpu().numpy()
    for w in range(W):
        ref = O.det_ratio_direct(A[w], O.onehot_matrix(n, rows[w]), Vd[w])
        assert abs(r[w] - ref) <= 1e-12 * abs(ref)
    st.check_device_error()


def test_selftest_rejects_out_of_range_polls():
    L = lrugb()
    st = L.LowRankState("det", 1, 8, k=1, dtype=torch.float64)
    for bad in (-1, (1 << 24) + 1):
        with pytest.raises(L.LRUError):
            st.wait_selftest(bad)
