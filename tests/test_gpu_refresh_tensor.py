"""GPU parity of the tensor-core refresh (FP64 Gauss-Jordan panels, trailing
updates as an exact BF16 split product on tcgen05) against the oracle's
inverse and slogdet, and against the all-FP64 Gauss-Jordan refresh.

Bound: the FP64 bar of the refresh, Frobenius relative 1e-10 on A^{-1} and
1e-12 on log|det| (the split product keeps the rounding of an FP64 update:
the FP64 Gauss-Jordan and the tensor form differ by O(cond * 2^-53)).
"""
import numpy as np
import pytest

from gpu_common import CEIL_CHAIN, O, check_ratios, det_workload, fro_rel, lrugb, tdev, torch

pytestmark = pytest.mark.gpu


def slater_batch(seed, W, n, var=None):
    g = np.random.Generator(np.random.PCG64(seed))
    Phi = g.standard_normal((2 * n, n)) * np.sqrt(var if var is not None else 1.0 / n)
    occ = np.stack([g.permutation(2 * n)[:n] for _ in range(W)])
    return np.stack([Phi[o] for o in occ])


@pytest.mark.parametrize("n", [128, 256, 384, 1152, 2048])
def test_tensor_refresh_matches_oracle_and_fp64(n):
    """n <= 1024: 16-column FP64 sub-panels; above: 8-column sub-panels with
    four rows per thread (1152: an odd number, nine, of 128-column tiles;
    2048 is the largest n).  At n = 2048 the oracle's pure-numpy LU takes
    ~20 s a matrix, so it checks walker 0 there and the FP64 Gauss-Jordan
    form checks every walker."""
    L = lrugb()
    W = 5 if n <= 1152 else 4
    A = slater_batch(810 + n, W, n)
    A[2] = A[2] * 1e3                   # scale spread between walkers
    A[3, :, 5] *= 1e-6                  # spread inside one matrix
    tc = L.LowRankState("det", W, n, k=1, dtype=torch.float64, refresh=L.REFRESH_TENSOR)
    fp = L.LowRankState("det", W, n, k=1, dtype=torch.float64, refresh=L.REFRESH_FP64)
    la_tc, s_tc = tc.init(tdev(A))
    la_fp, s_fp = fp.init(tdev(A))
    inv_tc, inv_fp = tc.inverse().cpu().numpy(), fp.inverse().cpu().numpy()
    la_tc, la_fp = la_tc.cpu().numpy(), la_fp.cpu().numpy()
    s_tc, s_fp = s_tc.cpu().numpy(), s_fp.cpu().numpy()
    for w in range(W):
        assert fro_rel(inv_tc[w], inv_fp[w]) <= 1e-10, (w, fro_rel(inv_tc[w], inv_fp[w]))
        assert abs(la_tc[w] - la_fp[w]) <= 1e-12 * max(1.0, abs(la_fp[w]))
        assert s_tc[w] == s_fp[w]
        if n > 1152 and w > 0:
            continue
        ref = O.inv(A[w])
        sgn, la = O.slogdet(A[w])
        assert fro_rel(inv_tc[w], ref) <= 1e-10, (w, fro_rel(inv_tc[w], ref))
        assert abs(la_tc[w] - la) <= 1e-12 * max(1.0, abs(la))
        assert s_tc[w] == sgn
    tc.check_device_error()


def test_tensor_refresh_respects_mask_and_resets_delay():
    L = lrugb()
    W, n, K = 4, 256, 8
    A = slater_batch(831, W, n)
    st = L.LowRankState("det", W, n, k=1, dtype=torch.float64, delay=K, refresh=L.REFRESH_TENSOR)
    st.init(tdev(A))
    g = np.random.Generator(np.random.PCG64(832))
    for s in range(3):   # three pending slots
        rows = g.integers(0, n, (W, 1)).astype(np.int32)
        Vd = g.standard_normal((W, 1, n)) * 0.05
        st.propose_det(L.Operand(idx=tdev(rows), onehot_mask=1), L.Operand(dense=tdev(Vd)))
        st.accept()
    before = st.inverse().cpu().numpy()
    B = slater_batch(833, W, n)
    mask = np.array([1, 0, 0, 1], np.uint8)
    st.refresh(tdev(B), mask=tdev(mask), want_drift=False)
    after = st.inverse().cpu().numpy()
    tau = st.tau().cpu().numpy()
    for w in range(W):
        if mask[w]:
            assert fro_rel(after[w], O.inv(B[w])) <= 1e-10
            assert tau[w] == 0
        else:
            assert np.array_equal(after[w], before[w])
            assert tau[w] == 3


def test_tensor_refresh_singular_matrix():
    L = lrugb()
    W, n = 2, 128
    A = slater_batch(841, W, n)
    A[1, 7] = A[1, 3]                  # two equal rows
    st = L.LowRankState("det", W, n, k=1, dtype=torch.float64, refresh=L.REFRESH_TENSOR)
    la, s = st.init(tdev(A))
    la, s = la.cpu().numpy(), s.cpu().numpy()
    assert np.isfinite(la[0]) and s[0] != 0
    # rounding leaves a tiny pivot or none: either way |det| collapses or it is flagged
    assert la[1] < la[0] - 20 or not np.isfinite(la[1])


def test_delayed_chain_with_tensor_refresh_matches_oracle():
    # the C2 recipe at reduced size: Slater chain, K = 16, a tensor-core
    # refresh every 32 steps; the oracle rebuilds its carrier at the same steps
    L = lrugb()
    W, n, steps, K, every = 4, 256, 70, 16, 32
    Phi, occ0, slot, new = det_workload(851, W, n, 2 * n, steps)
    st = L.LowRankState("det", W, n, k=1, dtype=torch.float64, delay=K, refresh=L.REFRESH_TENSOR)
    Phi_d, occ_d = tdev(Phi), tdev(occ0)
    st.init(st.gather_rows(Phi_d, occ_d))
    slot_d, new_d = tdev(slot), tdev(new)
    ratios = []
    for s in range(steps):
        V, idx = st.form_row_moves(Phi_d, occ_d, slot_d[s], new_d[s])
        r, status = st.propose_det(L.Operand(idx=idx, onehot_mask=1), L.Operand(dense=V))
        st.accept()
        st.commit_moves(occ_d, slot_d[s], new_d[s])
        ratios.append(r.cpu().numpy())
        assert (status.cpu().numpy() == 0).all()
        if (s + 1) % every == 0:
            st.refresh(st.gather_rows(Phi_d, occ_d), want_drift=False)
    ratios = np.array(ratios)
    inv = st.inverse().cpu().numpy()
    for w in range(W):
        occ = occ0[w].copy()
        car = O.init_det_carrier(O.slater_matrix(Phi, occ), K)
        chain, exact = [], []
        for s in range(steps):
            U, V = O.det_row_move(Phi, occ, slot[s, w], new[s, w])
            exact.append(O.det_ratio_direct(O.slater_matrix(Phi, occ), U, V))
            chain.append(O.det_lru_delayed(car, U, V))
            occ[slot[s, w]] = new[s, w]
            if (s + 1) % every == 0:
                car = O.init_det_carrier(O.slater_matrix(Phi, occ), K)
        check_ratios(ratios[:, w], chain, exact, what=w, refresh_every=every, ceiling=CEIL_CHAIN)
        assert fro_rel(inv[w], O.carrier_inverse(car)) <= 1e-10
    st.check_device_error()


def test_tensor_refresh_with_drift_and_mask():
    # the drift (tracked inverse with its pending slots vs the fresh one) and the
    # state after the refresh, tensor-core form against the all-FP64 form
    L = lrugb()
    W, n, K, steps = 4, 256, 8, 13           # one flush, then 5 pending slots
    Phi, occ0, slot, new = det_workload(861, W, n, 2 * n, steps)
    out = {}
    for mode in (L.REFRESH_TENSOR, L.REFRESH_FP64):
        st = L.LowRankState("det", W, n, k=1, dtype=torch.float64, delay=K, refresh=mode)
        Phi_d, occ_d = tdev(Phi), tdev(occ0)
        st.init(st.gather_rows(Phi_d, occ_d))
        slot_d, new_d = tdev(slot), tdev(new)
        for s in range(steps):
            V, idx = st.form_row_moves(Phi_d, occ_d, slot_d[s], new_d[s])
            st.propose_det(L.Operand(idx=idx, onehot_mask=1), L.Operand(dense=V))
            st.accept()
            st.commit_moves(occ_d, slot_d[s], new_d[s])
        before = st.inverse().cpu().numpy()
        mask = np.array([1, 0, 1, 1], np.uint8)
        A = st.gather_rows(Phi_d, occ_d)
        drift = st.refresh(A, tdev(mask)).cpu().numpy()
        out[mode] = (drift, before, st.inverse().cpu().numpy(), st.tau().cpu().numpy(), A.cpu().numpy())
        st.check_device_error()
    d_tc, before, after, tau, A = out[L.REFRESH_TENSOR]
    d_fp = out[L.REFRESH_FP64][0]
    for w in range(W):
        if mask[w]:
            assert fro_rel(after[w], O.inv(A[w])) <= 1e-10
            assert tau[w] == 0
            assert 0 < d_tc[w] <= 1e-9 and abs(d_tc[w] - d_fp[w]) <= max(1e-13, 0.1 * d_fp[w])
        else:
            assert np.isnan(d_tc[w]) and tau[w] == steps % K
            assert np.array_equal(after[w], before[w])
