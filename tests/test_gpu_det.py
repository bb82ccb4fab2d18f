"""GPU parity of the determinant path (Sec. 2) against the CPU oracle.

Every test runs the CUDA library through the C-ABI binding and compares with
the oracle on the same seeded inputs.  FP64 / complex128 tolerance: relative
error <= 1e-10 on every ratio and on A^{-1} after the chain.
"""
import numpy as np
import pytest

from gpu_common import (O, RTOL_F64, check_ratios, det_workload, fro_rel, lrugb, rel, replay_det_oracle,
                        run_det_chain_gpu, tdev, torch)

pytestmark = pytest.mark.gpu


def test_config_small_exact_chain():
    # 1 walker, n = 64, Phi 128 x 64 N(0,1), rows 0..63, 100 rank-1 row swaps,
    # every ratio against a from-scratch recompute; refresh at the end
    L = lrugb()
    Phi, occ0, slot, new = det_workload(1, 1, 64, 128, 100, var=1.0, first_rows=True)
    st, ratios, status, occ_end = run_det_chain_gpu(L, Phi, occ0, slot, new)
    assert (status == 0).all()
    occ = occ0[0].copy()
    for s in range(100):
        A = O.slater_matrix(Phi, occ)
        U, V = O.det_row_move(Phi, occ, slot[s, 0], new[s, 0])
        ref = O.det_ratio_direct(A, U, V)
        assert rel(ratios[s, 0], ref) <= RTOL_F64, (s, ratios[s, 0], ref)
        occ[slot[s, 0]] = new[s, 0]
    assert np.array_equal(occ, occ_end[0])
    A = O.slater_matrix(Phi, occ)
    inv_gpu = st.inverse().cpu().numpy()[0]
    assert fro_rel(inv_gpu, O.inv(A)) <= RTOL_F64
    logabs, sign = st.logvalue()
    s_ref, l_ref = O.slogdet(A)
    assert abs(logabs.item() - l_ref) <= 1e-9 * max(1.0, abs(l_ref))
    assert sign.item() == s_ref
    drift = st.refresh(tdev(A[None]))
    assert drift.item() <= RTOL_F64
    assert fro_rel(st.inverse().cpu().numpy()[0], O.inv(A)) <= 1e-12


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("delay", [0, 4, 5])
def test_batched_chain_matches_oracle(cplx, delay):
    # 6 walkers, n = 80 (a ragged tail of every 32-wide warp pass), 30 moves
    L = lrugb()
    W, n, m, steps = 6, 80, 160, 30
    Phi, occ0, slot, new = det_workload(20 + delay, W, n, m, steps, cplx)
    st, ratios, status, occ_end = run_det_chain_gpu(L, Phi, occ0, slot, new, delay=delay)
    assert (status == 0).all()
    inv_gpu = st.inverse().cpu().numpy()
    for w in range(W):
        rs, inv_ref, occ, ex = replay_det_oracle(Phi, occ0, slot, new, w, delay=delay)
        check_ratios(ratios[:, w], rs, ex, what=w)
        assert fro_rel(inv_gpu[w], inv_ref) <= RTOL_F64
        assert np.array_equal(occ, occ_end[w])
    if delay:
        assert (st.tau().cpu().numpy() == steps % delay).all()


def test_masked_rejections_delayed():
    L = lrugb()
    W, n, m, steps, K = 5, 64, 128, 24, 4
    Phi, occ0, slot, new = det_workload(31, W, n, m, steps)
    mask = (np.random.Generator(np.random.PCG64(5)).random((steps, W)) < 0.6)
    # a Metropolis step never accepts a node (a move onto a row another slot
    # already holds, ratio 0): reject those, as the moves assume all accepted
    occ = occ0.copy()
    for s in range(steps):
        for w in range(W):
            if new[s, w] in occ[w]:
                mask[s, w] = False
            if mask[s, w]:
                occ[w, slot[s, w]] = new[s, w]
    st, ratios, status, occ_end = run_det_chain_gpu(L, Phi, occ0, slot, new, delay=K, mask_seq=mask)
    inv_gpu = st.inverse().cpu().numpy()
    tau = st.tau().cpu().numpy()
    for w in range(W):
        rs, inv_ref, occ, ex = replay_det_oracle(Phi, occ0, slot, new, w, delay=K, mask_seq=mask)
        # rejected proposals were formed from the unchanged occupation; a move
        # onto a row another slot already holds is an exact node (ratio 0)
        check_ratios(ratios[:, w], rs, ex, what=w)
        assert fro_rel(inv_gpu[w], inv_ref) <= RTOL_F64
        assert np.array_equal(occ, occ_end[w])
        assert tau[w] == mask[:, w].sum() % K


@pytest.mark.parametrize("delay", [0, 3])
def test_dense_and_mixed_operands(delay):
    # rank-2 updates: dense U, V (backflow-like), and the simultaneous
    # row-and-column update of Sec. 2.2 in mixed one-hot / dense form
    L = lrugb()
    W, n, k, steps = 4, 40, 2, 7
    g = np.random.Generator(np.random.PCG64(41))
    A = g.standard_normal((W, n, n)) / np.sqrt(n) + 2 * np.eye(n)
    st = L.LowRankState("det", W, n, k=k, dtype=torch.float64, delay=delay)
    st.init(tdev(A))
    cars = [O.init_det_carrier(A[w], max(delay, 2)) if delay else None for w in range(W)]
    Ainv = [O.inv(A[w]) for w in range(W)]
    for s in range(steps):
        if s % 2 == 0:
            Ud = g.standard_normal((W, k, n)) * 0.2
            Vd = g.standard_normal((W, k, n)) * 0.2
            Uop, Vop = L.Operand(dense=tdev(Ud)), L.Operand(dense=tdev(Vd))
            Um = [Ud[w].T for w in range(W)]
            Vm = [Vd[w] for w in range(W)]
        else:
            # U = [xv, e_i] (column update + one-hot), V = [e_j^T; xu^T]
            xv = g.standard_normal((W, n)) * 0.3
            xu = g.standard_normal((W, n)) * 0.3
            i = g.integers(0, n, W)
            j = g.integers(0, n, W)
            Ud = np.zeros((W, k, n)); Ud[:, 0] = xv
            Vd = np.zeros((W, k, n)); Vd[:, 1] = xu
            Uidx = np.zeros((W, k), np.int32); Uidx[:, 1] = i
            Vidx = np.zeros((W, k), np.int32); Vidx[:, 0] = j
            Uop = L.Operand(dense=tdev(Ud), idx=tdev(Uidx), onehot_mask=0b10)
            Vop = L.Operand(dense=tdev(Vd), idx=tdev(Vidx), onehot_mask=0b01)
            Um = [np.stack([xv[w], O.onehot_matrix(n, [i[w]])[:, 0]], 1) for w in range(W)]
            Vm = [np.stack([O.onehot_matrix(n, [j[w]])[:, 0], xu[w]], 0) for w in range(W)]
        r, status = st.propose_det(Uop, Vop)
        st.accept()
        r = r.cpu().numpy()
        for w in range(W):
            if delay:
                ref = O.det_lru_delayed(cars[w], Um[w], Vm[w])
            else:
                ref, Ainv[w] = O.det_lru(Ainv[w], Um[w], Vm[w], return_update=True)
            assert rel(r[w], ref) <= RTOL_F64, (s, w)
            A[w] = A[w] + Um[w] @ Vm[w]
    inv_gpu = st.inverse().cpu().numpy()
    for w in range(W):
        assert fro_rel(inv_gpu[w], O.inv(A[w])) <= 1e-9


def test_singular_core_and_bad_index():
    L = lrugb()
    W, n = 3, 16
    A = np.eye(n)[None].repeat(W, 0) * 2.0
    st = L.LowRankState("det", W, n, k=1, dtype=torch.float64)
    st.init(tdev(A))
    # walker 0: row 3 replaced by zero -> R = 1 + V A^{-1} e_3 = 1 - 1 = 0 (a node)
    V = np.zeros((W, 1, n)); V[0, 0, 3] = -2.0; V[1, 0, 5] = 1.0; V[2, 0, 0] = 1.0
    idx = np.array([[3], [5], [n + 4]], np.int32)
    r, status = st.propose_det(L.Operand(idx=tdev(idx), onehot_mask=1), L.Operand(dense=tdev(V)))
    st.accept()
    r, status = r.cpu().numpy(), status.cpu().numpy()
    assert status[0] == L.WALKER_SINGULAR and r[0] == 0.0
    assert status[1] == L.WALKER_OK and r[1] == pytest.approx(1.5)
    assert status[2] == L.WALKER_BAD_INDEX
    inv = st.inverse().cpu().numpy()
    assert np.array_equal(inv[0], np.eye(n) / 2)            # unchanged
    assert np.array_equal(inv[2], np.eye(n) / 2)
    A1 = A[1].copy(); A1[5, 5] += 1.0
    assert np.allclose(inv[1], np.linalg.inv(A1), atol=1e-15)


def test_save_load_resume_bitwise():
    L = lrugb()
    W, n, m, steps, K = 3, 48, 96, 14, 4
    Phi, occ0, slot, new = det_workload(55, W, n, m, steps)
    st, ratios, _, _ = run_det_chain_gpu(L, Phi, occ0, slot, new, delay=K)
    inv_full = st.inverse().cpu().numpy()
    # first half, save, new handle, load, second half
    h = steps // 2
    st1, r1, _, occ_mid = run_det_chain_gpu(L, Phi, occ0, slot[:h], new[:h], delay=K)
    blob = st1.save()
    st2 = L.LowRankState("det", W, n, k=1, dtype=torch.float64, delay=K)
    st2.load(blob)
    Phi_d, occ_d = tdev(Phi), tdev(occ_mid)
    rs = []
    for s in range(h, steps):
        V, idx = st2.form_row_moves(Phi_d, occ_d, tdev(slot[s]), tdev(new[s]))
        r, _ = st2.propose_det(L.Operand(idx=idx, onehot_mask=1), L.Operand(dense=V))
        st2.accept()
        st2.commit_moves(occ_d, tdev(slot[s]), tdev(new[s]))
        rs.append(r.cpu().numpy())
    assert np.array_equal(np.concatenate([r1, np.array(rs)]), ratios)
    assert np.array_equal(st2.inverse().cpu().numpy(), inv_full)


@pytest.mark.parametrize("cplx", [False, True])
def test_slogdet_batched(cplx):
    L = lrugb()
    g = np.random.Generator(np.random.PCG64(61))
    for n in (1, 7, 33, 100):
        A = g.standard_normal((5, n, n)) + (1j * g.standard_normal((5, n, n)) if cplx else 0)
        sgn, logabs = L.slogdet_batched(tdev(A))
        for w in range(5):
            s_ref, l_ref = O.slogdet(A[w])
            assert abs(logabs[w].item() - l_ref) <= 1e-11 * max(1, abs(l_ref))
            assert abs(sgn[w].cpu().item() - s_ref) <= 1e-11


def test_refresh_mask_and_drift():
    L = lrugb()
    W, n, m, steps = 4, 64, 128, 12
    Phi, occ0, slot, new = det_workload(71, W, n, m, steps)
    st, _, _, occ_end = run_det_chain_gpu(L, Phi, occ0, slot, new, delay=5)
    A = np.stack([O.slater_matrix(Phi, occ_end[w]) for w in range(W)])
    mask = np.array([1, 0, 1, 0], np.uint8)
    before = st.inverse().cpu().numpy()
    drift = st.refresh(tdev(A), tdev(mask)).cpu().numpy()
    after = st.inverse().cpu().numpy()
    tau = st.tau().cpu().numpy()
    for w in range(W):
        if mask[w]:
            assert drift[w] <= RTOL_F64 and tau[w] == 0
            assert fro_rel(after[w], O.inv(A[w])) <= 1e-12
        else:
            assert np.isnan(drift[w]) and tau[w] == steps % 5
            assert np.array_equal(after[w], before[w])
