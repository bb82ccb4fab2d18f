"""GPU parity of the delayed flush in its precisions (Sec. 2.3 Eq. delayed_Ainv,
Sec. 3.3 Eq. pf_delayed_Ainv) and of the double-float GEMV.

- Tensor-core flush (tcgen05, TF32 or BF16 splits, FP32 accumulation):
  checked on a well-conditioned chain, where the error is the flush's own.
  Bounds from the arithmetic: TF32x3 (3-term split, ~2^-21 per product) 2e-6
  relative on ratios and A^{-1}; TF32 (11-bit operands) 2e-3; BF16x3 6e-5;
  BF16 (8-bit operands) 1.6e-2.  On ill-conditioned Slater chains
  the condition number amplifies any FP32-class flush error (even an exact
  FP32 GEMM); bench.py reports that drift instead of asserting it.
- Double-float flush and GEMV (FP32 pipe, ~1e-14): the FP64 bar (relative
  1e-10, condition-aware) on realistic Slater and pairing chains.
"""
import numpy as np
import pytest

from gpu_common import (CEIL_CHAIN, O, check_inverse, check_ratios, det_workload, fro_rel, lrugb, pf_workload, rel,
                        replay_det_oracle, run_det_chain_gpu, tdev, torch)

pytestmark = pytest.mark.gpu

# relative bounds from the flush arithmetic (operand splits x FP32 accumulation)
# TF32x3 ~2^-21, TF32 2 * 2^-11, BF16x3 ~2 * 2^-16, BF16 2 * 2^-8 per product, with margin
BOUND = {1: 2e-6, 2: 2e-3, 3: 1.6e-2, 4: 6e-5}


def well_conditioned_chain(L, W, n, K, steps, flush, arith, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    A = 3.0 * np.eye(n) + g.standard_normal((W, n, n)) / np.sqrt(n)
    st = L.LowRankState("det", W, n, k=1, dtype=torch.float64, delay=K, flush=flush, arith=arith)
    st.init(tdev(A))
    cars = [O.init_det_carrier(A[w], K) for w in range(W)]
    worst = 0.0
    for s in range(steps):
        rows = g.integers(0, n, (W, 1)).astype(np.int32)
        Vd = g.standard_normal((W, 1, n)) * 0.3 / np.sqrt(n)
        r, status = st.propose_det(L.Operand(idx=tdev(rows), onehot_mask=1), L.Operand(dense=tdev(Vd)))
        st.accept()
        r = r.cpu().numpy()
        assert (status.cpu().numpy() == 0).all()
        for w in range(W):
            ref = O.det_lru_delayed(cars[w], O.onehot_matrix(n, rows[w]), Vd[w])
            worst = max(worst, rel(r[w], ref))
    inv = st.inverse().cpu().numpy()
    inv_err = max(fro_rel(inv[w], O.carrier_inverse(cars[w])) for w in range(W))
    return st, worst, inv_err


@pytest.mark.parametrize("mode", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [200, 256])
def test_tc_flush_precision(mode, n):
    # K = 16: 40 steps = two full flushes + 8 pending; n = 200 leaves partial
    # 128-row tiles that cross into the next walker's rows
    L = lrugb()
    st, worst, inv_err = well_conditioned_chain(L, 5, n, 16, 40, mode, L.ARITH_DF, 500 + n)
    assert worst <= BOUND[mode], worst
    assert inv_err <= BOUND[mode], inv_err
    st.check_device_error()


@pytest.mark.parametrize("n", [200, 256])
def test_df_flush_precision(n):
    L = lrugb()
    st, worst, inv_err = well_conditioned_chain(L, 5, n, 16, 40, L.FLUSH_DF, L.ARITH_DF, 600 + n)
    assert worst <= 1e-12 and inv_err <= 1e-12, (worst, inv_err)


@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("flush", [0, 5, 6])
def test_det_delayed_fp64_class_on_slater_chain(arith, flush):
    # realistic Slater chain (Phi N(0, 1/n), ill-conditioned): native FP64 or
    # double-float GEMV, FP64 or double-float flush, all at the FP64 bar
    L = lrugb()
    W, n, K, steps = 5, 256 if flush == 6 else 200, 16, 40
    Phi, occ0, slot, new = det_workload(700 + n, W, n, 2 * n, steps)
    st, ratios, status, _ = run_det_chain_gpu(L, Phi, occ0, slot, new, delay=K, flush=flush, arith=arith)
    assert (status == 0).all()
    inv = st.inverse().cpu().numpy()
    # products of double-float splits: unit roundoff 2^-46, two of them per chain: 2^8 x FP64's
    scale = 256.0 if (arith != 0 or flush == 5) else 1.0
    for w in range(W):
        rs, inv_ref, _, ex = replay_det_oracle(Phi, occ0, slot, new, w, delay=K)
        check_ratios(ratios[:, w], rs, ex, what=(arith, flush, w), eps_scale=scale, ceiling=CEIL_CHAIN * scale)
        assert fro_rel(inv[w], inv_ref) <= 1e-10 * scale


def test_det_tc_matches_native_before_first_flush():
    # until the first flush the two flush modes run identical FP64 arithmetic
    L = lrugb()
    W, n, m, steps, K = 3, 128, 256, 15, 16
    Phi, occ0, slot, new = det_workload(401, W, n, m, steps)
    _, r_tc, _, _ = run_det_chain_gpu(L, Phi, occ0, slot, new, delay=K, flush=1)
    _, r_nat, _, _ = run_det_chain_gpu(L, Phi, occ0, slot, new, delay=K, flush=0)
    assert np.array_equal(r_tc, r_nat)


def test_det_rank2_two_k_chunks():
    # k = 2 two-row moves, K = 32: 64 slot columns = two 32-wide K chunks of the MMA
    L = lrugb()
    W, n, K, steps = 3, 300, 32, 70
    g = np.random.Generator(np.random.PCG64(411))
    A = g.standard_normal((W, n, n)) / np.sqrt(n) + 2.0 * np.eye(n)
    st = L.LowRankState("det", W, n, k=2, dtype=torch.float64, delay=K, flush=1)
    st.init(tdev(A))
    cars = [O.init_det_carrier(A[w], K) for w in range(W)]
    worst = 0.0
    for s in range(steps):
        rows = np.stack([g.choice(n, 2, replace=False) for _ in range(W)]).astype(np.int32)
        Vd = g.standard_normal((W, 2, n)) * 0.05
        r, status = st.propose_det(L.Operand(idx=tdev(rows), onehot_mask=0b11), L.Operand(dense=tdev(Vd)))
        st.accept()
        r = r.cpu().numpy()
        for w in range(W):
            U = O.onehot_matrix(n, rows[w])
            ref = O.det_lru_delayed(cars[w], U, Vd[w])
            worst = max(worst, rel(r[w], ref))
    assert worst <= 2e-6, worst
    inv = st.inverse().cpu().numpy()
    for w in range(W):
        assert fro_rel(inv[w], O.carrier_inverse(cars[w])) <= 2e-6
    assert (st.tau().cpu().numpy() == steps % K).all()


@pytest.mark.parametrize("flush", [1, 5, 6])
def test_pf_delayed_flush_exactly_skew(flush):
    # realistic pairing chain: the flushed A_0^{-1} is exactly skew in both
    # precisions; the double-float flush also meets the FP64 bar (64x roundoff)
    L = lrugb()
    W, n, m, steps, K = 4, 256 if flush == 6 else 136, 512 if flush == 6 else 300, 16, 8
    F, pos0, slot, new = pf_workload(421, W, n, m, steps)
    st = L.LowRankState("pf", W, n, k=1, dtype=torch.float64, delay=K, flush=flush)
    F_d, pos_d = tdev(F), tdev(pos0)
    st.init(st.gather_pairs(F_d, pos_d))
    ratios = []
    for s in range(steps):
        B, idx = st.form_pf_moves(F_d, pos_d, tdev(slot[s]), tdev(new[s]))
        r, _ = st.propose_pf(L.Operand(dense=B, idx=idx, onehot_mask=0b10))
        st.accept()
        st.commit_moves(pos_d, tdev(slot[s]), tdev(new[s]))
        ratios.append(r.cpu().numpy())
    ratios = np.array(ratios)
    assert (st.tau().cpu().numpy() == 0).all()
    inv = st.inverse().cpu().numpy()      # = A_0^{-1} right after the second flush
    for w in range(W):
        assert np.array_equal(inv[w], -inv[w].T)
        if flush == 1:
            continue
        pos = pos0[w].copy()
        car = O.init_pf_carrier(O.pairing_matrix(F, pos), K)
        chain, exact = [], []
        for s in range(steps):
            B, C = O.pf_row_col_move(F, pos, slot[s, w], new[s, w])
            exact.append(O.pf_ratio_direct(O.pairing_matrix(F, pos), B, C))
            chain.append(O.pf_lru_delayed(car, B, C))
            pos[slot[s, w]] = new[s, w]
        scale = 256.0 if flush == 5 else 1.0     # double-float flush; the split product rounds as FP64
        check_ratios(ratios[:, w], chain, exact, what=(flush, w), eps_scale=scale, ceiling=CEIL_CHAIN * scale)
        check_inverse(inv[w], O.carrier_inverse(car), O.inv(O.pairing_matrix(F, pos)), what=(flush, w),
                      eps_scale=scale)


@pytest.mark.parametrize("mode", [1, 2, 3, 4])
def test_pf_tc_flush_precision(mode):
    # well-conditioned skew chain: A = 3 J + small skew noise, small row+column moves
    L = lrugb()
    W, n, K, steps = 4, 200, 8, 20
    g = np.random.Generator(np.random.PCG64(441))
    G = g.standard_normal((W, n, n)) * np.sqrt(0.1 / n)
    A = 3.0 * O.skew_eye(n // 2)[None] + G - G.transpose(0, 2, 1)
    st = L.LowRankState("pf", W, n, k=1, dtype=torch.float64, delay=K, flush=mode)
    st.init(tdev(A))
    cars = [O.init_pf_carrier(A[w], K) for w in range(W)]
    worst = 0.0
    for s in range(steps):
        x = g.standard_normal((W, n)) * 0.3 / np.sqrt(n)
        i = g.integers(0, n, W).astype(np.int32)
        Bd = np.zeros((W, 2, n)); Bd[:, 0] = x
        idx = np.zeros((W, 2), np.int32); idx[:, 1] = i
        r, status = st.propose_pf(L.Operand(dense=tdev(Bd), idx=tdev(idx), onehot_mask=0b10))
        st.accept()
        r = r.cpu().numpy()
        for w in range(W):
            B = np.stack([x[w], O.onehot_matrix(n, [i[w]])[:, 0]], 1)
            worst = max(worst, rel(r[w], O.pf_lru_delayed(cars[w], B)))
    assert worst <= BOUND[mode], worst
    inv = st.inverse().cpu().numpy()
    for w in range(W):
        assert fro_rel(inv[w], O.carrier_inverse(cars[w])) <= BOUND[mode]


@pytest.mark.parametrize("flush", [1, 5])
def test_forced_partial_flush(flush):
    # lru_flush_delayed folds tau < K slots; stale columns of earlier windows must not leak in
    L = lrugb()
    W, n, K, steps = 4, 160, 8, 23        # 2 full windows, then 7 pending
    st, _, _ = well_conditioned_chain(L, W, n, K, steps, flush, L.ARITH_DF, 431)
    before = st.inverse().cpu().numpy()
    mask = np.array([1, 0, 1, 1], np.uint8)
    st.flush(tdev(mask))
    tau = st.tau().cpu().numpy()
    after = st.inverse().cpu().numpy()
    tol = 1e-12 if flush == 5 else 2e-6
    for w in range(W):
        assert fro_rel(after[w], before[w]) <= tol
        assert tau[w] == (0 if mask[w] else steps % K)
        if not mask[w]:
            assert np.array_equal(after[w], before[w])
    st.check_device_error()


# ---- exact split-product flush on the tensor cores (FP64 bar) -------------------

def test_split_flush_precision_well_conditioned():
    L = lrugb()
    st, worst, inv_err = well_conditioned_chain(L, 5, 256, 16, 40, L.FLUSH_SPLIT, L.ARITH_NATIVE, 611)
    assert worst <= 1e-12 and inv_err <= 1e-12, (worst, inv_err)
    st.check_device_error()


@pytest.mark.parametrize("K", [8, 16])
def test_split_flush_on_slater_chain(K):
    # realistic Slater chain at the FP64 bar (plain FP64 rounding scale)
    L = lrugb()
    W, n, steps = 4, 256, 40
    Phi, occ0, slot, new = det_workload(720 + K, W, n, 2 * n, steps)
    st, ratios, status, _ = run_det_chain_gpu(L, Phi, occ0, slot, new, delay=K, flush=L.FLUSH_SPLIT)
    assert (status == 0).all()
    inv = st.inverse().cpu().numpy()
    for w in range(W):
        rs, inv_ref, occ, ex = replay_det_oracle(Phi, occ0, slot, new, w, delay=K)
        check_ratios(ratios[:, w], rs, ex, what=w, ceiling=CEIL_CHAIN)
        # A^{-1} against the exact inverse, with the oracle chain's own FP64 drift as the scale
        exact = O.inv(O.slater_matrix(Phi, occ))
        assert fro_rel(inv[w], exact) <= max(1e-10, 10 * fro_rel(inv_ref, exact))
    st.check_device_error()


def test_split_flush_forced_partial():
    L = lrugb()
    W, n, K, steps = 4, 128, 8, 23        # 2 full windows, then 7 pending
    st, _, _ = well_conditioned_chain(L, W, n, K, steps, L.FLUSH_SPLIT, L.ARITH_NATIVE, 631)
    before = st.inverse().cpu().numpy()
    mask = np.array([1, 0, 1, 1], np.uint8)
    st.flush(tdev(mask))
    tau = st.tau().cpu().numpy()
    after = st.inverse().cpu().numpy()
    for w in range(W):
        assert fro_rel(after[w], before[w]) <= 1e-12
        assert tau[w] == (0 if mask[w] else steps % K)
        if not mask[w]:
            assert np.array_equal(after[w], before[w])
    st.check_device_error()


def test_split_flush_rejects_unsupported_shapes():
    L = lrugb()
    with pytest.raises(L.LRUError):   # n not a multiple of 128
        L.LowRankState("det", 2, 200, k=1, dtype=torch.float64, delay=8, flush=L.FLUSH_SPLIT)
    with pytest.raises(L.LRUError):   # Pfaffian, n not a multiple of 128
        L.LowRankState("pf", 2, 200, k=1, dtype=torch.float64, delay=8, flush=L.FLUSH_SPLIT)
    with pytest.raises(L.LRUError):   # complex
        L.LowRankState("pf", 2, 256, k=1, dtype=torch.complex128, delay=8, flush=L.FLUSH_SPLIT)


def _column_balance(P, Q):
    """The flush's exact column balance: column c of P times 2^s_c and of Q
    times 2^-s_c, s_c = (eQ_c - eP_c) / 2 truncated, eX_c the biased exponent
    of the column's largest entry (the product P Q^T is unchanged)."""
    def bexp(x):
        m = np.abs(x).max(0)
        return np.where(m > 0, np.frexp(m)[1] + 1022, 0)
    ep, eq = bexp(P), bexp(Q)
    s = np.where((ep > 0) & (eq > 0), np.trunc((eq - ep) / 2), 0).astype(int)
    return P * 2.0 ** s, Q * 2.0 ** -s


def test_split_flush_against_exact_rational_arithmetic():
    # A_0^{-1} -= P Q^T on planted slots with a wide dynamic range across slot
    # columns, against exact rational arithmetic.  The split product's error
    # bound is relative to the row maxima of the column-balanced slots P~, Q~:
    # |err| <= 2^-52 (maxP~_j sum|Q~_l| + sum|P~_j| maxQ~_l) + 2^-52 |result|
    # (quantisation to 2^-56 of the maxima, levels kept down to 2^-66, two
    # FP64 roundings).  The balance brings that bound to within a small factor
    # of an FP64 flush's, 2^-52 (K sum_c |P_jc Q_lc| + |result|).
    from fractions import Fraction
    L = lrugb()
    W, n, K = 2, 128, 16
    st = L.LowRankState("det", W, n, k=1, dtype=torch.float64, delay=K, flush=L.FLUSH_SPLIT)
    g = np.random.Generator(np.random.PCG64(641))
    st.init(tdev(g.standard_normal((W, n, n)) + 4 * np.eye(n)))
    buf = st.save().cpu().numpy().copy()
    al = lambda x: (x + 255) // 256 * 256
    oG, oP = 0, al(W * n * n * 8)
    oQ = oP + al(W * n * K * 8)
    oT = oQ + al(W * n * K * 8)
    G0 = g.standard_normal((W, n, n))
    ea, eb = g.uniform(-3, 3, K), g.uniform(-2, 2, K)
    P = g.standard_normal((W, n, K)) * 10.0 ** ea
    Q = g.standard_normal((W, n, K)) * 10.0 ** (eb - ea)
    buf[oG:oG + W * n * n * 8] = G0.reshape(-1).view(np.uint8)
    buf[oP:oP + W * n * K * 8] = P.reshape(-1).view(np.uint8)
    buf[oQ:oQ + W * n * K * 8] = Q.reshape(-1).view(np.uint8)
    buf[oT:oT + W * 4] = np.full(W, K, np.int32).view(np.uint8)
    st.load(tdev(buf))
    st.flush(tdev(np.ones(W, np.uint8)))
    G1 = st.save().cpu().numpy()[oG:oG + W * n * n * 8].view(np.float64).reshape(W, n, n)
    worst, worst64 = 0.0, 0.0
    for w in range(W):
        Pb, Qb = _column_balance(P[w], Q[w])
        for _ in range(1500):
            l, j = g.integers(0, n, 2)          # storage row l, column j: (A^{-1})_{jl}
            ex = Fraction(G0[w, l, j]) - sum(Fraction(P[w, j, c]) * Fraction(Q[w, l, c]) for c in range(K))
            bound = 2.0 ** -52 * (np.abs(Pb[j]).max() * np.abs(Qb[l]).sum() +
                                  np.abs(Pb[j]).sum() * np.abs(Qb[l]).max() + abs(float(ex)))
            err = abs(float(Fraction(G1[w, l, j]) - ex))
            worst = max(worst, err / bound)
            fp64 = 2.0 ** -52 * (K * np.abs(P[w, j] * Q[w, l]).sum() + abs(float(ex)))
            worst64 = max(worst64, err / fp64)
    print("split flush: worst error / own bound %.3f, / FP64 bound %.3f" % (worst, worst64))
    assert worst <= 1.0, worst
    assert worst64 <= 8.0, worst64
    assert (st.tau().cpu().numpy() == 0).all()
