"""Walkers of uneven n and rank k in one persistent launch (CUDA-graph
capturable), its adjoint, Metropolis acceptance, and the autotuner.

Shapes follow the differentiation + uneven batching workload (backflow-style
dense U, V with N(0, 1/n) entries, complex64 / complex128) at sizes the
oracle finishes quickly; the full-size case is in test_gpu_fullsize.py.
"""
import numpy as np
import pytest

from gpu_common import O, fro_rel, lrugb, rel, tdev, torch

GO = pytest.importorskip("oracle.grad_oracle")

pytestmark = pytest.mark.gpu


def ragged_case(seed, W, ns, ks, cplx):
    g = np.random.Generator(np.random.PCG64(seed))
    n_w = g.choice(ns, W)
    k_w = g.choice(ks, W)
    kmax = int(max(ks))
    rnd = lambda *sh: (g.standard_normal(sh) + (1j * g.standard_normal(sh) if cplx else 0))
    A = [rnd(n, n) / np.sqrt(n) + 2.5 * np.eye(n) for n in n_w]
    U = [rnd(k, n) / np.sqrt(n) for n, k in zip(n_w, k_w)]
    V = [rnd(k, n) / np.sqrt(n) for n, k in zip(n_w, k_w)]
    return g, n_w, k_w, kmax, A, U, V


def flat_ops(vecs, n_w, kmax, dtype):
    """Operand vector layout of a ragged handle: walker w at sum(n_<w) * kmax, slot a at + a n_w."""
    out = np.zeros(int(np.sum(n_w)) * kmax, dtype=dtype)
    off = 0
    for v, n in zip(vecs, n_w):
        for a in range(v.shape[0]):
            out[off + a * n: off + (a + 1) * n] = v[a]
        off += n * kmax
    return out


def unflat_ops(flat, n_w, k_w, kmax):
    res, off = [], 0
    for n, k in zip(n_w, k_w):
        res.append(np.stack([flat[off + a * n: off + (a + 1) * n] for a in range(k)]))
        off += n * kmax
    return res


def flat_mats(mats):
    return np.concatenate([m.reshape(-1) for m in mats])


def unflat_mats(flat, n_w):
    res, off = [], 0
    for n in n_w:
        res.append(flat[off: off + n * n].reshape(n, n))
        off += n * n
    return res


@pytest.mark.parametrize("dt", ["c128", "c64", "f64"])
def test_ragged_persistent_propose_backward_accept(dt):
    L = lrugb()
    tdt = {"c128": torch.complex128, "c64": torch.complex64, "f64": torch.float64}[dt]
    cplx = dt != "f64"
    tol = 1e-3 if dt == "c64" else 1e-9
    W = 24
    g, n_w, k_w, kmax, A, U, V = ragged_case(1200, W, [16, 24, 40, 64, 100], [1, 2, 4], cplx)
    npdt = np.complex128 if cplx else np.float64
    st = L.LowRankState("det", W, [int(x) for x in n_w], k=kmax, dtype=tdt, k_per_walker=[int(x) for x in k_w])
    st.init(tdev(flat_mats(A), tdt))
    Ud = tdev(flat_ops(U, n_w, kmax, npdt), tdt)
    Vd = tdev(flat_ops(V, n_w, kmax, npdt), tdt)
    # propose only (one persistent launch), then the adjoint, then accept
    ratio, status, acc = st.step_persistent(L.Operand(dense=Ud), L.Operand(dense=Vd), accept=False)
    r = ratio.cpu().numpy()
    assert (status.cpu().numpy() == 0).all() and (acc.cpu().numpy() == 0).all()
    for w in range(W):
        ref = O.det_lru(O.inv(A[w]), U[w].T, V[w])
        assert rel(r[w], ref) <= tol, (w, r[w], ref)
    gvec = g.standard_normal(W) + (1j * g.standard_normal(W) if cplx else 0)
    gU, gV, gA = st.backward_det(tdev(gvec, tdt))
    gUl = unflat_ops(gU.cpu().numpy(), n_w, k_w, kmax)
    gVl = unflat_ops(gV.cpu().numpy(), n_w, k_w, kmax)
    gAl = unflat_mats(gA.cpu().numpy(), n_w)
    for w in range(W):
        rA, rU, rV = GO.vjp(GO.det_log_ratio, [torch.tensor(A[w]), torch.tensor(U[w].T), torch.tensor(V[w])],
                            gvec[w])
        assert fro_rel(gUl[w], rU.numpy().T) <= tol
        assert fro_rel(gVl[w], rV.numpy()) <= tol
        assert fro_rel(gAl[w], rA.numpy()) <= tol
    ratio2, status2, acc2 = st.step_persistent(L.Operand(dense=Ud), L.Operand(dense=Vd), accept=True)
    assert np.array_equal(ratio2.cpu().numpy(), r)
    assert (acc2.cpu().numpy() == 1).all()
    inv = unflat_mats(st.inverse().cpu().numpy(), n_w)
    logabs, _ = st.logvalue()
    for w in range(W):
        A1 = A[w] + U[w].T @ V[w]
        assert fro_rel(inv[w], O.inv(A1)) <= tol
        assert abs(logabs[w].item() - O.slogdet(A1)[1]) <= tol * max(1, abs(O.slogdet(A1)[1]))
    st.check_device_error()


def test_metropolis_acceptance_in_the_persistent_step():
    L = lrugb()
    W, n = 64, 32
    g = np.random.Generator(np.random.PCG64(1300))
    A = g.standard_normal((W, n, n)) / np.sqrt(n) + 2 * np.eye(n)
    st = L.LowRankState("det", W, n, k=1, dtype=torch.float64)
    st.init(tdev(A))
    rows = g.integers(0, n, (W, 1)).astype(np.int32)
    Vd = g.standard_normal((W, 1, n)) * 0.8
    u = g.random(W)
    ratio, status, acc = st.step_persistent(L.Operand(idx=tdev(rows), onehot_mask=1), L.Operand(dense=tdev(Vd)),
                                            u=tdev(u))
    r, acc = ratio.cpu().numpy(), acc.cpu().numpy()
    assert np.array_equal(acc.astype(bool), r ** 2 >= u)
    assert 0 < acc.sum() < W
    inv = st.inverse().cpu().numpy()
    for w in range(W):
        A1 = A[w].copy()
        if acc[w]:
            A1[rows[w, 0]] += Vd[w, 0]
        assert fro_rel(inv[w], O.inv(A1)) <= 1e-12


def test_graph_capture_replays_the_persistent_step():
    L = lrugb()
    W, n, steps = 48, 40, 4
    g = np.random.Generator(np.random.PCG64(1400))
    A = g.standard_normal((W, n, n)) / np.sqrt(n) + 2 * np.eye(n)
    rows_all = g.integers(0, n, (steps, W, 1)).astype(np.int32)
    V_all = g.standard_normal((steps, W, 1, n)) * 0.3
    # eager reference on one handle
    ref = L.LowRankState("det", W, n, k=1, dtype=torch.float64)
    ref.init(tdev(A))
    ref_ratios = []
    for s in range(steps):
        r, _, _ = ref.step_persistent(L.Operand(idx=tdev(rows_all[s]), onehot_mask=1),
                                      L.Operand(dense=tdev(V_all[s])))
        ref_ratios.append(r.cpu().numpy())
    # captured: static input buffers refilled before every replay
    st = L.LowRankState("det", W, n, k=1, dtype=torch.float64)
    st.init(tdev(A))
    rows_b = torch.zeros(W, 1, dtype=torch.int32, device="cuda")
    V_b = torch.zeros(W, 1, n, dtype=torch.float64, device="cuda")
    ratio_b = torch.zeros(W, dtype=torch.float64, device="cuda")
    status_b = torch.zeros(W, dtype=torch.int32, device="cuda")
    acc_b = torch.zeros(W, dtype=torch.uint8, device="cuda")
    Uo, Vo = L.Operand(idx=rows_b, onehot_mask=1), L.Operand(dense=V_b)
    side = L.LowRankState("det", W, n, k=1, dtype=torch.float64)   # warm-up outside the capture
    side.init(tdev(A))
    side.step_persistent(Uo, Vo, ratio=ratio_b, status=status_b, acc=acc_b)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        st.step_persistent(Uo, Vo, ratio=ratio_b, status=status_b, acc=acc_b)
    for s in range(steps):
        rows_b.copy_(tdev(rows_all[s]))
        V_b.copy_(tdev(V_all[s]))
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(ratio_b.cpu().numpy(), ref_ratios[s]), s
    assert np.array_equal(st.inverse().cpu().numpy(), ref.inverse().cpu().numpy())


def test_autotuner_returns_a_measured_setting(tmp_path, monkeypatch):
    monkeypatch.setenv("LRUGB_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    import importlib
    import paper_2602_05255_gb300.autotune as AT
    AT = importlib.reload(AT)
    res = AT.tune("det", 256, 1, walkers=64, steps=24, delays=[4, 8], tiles=[32, 64])
    L = AT.L
    assert res["delay"] in (0, 4, 8) and res["tile_chunks"] in (0, 32, 64)
    assert res["flush"] in (L.FLUSH_NATIVE, L.FLUSH_SPLIT, L.FLUSH_DF) and res["arith"] in (0, 1)
    # 2 GEMV arithmetics x (plain + 2 delays x 3 flush kernels), then 2 accept tiles
    assert len(res["trials"]) == 2 * (1 + 2 * 3) + 2 and all(t["updates_per_s"] > 0 for t in res["trials"])
    st = AT.make_state("det", 8, 256, tuned=res)      # the handle takes the tuned setting
    assert st.delay == res["delay"]
    st.close()
    assert res["heuristic_delay"] == AT.heuristic_delay("det", 256, 1) == 26
    assert (tmp_path / "tune.json").exists()
    again = AT.tune("det", 256, 1, walkers=64, steps=24, delays=[4, 8], tiles=[32, 64])
    assert again == res   # served from the cache


@pytest.mark.parametrize("dt", ["c128", "f64"])
@pytest.mark.parametrize("kind", ["det", "pf"])
def test_ragged_delayed_persistent_chain_graph(dt, kind):
    """The delayed form inside the persistent launch (Sec. 2.3 / 3.3): walkers
    of uneven n and k, a Metropolis-like mask so that every walker has its own
    delay counter, the slots of walkers that reach K folded into A_0^{-1} in
    the same launch; one step captured in a CUDA graph and replayed with new
    operands.  Every walker against the oracle's delayed chain, replaying the
    GPU's acceptance decisions."""
    L = lrugb()
    tdt = torch.complex128 if dt == "c128" else torch.float64
    cplx = dt == "c128"
    npdt = np.complex128 if cplx else np.float64
    W, K, steps = 12, 3, 11
    g = np.random.Generator(np.random.PCG64(1300 + (kind == "pf")))
    n_w = g.choice([16, 32, 48, 96] if kind == "det" else [16, 32, 48, 96], W)
    k_w = g.choice([1, 2, 3] if kind == "det" else [1, 2], W)
    kmax = int(k_w.max())
    slots = kmax if kind == "det" else 2 * kmax
    rnd = lambda *sh: (g.standard_normal(sh) + (1j * g.standard_normal(sh) if cplx else 0))
    if kind == "det":
        A = [rnd(n, n) / np.sqrt(n) + 2.5 * np.eye(n) for n in n_w]
    else:
        A = []
        for n in n_w:
            M = rnd(n, n) / np.sqrt(n)
            A.append(M - M.T + 2.5 * np.kron(np.eye(n // 2), np.array([[0, 1], [-1, 0]])))
    st = L.LowRankState(kind, W, [int(x) for x in n_w], k=kmax, dtype=tdt, delay=K,
                        k_per_walker=[int(x) for x in k_w])
    st.init(tdev(flat_mats(A), tdt))
    kk_w = k_w if kind == "det" else 2 * k_w
    Ud = torch.zeros(int(np.sum(n_w)) * slots, dtype=tdt, device="cuda")
    Vd = torch.zeros_like(Ud)
    Cd = torch.zeros(W * slots * slots, dtype=tdt, device="cuda")   # pf: C per walker (2k x 2k, skew)
    mask = torch.zeros(W, dtype=torch.uint8, device="cuda")
    ratio = torch.empty(W, dtype=tdt, device="cuda")
    status = torch.empty(W, dtype=torch.int32, device="cuda")
    acc = torch.empty(W, dtype=torch.uint8, device="cuda")

    def ops_for_step():
        U = [rnd(kk, n) * 0.3 / np.sqrt(n) for n, kk in zip(n_w, kk_w)]
        V = [rnd(kk, n) * 0.3 / np.sqrt(n) for n, kk in zip(n_w, kk_w)]
        Cs = []
        for kk in kk_w:
            Cm = rnd(kk, kk)
            Cs.append(Cm - Cm.T)
        return U, V, Cs

    def fill(U, V, Cs, m):
        Ud.copy_(tdev(flat_ops(U, n_w, slots, npdt), tdt))
        Vd.copy_(tdev(flat_ops(V, n_w, slots, npdt), tdt))
        Cflat = np.zeros(W * slots * slots, dtype=npdt)
        for w, Cm in enumerate(Cs):
            kk = Cm.shape[0]
            # walker w's 2k_w x 2k_w C, row-major, at w (2 kmax)^2
            Cflat[w * slots * slots: w * slots * slots + kk * kk] = Cm.reshape(-1)
        Cd.copy_(tdev(Cflat, tdt))
        mask.copy_(tdev(m.astype(np.uint8)))

    def step():
        Cp = Cd if kind == "pf" else None
        st.step_persistent(L.Operand(dense=Ud), None if kind == "pf" else L.Operand(dense=Vd), Cmat=Cp,
                           accept=True, mask=mask, ratio=ratio, status=status, acc=acc)

    rec = []
    graph = None
    for s in range(steps):
        U, V, Cs = ops_for_step()
        m = g.random(W) < 0.7
        fill(U, V, Cs, m)
        if s == 0:
            step()                              # one eager call before capturing
        elif s == 1:
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                step()
            graph.replay()
        else:
            graph.replay()
        torch.cuda.synchronize()
        rec.append((U, V, Cs, ratio.cpu().numpy().copy(), status.cpu().numpy().copy(), acc.cpu().numpy().copy()))
    st.check_device_error()
    tau = st.tau().cpu().numpy()
    inv = unflat_mats(st.inverse().cpu().numpy(), n_w)
    for w in range(W):
        car = O.init_det_carrier(A[w], K) if kind == "det" else O.init_pf_carrier(A[w], K)
        for s, (U, V, Cs, r, stt, ac) in enumerate(rec):
            assert stt[w] == 0
            if kind == "det":
                ref = O.det_lru_delayed(car, U[w].T, V[w], accept=bool(ac[w]))
            else:
                ref = O.pf_lru_delayed(car, U[w].T, Cs[w], accept=bool(ac[w]))
            assert rel(r[w], ref) <= 1e-9, (w, s, r[w], ref)
        assert tau[w] == car.tau, (w, tau[w], car.tau)
        assert fro_rel(inv[w], O.carrier_inverse(car)) <= 1e-9, w
    # every walker was due at some step, and not all at the same ones
    accepted = np.array([a for (_, _, _, _, _, a) in rec])
    assert (accepted.sum(0) >= K).all() and len(set(accepted.sum(0) % K)) > 1
