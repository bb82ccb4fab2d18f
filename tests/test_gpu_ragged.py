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
    assert res["delay"] in (0, 4, 8) and res["tile_chunks"] in (32, 64)
    assert len(res["trials"]) == 6 and all(t["updates_per_s"] > 0 for t in res["trials"])
    assert res["heuristic_delay"] == AT.heuristic_delay("det", 256, 1) == 26
    assert (tmp_path / "tune.json").exists()
    again = AT.tune("det", 256, 1, walkers=64, steps=24, delays=[4, 8], tiles=[32, 64])
    assert again == res   # served from the cache
