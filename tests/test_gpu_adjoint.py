"""GPU adjoint of the log ratios (hand-written backward kernels behind
torch.autograd.Function) against the FP64 autograd reference and central
finite differences.

Bounds: FP64 / complex128 relative error 1e-9 against the reference (the
reference itself is pinned by finite differences in test_oracle_grad.py);
complex64 1e-3 (single precision arithmetic, conditioning ~10).
"""
import numpy as np
import pytest

from gpu_common import O, lrugb, tdev, torch

GO = pytest.importorskip("oracle.grad_oracle")

pytestmark = pytest.mark.gpu

DT = {"f64": (torch.float64, np.float64, 1e-9), "c128": (torch.complex128, np.complex128, 1e-9),
      "c64": (torch.complex64, np.complex64, 1e-3)}


def rand(g, shape, cplx):
    x = g.standard_normal(shape)
    return x + 1j * g.standard_normal(shape) if cplx else x


def close(a, b, tol):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) <= tol * max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("dt", ["f64", "c128", "c64"])
@pytest.mark.parametrize("delay", [0, 3])
def test_det_adjoint(dt, delay):
    L = lrugb()
    tdt, ndt, tol = DT[dt]
    cplx = np.iscomplexobj(np.zeros(1, ndt))
    g = np.random.Generator(np.random.PCG64(901 + delay))
    W, n, k = 3, 24, 2
    A = rand(g, (W, n, n), cplx) / np.sqrt(n) + 2.5 * np.eye(n)
    st = L.LowRankState("det", W, n, k=k, dtype=tdt, delay=delay)
    st.init(tdev(A, tdt))
    # a few accepted updates (pending slots in the delayed form), tracked on the host
    for s in range(4):
        Ud = rand(g, (W, k, n), cplx) * 0.2
        Vd = rand(g, (W, k, n), cplx) * 0.2
        st.propose_det(L.Operand(dense=tdev(Ud, tdt)), L.Operand(dense=tdev(Vd, tdt)))
        st.accept()
        A = A + np.einsum("wkj,wkl->wjl", Ud, Vd)
    U = tdev(rand(g, (W, k, n), cplx) * 0.3, tdt).requires_grad_(True)
    V = tdev(rand(g, (W, k, n), cplx) * 0.3, tdt).requires_grad_(True)
    At = tdev(A, tdt).requires_grad_(True)
    logr = L.det_log_ratio(st, U, V, At)
    c = tdev(rand(g, (W,), cplx), tdt)
    (logr * c).real.sum().backward() if cplx else (logr * c).sum().backward()
    for w in range(W):
        Uw = U.detach()[w].cpu().numpy().astype(np.complex128 if cplx else np.float64).T
        Vw = V.detach()[w].cpu().numpy().astype(np.complex128 if cplx else np.float64)
        ref_logr = GO.det_log_ratio(torch.tensor(A[w]), torch.tensor(Uw), torch.tensor(Vw)).item()
        assert abs(logr[w].item() - ref_logr) <= tol * max(1, abs(ref_logr))
        # d(Re(c logr))/dz^* convention: torch's vjp with grad_output conj(c) for complex
        gw = np.conj(c[w].item()) if cplx else c[w].item()
        gA, gU, gV = GO.vjp(GO.det_log_ratio, [torch.tensor(A[w]), torch.tensor(Uw), torch.tensor(Vw)], gw)
        assert close(U.grad[w].cpu().numpy(), gU.numpy().T, tol), "gU"
        assert close(V.grad[w].cpu().numpy(), gV.numpy(), tol), "gV"
        assert close(At.grad[w].cpu().numpy(), gA.numpy(), tol), "gA"


@pytest.mark.parametrize("dt", ["f64", "c128"])
@pytest.mark.parametrize("delay", [0, 3])
def test_pf_adjoint(dt, delay):
    L = lrugb()
    tdt, ndt, tol = DT[dt]
    cplx = dt == "c128"
    g = np.random.Generator(np.random.PCG64(911 + delay))
    W, n, k = 3, 20, 2
    A = np.stack([O.skew_part(a) + 2 * O.skew_eye(n // 2) for a in rand(g, (W, n, n), cplx)])
    st = L.LowRankState("pf", W, n, k=k, dtype=tdt, delay=delay)
    st.init(tdev(A, tdt))
    for s in range(4):
        Bd = rand(g, (W, 2 * k, n), cplx) * 0.2
        Cd = np.stack([O.skew_part(x) for x in rand(g, (W, 2 * k, 2 * k), cplx)])
        st.propose_pf(L.Operand(dense=tdev(Bd, tdt)), tdev(Cd, tdt))
        st.accept()
        A = A + np.einsum("wbj,wbc,wcl->wjl", Bd, Cd, Bd)
    B = tdev(rand(g, (W, 2 * k, n), cplx) * 0.3, tdt).requires_grad_(True)
    Cm = tdev(np.stack([O.skew_part(x) for x in rand(g, (W, 2 * k, 2 * k), cplx)]) + 0.5 * O.skew_eye(k),
              tdt).requires_grad_(True)
    At = tdev(A, tdt).requires_grad_(True)
    logr = L.pf_log_ratio(st, B, Cm, At)
    c = tdev(rand(g, (W,), cplx), tdt)
    (logr * c).real.sum().backward() if cplx else (logr * c).sum().backward()
    for w in range(W):
        Bw = B.detach()[w].cpu().numpy().T
        Cw = Cm.detach()[w].cpu().numpy()
        gw = np.conj(c[w].item()) if cplx else c[w].item()
        r_ref = O.pf_ratio_direct(O.skew_part(A[w]), Bw, O.skew_part(Cw))
        r_gpu = np.exp(logr[w].item())
        if cplx:
            assert abs(r_gpu - r_ref) <= 1e-9 * abs(r_ref)
        else:
            assert abs(r_gpu - abs(r_ref)) <= 1e-9 * abs(r_ref)
        gA, gB, gC = GO.vjp(GO.pf_log_ratio, [torch.tensor(A[w]), torch.tensor(Bw), torch.tensor(Cw)], gw)
        assert close(B.grad[w].cpu().numpy(), gB.numpy().T, tol), "gB"
        assert close(Cm.grad[w].cpu().numpy(), gC.numpy(), tol), "gC"
        assert close(At.grad[w].cpu().numpy(), gA.numpy(), tol), "gA"


@pytest.mark.parametrize("cplx", [False, True])
def test_orbital_gradient_and_finite_differences(cplx):
    # d log ratio / d Phi through A = Phi[rows], plus dU, dV (backflow-style dense operands)
    L = lrugb()
    tdt = torch.complex128 if cplx else torch.float64
    g = np.random.Generator(np.random.PCG64(921))
    W, n, m, k = 3, 16, 40, 2
    Phi = rand(g, (m, n), cplx) / np.sqrt(n)
    rows = np.stack([g.permutation(m)[:n] for _ in range(W)]).astype(np.int32)
    st = L.LowRankState("det", W, n, k=k, dtype=tdt)
    Phi_d, rows_d = tdev(Phi, tdt), tdev(rows)
    st.init(st.gather_rows(Phi_d, rows_d))
    Ud = rand(g, (W, k, n), cplx) / np.sqrt(n)
    Vd = rand(g, (W, k, n), cplx) / np.sqrt(n)
    Phi_t = Phi_d.clone().requires_grad_(True)
    U, V = tdev(Ud, tdt).requires_grad_(True), tdev(Vd, tdt).requires_grad_(True)
    logr = L.orbital_log_ratio(st, Phi_t, rows_d, U, V)
    logr.real.sum().backward() if cplx else logr.sum().backward()
    # reference: autograd through torch indexing of Phi
    P = torch.tensor(Phi).requires_grad_(True)
    tot = 0
    for w in range(W):
        Aw = P[torch.tensor(rows[w]).long()]
        tot = tot + GO.det_log_ratio(Aw, torch.tensor(Ud[w].T), torch.tensor(Vd[w]))
    (tot.real if cplx else tot).backward()
    assert close(Phi_t.grad.cpu().numpy(), P.grad.numpy(), 1e-9)
    # central finite differences along a random direction of Phi (h = 1e-6, FP64)
    if not cplx:
        D = g.standard_normal((m, n))
        h = 1e-6

        def F(Ph):
            return sum(np.log(abs(O.det_ratio_direct(Ph[rows[w]], Ud[w].T, Vd[w]))) for w in range(W))

        fd = (F(Phi + h * D) - F(Phi - h * D)) / (2 * h)
        an = np.sum(Phi_t.grad.cpu().numpy() * D)
        assert abs(fd - an) <= 1e-6 * max(1, abs(an))


@pytest.mark.parametrize("kind", ["det", "pf"])
def test_logvalue_gradient(kind):
    L = lrugb()
    g = np.random.Generator(np.random.PCG64(931))
    W, n = 2, 18
    A = g.standard_normal((W, n, n)) + (0 if kind == "pf" else 3 * np.eye(n))
    if kind == "pf":
        A = A - A.transpose(0, 2, 1)
    st = L.LowRankState(kind, W, n, k=1, dtype=torch.float64, delay=4)
    st.init(tdev(A))
    gv = np.array([1.5, -0.5])
    gA = st.backward_logvalue(tdev(gv)).cpu().numpy()
    f = GO.log_det if kind == "det" else GO.log_pf
    for w in range(W):
        (ref,) = GO.vjp(f, [torch.tensor(A[w])], gv[w])
        assert close(gA[w], ref.numpy(), 1e-10)
