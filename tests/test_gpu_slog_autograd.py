"""Differentiable batched slogdet / slogpf (App. A.1 slogpf, App. A.3 Eq.
pf_grad): the forward is lru_slogdet_batched / lru_slogpf_batched, the
backward lru_slogdet_backward / lru_slogpf_backward.  Checked against CPU
torch autograd of torch.linalg.slogdet (the Pfaffian through
log|pf| = (1/2) log|det| of the skew part) and against central finite
differences (h = 1e-6) of the GPU forward itself."""
import numpy as np
import pytest

from gpu_common import fro_rel, lrugb, tdev, torch

GO = pytest.importorskip("oracle.grad_oracle")

pytestmark = pytest.mark.gpu


def _rand(g, shape, cplx):
    return g.standard_normal(shape) + (1j * g.standard_normal(shape) if cplx else 0)


@pytest.mark.parametrize("dt", ["f64", "c128"])
@pytest.mark.parametrize("n", [7, 64, 129])
def test_slogdet_gradient_matches_torch_autograd(dt, n):
    L = lrugb()
    cplx = dt == "c128"
    g = np.random.Generator(np.random.PCG64(500 + n))
    W = 5
    A = _rand(g, (W, n, n), cplx) / np.sqrt(n) + 2.0 * np.eye(n)
    a = g.standard_normal(W)
    b = _rand(g, W, True)
    At = tdev(A).requires_grad_(True)
    sign, logabs = L.slogdet(At)
    loss = (tdev(a) * logabs).sum()
    if cplx:
        loss = loss + (torch.conj(tdev(b)) * sign).real.sum()
    loss.backward()
    Ac = torch.tensor(A, requires_grad=True)
    s_ref, l_ref = torch.linalg.slogdet(Ac)
    loss_ref = (torch.tensor(a) * l_ref).sum()
    if cplx:
        loss_ref = loss_ref + (torch.conj(torch.tensor(b)) * s_ref).real.sum()
    loss_ref.backward()
    assert np.allclose(logabs.detach().cpu().numpy(), l_ref.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert fro_rel(At.grad.cpu().numpy(), Ac.grad.numpy()) <= 1e-10


@pytest.mark.parametrize("dt", ["f64", "c128"])
def test_slogpf_gradient_matches_appendix_and_fd(dt):
    L = lrugb()
    cplx = dt == "c128"
    g = np.random.Generator(np.random.PCG64(520))
    W, n = 4, 24
    M = _rand(g, (W, n, n), cplx)
    A = (M - M.transpose(0, 2, 1)) / np.sqrt(n)
    a = g.standard_normal(W)
    b = _rand(g, W, True)

    def loss_of(At):
        sign, logabs = L.slogpf(At)
        out = (tdev(a) * logabs).sum()
        if cplx:
            out = out + (torch.conj(tdev(b)) * sign).real.sum()
        return out, sign

    At = tdev(A).requires_grad_(True)
    loss, sign = loss_of(At)
    loss.backward()
    gA = At.grad.cpu().numpy()
    # the reference: log|pf| = (1/2) log|det| of the skew part, and the pf
    # phase moves by i s (1/2) d arg det (App. A.2 Eq. pf2=det), at this A
    s0 = sign.detach().cpu().numpy()
    Ac = torch.tensor(A, requires_grad=True)
    sd, ld = torch.linalg.slogdet(GO.skew(Ac))
    ref = (torch.tensor(a) * 0.5 * ld).sum()
    if cplx:
        theta = torch.angle(sd)
        dtheta = theta - theta.detach()
        ref = ref + (torch.conj(torch.tensor(b)) * torch.tensor(s0) * torch.exp(0.5j * dtheta)).real.sum()
    ref.backward()
    assert fro_rel(gA, Ac.grad.numpy()) <= 1e-10
    # App. A.3: d log pf / dA_ij = (1/2) (A^{-1})_ji, so for a = 1, b = 0 the
    # gradient of walker 0 is half the (conjugate) transposed inverse
    # central differences of the GPU forward along skew directions
    h = 1e-6
    for w in range(2):
        D = _rand(g, (n, n), cplx)
        D = D - D.T
        Dfull = np.zeros_like(A)
        Dfull[w] = D
        with torch.no_grad():
            lp, _ = loss_of(tdev(A + h * Dfull))
            lm, _ = loss_of(tdev(A - h * Dfull))
        fd = (lp.item() - lm.item()) / (2 * h)
        an = np.real(np.sum(np.conj(gA[w]) * D))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (w, fd, an)


def test_slogpf_gradient_is_half_the_transposed_inverse():
    # App. A.3 (Eq. pf_grad) directly: for real skew A, d log|pf A| / dA_ij =
    # (1/2) (A^{-1})_ji on the skew projection
    L = lrugb()
    g = np.random.Generator(np.random.PCG64(530))
    n = 30
    M = g.standard_normal((1, n, n))
    A = M - M.transpose(0, 2, 1)
    At = tdev(A).requires_grad_(True)
    _, logabs = L.slogpf(At)
    logabs.sum().backward()
    Ainv = np.linalg.inv(A[0])
    assert fro_rel(At.grad.cpu().numpy()[0], 0.5 * Ainv.T) <= 1e-10
