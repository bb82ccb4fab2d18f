"""FP64 automatic-differentiation reference for the log ratios.

TEST INFRASTRUCTURE ONLY (see lru_oracle.py): imported by tests/ only.

Plain PyTorch CPU autograd in float64 / complex128 on the definitions:
  det: log r = log det(A + U V) - log det(A)                    (Sec. 2.1)
  pf : log r = log pf(A_s + B C_s B^T) - log pf(A_s),  X_s = (X - X^T)/2,
       the skew projection App. A.3 applies before differentiating; for
       gradients log pf = (1/2) log det (App. A.2 Eq. pf2=det: the branch
       constant does not change the derivative).
Real dtypes use log|.|, complex dtypes the holomorphic log; torch returns
the conjugate-Wirtinger vector-Jacobian products.
"""
import torch


def _logdet(M):
    sign, logabs = torch.linalg.slogdet(M)
    if M.is_complex():
        return torch.log(sign) + logabs
    return logabs


def skew(M):
    return (M - M.transpose(-1, -2)) / 2


def det_log_ratio(A, U, V):
    return _logdet(A + U @ V) - _logdet(A)


def pf_log_ratio(A, B, C):
    As = skew(A)
    return 0.5 * (_logdet(As + B @ skew(C) @ B.transpose(-1, -2)) - _logdet(As))


def log_det(A):
    return _logdet(A)


def log_pf(A):
    return 0.5 * _logdet(skew(A))


def vjp(f, inputs, g):
    """Gradients of sum(g * f(inputs)) (torch's convention for complex g)."""
    ins = [x.detach().clone().requires_grad_(True) for x in inputs]
    out = f(*ins)
    grads = torch.autograd.grad(out, ins, grad_outputs=torch.as_tensor(g, dtype=out.dtype))
    return [gr.detach() for gr in grads]
