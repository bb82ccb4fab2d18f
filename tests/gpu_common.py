"""Shared helpers of the GPU parity tests: run a chain through the C-ABI and
replay the same seeded inputs on the CPU oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lru_oracle as O  # noqa: E402
from paper_2602_05255_gb300 import workloads  # noqa: E402

RTOL_F64 = 1e-10


def lrugb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_05255_gb300 import lrugb as L
    return L


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def check_ratios(gpu, chain, exact, base=RTOL_F64, what="", eps_scale=1.0):
    """Ratio parity with a condition-aware bound.

    A step compares GPU and oracle-chain ratios with relative tolerance
    max(base, 10 * eps_scale * e) where e is the largest |r_chain - r_exact| /
    |r_exact| so far: the oracle chain's own accumulated FP64 rounding error
    against the from-scratch ratios (large after near-node steps); eps_scale is the unit roundoff of the GPU
    arithmetic over FP64's (256 for the double-float paths).  Near-node
    steps (|r_exact| < 1e-6 median |r|) compare absolute errors against
    base * median |r|."""
    gpu, chain, exact = (np.asarray(x) for x in (gpu, chain, exact))
    med = np.median(np.abs(exact))
    e_run = 0.0   # rounding errors accumulate along a chain: the running maximum sets the scale
    for s in range(len(exact)):
        if abs(exact[s]) < 1e-6 * med:
            assert abs(gpu[s] - chain[s]) <= base * med, (what, s, gpu[s], chain[s], exact[s])
            continue
        e_run = max(e_run, abs(chain[s] - exact[s]) / abs(exact[s]))
        tol = max(base, 10 * eps_scale * e_run)
        assert abs(gpu[s] - chain[s]) <= tol * abs(chain[s]), (what, s, gpu[s], chain[s], exact[s], tol)


def fro_rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def tdev(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def det_workload(seed, W, n, m, steps, cplx=False, var=None, first_rows=False):
    var = 1.0 / n if var is None else var
    Phi = workloads.orbital_matrix(seed, m, n, var, cplx)
    occ0 = workloads.initial_occupation(seed + 1, W, m, n, first_rows=first_rows)
    slot, new = workloads.move_sequence(seed + 2, occ0, m, steps)
    return Phi, occ0, slot, new


def pf_workload(seed, W, n, m, steps, cplx=False):
    G = workloads.pairing_generator(seed, m, 1.0 / n, cplx)
    F = G - G.T
    pos0 = workloads.initial_occupation(seed + 1, W, m, n)
    slot, new = workloads.move_sequence(seed + 2, pos0, m, steps)
    return F, pos0, slot, new


def run_det_chain_gpu(L, Phi, occ0, slot, new, delay=0, flush=0, refresh_every=0, mask_seq=None, dtype=None,
                      arith=0):
    W, n = occ0.shape
    dtype = dtype or (torch.complex128 if np.iscomplexobj(Phi) else torch.float64)
    st = L.LowRankState("det", W, n, k=1, dtype=dtype, delay=delay, flush=flush, arith=arith)
    Phi_d = tdev(Phi, dtype)
    occ_d = tdev(occ0)
    A0 = torch.stack([Phi_d[occ_d[w].long()] for w in range(W)]).contiguous()
    st.init(A0)
    slot_d, new_d = tdev(slot), tdev(new)
    ratios, statuses = [], []
    for s in range(slot.shape[0]):
        V, idx = st.form_row_moves(Phi_d, occ_d, slot_d[s], new_d[s])
        r, status = st.propose_det(L.Operand(idx=idx, onehot_mask=1), L.Operand(dense=V))
        mask = None if mask_seq is None else tdev(mask_seq[s].astype(np.uint8))
        st.accept(mask)
        st.commit_moves(occ_d, slot_d[s], new_d[s], mask)
        ratios.append(r.cpu().numpy())
        statuses.append(status.cpu().numpy())
        if refresh_every and (s + 1) % refresh_every == 0:
            A = torch.stack([Phi_d[occ_d[w].long()] for w in range(W)]).contiguous()
            st.refresh(A)
    torch.cuda.synchronize()
    return st, np.array(ratios), np.array(statuses), occ_d.cpu().numpy()


def replay_det_oracle(Phi, occ0, slot, new, w, delay=0, mask_seq=None):
    occ = occ0[w].copy()
    A = O.slater_matrix(Phi, occ)
    if delay >= 2:
        car = O.init_det_carrier(A, delay)
    else:
        Ainv = O.inv(A)
    rs, ex = [], []
    for s in range(slot.shape[0]):
        U, V = O.det_row_move(Phi, occ, slot[s, w], new[s, w])
        ex.append(O.det_ratio_direct(O.slater_matrix(Phi, occ), U, V))
        acc = True if mask_seq is None else bool(mask_seq[s, w])
        if delay >= 2:
            r = O.det_lru_delayed(car, U, V, accept=acc)
        else:
            if acc:
                r, Ainv = O.det_lru(Ainv, U, V, return_update=True)
            else:
                r = O.det_lru(Ainv, U, V)
        if acc:
            occ[slot[s, w]] = new[s, w]
        rs.append(r)
    inv_now = O.carrier_inverse(car) if delay >= 2 else Ainv
    return np.array(rs), inv_now, occ, np.array(ex)
