"""Shared helpers of the GPU parity tests: run a chain through the C-ABI and
replay the same seeded inputs on the CPU oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lru_oracle as O  # noqa: E402
from paper_2602_05255_gb300 import workloads  # noqa: E402

RTOL_F64 = 1e-10
# Ceiling of the conditioning-limited bar on chains over the paper's Slater
# and pairing matrices (N(0, 1/n) entries): their condition numbers reach
# ~1e6, where the oracle's own FP64 chain is up to 6e-9 away from the exact
# ratio (checked against 200-bit arithmetic), a bar of 6e-8.
CEIL_CHAIN = 1e-7


def lrugb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_05255_gb300 import lrugb as L
    return L


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


# One summary per check_ratios / check_inverse call, printed by the tests
# (pytest -s shows them): (what, steps, steps below the median ratio,
# conditioning-limited steps, largest bar used, largest GPU error against the
# oracle chain and against the exact ratio), or the inverse errors and bar.
PARITY_LOG = []


def exact_det_ratio(A, U, V):
    """det(A + U V) / det(A) = det(I + V A^{-1} U), with A^{-1} U from a fresh
    LAPACK solve of the current matrix (more accurate than a quotient of two
    slogdet values at ill-conditioned steps)."""
    A, U, V = (np.asarray(x) for x in (A, U, V))
    R = np.eye(U.shape[1], dtype=np.result_type(A, U, V)) + V @ np.linalg.solve(A, U)
    return np.linalg.det(R) if R.shape[0] > 1 else R[0, 0]


def exact_pf_ratio(A, B, C):
    """pf(A + B C B^T) / pf(A) = pf(C^{-1} + B^T A^{-1} B) / pf(C^{-1}) (App. A.2),
    with A^{-1} B from a fresh LAPACK solve of the current matrix and the
    2k x 2k Pfaffians from the oracle's pairing sum."""
    A, B, C = (np.asarray(x) for x in (A, B, C))
    Ci = np.linalg.inv(C)
    Ci = (Ci - Ci.T) / 2
    M = Ci + B.T @ np.linalg.solve(A, B)
    M = (M - M.T) / 2
    return O.pf_pairings(M) / O.pf_pairings(Ci)


def check_ratios(gpu, chain, exact, base=RTOL_F64, what="", eps_scale=1.0, refresh_every=0, ceiling=None,
                 alt=None):
    """Ratio parity against the oracle's chain and against the exact ratios.

    A ratio is 1 + v^T A^{-1} u (Eq. det_ratio) or the Pfaffian of the core
    C^{-1} + B^T A^{-1} B (Eq. pf_low_rank): a sum of terms of the size of a
    typical ratio.  A small ratio comes from cancellation among such terms,
    and its rounding error is that of the terms, so every error is measured on
    the scale max(|exact|, median |exact|): relative for ratios above the
    median, absolute in units of the median below it (a node of the wave
    function is the limit).  The bar is `base` (1e-10 in FP64), against both
    the chain and the exact ratio.  A chain of low-rank updates carries the
    rounding of every update since the last from-scratch refresh, amplified by
    the conditioning of the matrices it passed through, and the oracle's own
    FP64 chain measures that amount: e_run is its largest scaled error against
    the exact ratio since the last refresh (reset at every refresh).  One chain
    is one sample of that rounding: after a step whose core is nearly singular
    two FP64 chains that differ only in the order of their sums (another BLAS,
    the GPU) can sit a decade apart.  `alt` holds further oracle chains of the
    same moves in another mathematically equal form (plain and delayed); e_run
    then takes the largest error of all of them.  A step
    where 10 * eps_scale * e_run exceeds `base` is conditioning-limited, and its
    bar is 10 * eps_scale * e_run; eps_scale is the unit roundoff of the GPU
    arithmetic over FP64's (1 for FP64, 256 for the double-float paths).  The
    largest bar used must stay within `ceiling` (default 100 * eps_scale *
    base).  Returns the summary it appends to PARITY_LOG."""
    gpu, chain, exact = (np.asarray(x) for x in (gpu, chain, exact))
    refs = [chain] + [np.asarray(a) for a in (alt or [])]
    ceiling = 100.0 * eps_scale * base if ceiling is None else ceiling
    med = np.median(np.abs(exact))
    e_run = 0.0
    out = {"what": str(what), "steps": len(exact), "below_median": 0, "cond_limited": 0, "max_bar": base,
           "max_err_vs_chain": 0.0, "max_err_vs_exact": 0.0, "ceiling": ceiling}
    for s in range(len(exact)):
        if refresh_every and s % refresh_every == 0:
            e_run = 0.0
        sc = max(abs(exact[s]), med)
        out["below_median"] += int(abs(exact[s]) < med)
        e_run = max(e_run, max(abs(c[s] - exact[s]) for c in refs) / sc)
        bar = max(base, 10 * eps_scale * e_run)
        if bar > base:
            out["cond_limited"] += 1
        out["max_bar"] = max(out["max_bar"], bar)
        ec = abs(gpu[s] - chain[s]) / sc
        ee = abs(gpu[s] - exact[s]) / sc
        out["max_err_vs_chain"] = max(out["max_err_vs_chain"], ec)
        out["max_err_vs_exact"] = max(out["max_err_vs_exact"], ee)
        assert ec <= bar and ee <= bar, (what, s, gpu[s], chain[s], exact[s], bar)
    assert out["max_bar"] <= ceiling, (what, out)
    PARITY_LOG.append(out)
    print("parity:", out)
    return out


def check_inverse(gpu_inv, chain_inv, exact_inv, base=RTOL_F64, what="", eps_scale=1.0):
    """The carried inverse against the exact inverse of the current matrix
    (Frobenius-relative), on the same conditioning-limited bar as the ratios:
    max(base, 10 * eps_scale * the oracle chain's own inverse error)."""
    e_chain = fro_rel(chain_inv, exact_inv)
    bar = max(base, 10 * eps_scale * e_chain)
    e = fro_rel(gpu_inv, exact_inv)
    out = {"what": str(what), "inverse_err": e, "chain_inverse_err": e_chain, "bar": bar}
    assert e <= bar, out
    PARITY_LOG.append(out)
    print("parity:", out)
    return out


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
