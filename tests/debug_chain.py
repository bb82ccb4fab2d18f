"""Small determinant and Pfaffian chains through the debug build of the
library (LRUGB_DEBUG=1: device-side index checks, canary-guarded handle
allocations), against the oracle.  Run by test_gpu_debug_build.py in a child
process; prints "debug chains ok" on success."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import lru_oracle as O  # noqa: E402
from paper_2602_05255_gb300 import lrugb as L, workloads  # noqa: E402


def rel(a, b):
    return abs(a - b) / abs(b)


def det_chain(delay):
    W, n, m, steps = 3, 64, 128, 20
    Phi = workloads.orbital_matrix(301, m, n, 1.0 / n)
    occ0 = workloads.initial_occupation(302, W, m, n)
    slot, new = workloads.move_sequence(303, occ0, m, steps)
    st = L.LowRankState("det", W, n, k=1, dtype=torch.float64, delay=delay)
    Phi_d, occ_d = torch.tensor(Phi).cuda(), torch.tensor(occ0).cuda()
    st.init(st.gather_rows(Phi_d, occ_d))
    rs = []
    for s in range(steps):
        V, idx = st.form_row_moves(Phi_d, occ_d, torch.tensor(slot[s]).cuda(), torch.tensor(new[s]).cuda())
        r, _ = st.propose_det(L.Operand(idx=idx, onehot_mask=1), L.Operand(dense=V))
        st.accept()
        st.commit_moves(occ_d, torch.tensor(slot[s]).cuda(), torch.tensor(new[s]).cuda())
        rs.append(r.cpu().numpy())
    st.check_device_error()
    for w in range(W):
        occ = occ0[w].copy()
        Ainv = O.inv(O.slater_matrix(Phi, occ))
        for s in range(steps):
            U, V = O.det_row_move(Phi, occ, slot[s, w], new[s, w])
            r, Ainv = O.det_lru(Ainv, U, V, return_update=True)
            occ[slot[s, w]] = new[s, w]
            assert rel(rs[s][w], r) <= 1e-9, ("det", delay, w, s)


def pf_chain(delay):
    W, n, m, steps = 3, 32, 80, 20
    G = workloads.pairing_generator(311, m, 1.0 / n)
    F = G - G.T
    pos0 = workloads.initial_occupation(312, W, m, n)
    slot, new = workloads.move_sequence(313, pos0, m, steps)
    st = L.LowRankState("pf", W, n, k=1, dtype=torch.float64, delay=delay)
    F_d, pos_d = torch.tensor(F).cuda(), torch.tensor(pos0).cuda()
    st.init(st.gather_pairs(F_d, pos_d))
    rs = []
    for s in range(steps):
        B, idx = st.form_pf_moves(F_d, pos_d, torch.tensor(slot[s]).cuda(), torch.tensor(new[s]).cuda())
        r, _ = st.propose_pf(L.Operand(dense=B, idx=idx, onehot_mask=0b10))
        st.accept()
        st.commit_moves(pos_d, torch.tensor(slot[s]).cuda(), torch.tensor(new[s]).cuda())
        rs.append(r.cpu().numpy())
    st.check_device_error()
    for w in range(W):
        pos = pos0[w].copy()
        Ainv = O.skew_part(O.inv(O.pairing_matrix(F, pos)))
        for s in range(steps):
            B, C = O.pf_row_col_move(F, pos, slot[s, w], new[s, w])
            r, Ainv = O.pf_lru(Ainv, B, C, return_update=True)
            pos[slot[s, w]] = new[s, w]
            assert rel(rs[s][w], r) <= 1e-9, ("pf", delay, w, s)


def ragged_step():
    # the persistent step of a delayed ragged handle, against the oracle
    W, K = 4, 3
    n_w, k_w = [16, 32, 48, 16], [1, 2, 1, 2]
    g = np.random.Generator(np.random.PCG64(321))
    A = [g.standard_normal((n, n)) / np.sqrt(n) + 2.5 * np.eye(n) for n in n_w]
    st = L.LowRankState("det", W, n_w, k=2, dtype=torch.float64, delay=K, k_per_walker=k_w)
    st.init(torch.tensor(np.concatenate([a.reshape(-1) for a in A])).cuda())
    cars = [O.init_det_carrier(a, K) for a in A]
    for s in range(5):
        U = [g.standard_normal((k, n)) * 0.2 / np.sqrt(n) for n, k in zip(n_w, k_w)]
        V = [g.standard_normal((k, n)) * 0.2 / np.sqrt(n) for n, k in zip(n_w, k_w)]
        flat = lambda vs: np.concatenate([np.concatenate([v.reshape(-1), np.zeros((2 - v.shape[0]) * v.shape[1])])
                                          for v in vs])
        r, status, acc = st.step_persistent(L.Operand(dense=torch.tensor(flat(U)).cuda()),
                                            L.Operand(dense=torch.tensor(flat(V)).cuda()), accept=True)
        r = r.cpu().numpy()
        for w in range(W):
            ref = O.det_lru_delayed(cars[w], U[w].T, V[w])
            assert rel(r[w], ref) <= 1e-9, ("ragged", w, s)
    st.check_device_error()


if __name__ == "__main__":
    assert L.DEBUG and b"debug" in L._lib.lru_version(), L._lib.lru_version()
    for d in (0, 4):
        det_chain(d)
        pf_chain(d)
    ragged_step()
    print("debug chains ok:", L.version())
