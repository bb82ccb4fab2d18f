"""The N > 1 path on CPU: two gloo ranks, one walker shard each.

Walkers are independent chains, so a rank's results must equal those of a
single process that runs the same shard (no data crosses ranks); the only
collectives are the barrier and the MAX of the per-rank times, and the
whole-job rate counts every rank's walkers.  Each rank advances its shard
with the oracle's rank-1 chain (Eq. det_inv), standing in for the GPU step.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2602_05255_gb300 import multigpu, workloads  # noqa: E402

SEED, W, N, M, STEPS = 6, 3, 8, 16, 5


def shard_chain(rank):
    """Ratios of one rank's walker shard: plain oracle chain, inverse updated every step."""
    from oracle import lru_oracle as O
    seed = multigpu.shard_seed(SEED, rank)
    Phi = workloads.orbital_matrix(seed, M, N, 1.0 / N)
    occ0 = workloads.initial_occupation(seed + 1, W, M, N)
    slot, new = workloads.move_sequence(seed + 2, occ0, M, STEPS)
    out = np.zeros((STEPS, W))
    for w in range(W):
        occ = occ0[w].copy()
        Ainv = O.inv(O.slater_matrix(Phi, occ))
        for s in range(STEPS):
            U, V = O.det_row_move(Phi, occ, slot[s, w], new[s, w])
            out[s, w], Ainv = O.det_lru(Ainv, U, V, return_update=True)
            occ[slot[s, w]] = new[s, w]
    return occ0, out


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, wsz, local = multigpu.rank_env()
    assert (r, wsz, local) == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    occ0, ratios = shard_chain(rank)
    ms = 10.0 + 5.0 * rank                     # stand-in per-rank elapsed time
    ms_max = multigpu.max_over_ranks(ms, dist, "cpu")
    rate = multigpu.whole_job_rate(W * STEPS, world, ms_max)
    dist.barrier()
    np.savez(os.path.join(outdir, f"rank{rank}.npz"), occ0=occ0, ratios=ratios, ms_max=ms_max, rate=rate)
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks_shard_walkers(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    # max over ranks reaches every rank; the rate counts all ranks' walker-updates
    for d in res:
        assert float(d["ms_max"]) == 15.0
        assert float(d["rate"]) == pytest.approx(world * W * STEPS / 15e-3)
    # the shards differ, and each equals a single-process run of the same shard
    assert not np.array_equal(res[0]["occ0"], res[1]["occ0"])
    for r in range(world):
        occ0, ratios = shard_chain(r)
        assert np.array_equal(res[r]["occ0"], occ0)
        assert np.array_equal(res[r]["ratios"], ratios)


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert multigpu.rank_env() == (0, 1, 0)
    assert multigpu.shard_seed(SEED, 0) == SEED
    assert multigpu.max_over_ranks(3.5) == 3.5
    assert multigpu.whole_job_rate(100, 1, 50.0) == pytest.approx(2000.0)
