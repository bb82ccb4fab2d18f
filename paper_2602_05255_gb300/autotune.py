"""Autotuner for the delayed update: delay K, flush kernel and accept tile.

The paper leaves the delay bound T to the user ("typically T ~ n/10k" for
determinants, Sec. 2.3, and n/20k for Pfaffians, Sec. 3.3; Sec. 4.2 finds the
best T by experiment).  This module does that experiment on the GPU: for a
given (kind, n, k, dtype) it times short synthetic chains of one-hot row (det)
or row-and-column (pf) moves through the C-ABI with CUDA events, for

  * delay candidates around the paper's heuristic (and the plain form),
  * the flush kernels that keep FP64-class accuracy, each with its own tiling:
    FP64 tiles of 32 x 32 on the CUDA cores, the exact split product on the
    tensor cores (128 x 64 tiles of BF16 slices; F64, n % 128 == 0), and
    double-float tiles on the FP32 pipe (F64),
  * the GEMV arithmetic (FP64 or double-float, F64 rank-1),
  * accept-pass tiles (columns of A^{-1} per CTA work item) for the best of
    those,

and returns the fastest setting.  Reduced-precision flushes (TF32, BF16) are
left out unless asked for: they change the results, not just the speed.
Results are cached in a JSON file keyed by the device name.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Iterable, Optional

import torch

from . import lrugb as L

CACHE = os.environ.get("LRUGB_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "lrugb_autotune.json"))


def heuristic_delay(kind: str, n: int, k: int) -> int:
    """T ~ n / (10 k) (det) or n / (20 k) (pf), at least 2, T < n / k."""
    t = n / ((10 if kind == "det" else 20) * k)
    return int(max(2, min(round(t), max(2, n // k - 1))))


def candidates(kind: str, n: int, k: int, kmax_cols: int = 64) -> list:
    base = heuristic_delay(kind, n, k)
    cset = {base, max(2, base // 2), base * 2, 4, 8, 16, 32}
    kk = k if kind == "det" else 2 * k
    return sorted(c for c in cset if 2 <= c and c * kk <= kmax_cols)


def _time_chain(kind, n, k, dtype, delay, flush, arith, tile, walkers, steps, seed=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    cplx = dtype.is_complex
    rdt = torch.float64 if dtype in (torch.float64, torch.complex128) else torch.float32

    def rnd(*shape):
        x = torch.randn(*shape, generator=g, dtype=rdt)
        if cplx:
            x = torch.complex(x, torch.randn(*shape, generator=g, dtype=rdt))
        return x.to(dtype)

    A = rnd(walkers, n, n) / math.sqrt(n)
    eye = torch.eye(n, dtype=dtype)
    if kind == "det":
        A = A + 3 * eye
    else:
        J = torch.zeros(n, n, dtype=dtype)
        J[: n // 2, n // 2:] = torch.eye(n // 2, dtype=dtype)
        J[n // 2:, : n // 2] = -torch.eye(n // 2, dtype=dtype)
        A = (A - A.transpose(1, 2)) / 2 + 3 * J
    st = L.LowRankState(kind, walkers, n, k=k, dtype=dtype, delay=delay, flush=flush, arith=arith,
                        tile_chunks=tile)
    st.init(A.cuda().contiguous())
    kk = k if kind == "det" else 2 * k
    idx = torch.randint(0, n, (steps, walkers, kk), generator=g, dtype=torch.int32).cuda()
    dense = (rnd(steps, walkers, kk, n) * 0.1 / math.sqrt(n)).cuda()
    mask = 0 if kind == "pf" else (1 << kk) - 1
    if kind == "pf":
        mask = sum(1 << b for b in range(k, 2 * k))   # columns k..2k-1 one-hot, 0..k-1 dense

    def one(s):
        if kind == "det":
            st.propose_det(L.Operand(idx=idx[s], onehot_mask=mask), L.Operand(dense=dense[s]))
        else:
            st.propose_pf(L.Operand(dense=dense[s], idx=idx[s], onehot_mask=mask))
        st.accept()

    warm = min(3, steps // 4)
    for s in range(warm):
        one(s)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for s in range(warm, steps):
        one(s)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st.close()
    return walkers * (steps - warm) / (ms / 1e3)


def flush_candidates(kind: str, n: int, k: int, dtype) -> list:
    """Flush kernels that keep FP64-class results for this shape."""
    out = [L.FLUSH_NATIVE]
    if dtype == torch.float64:
        if n % 128 == 0 and 128 <= n <= 2048:
            out.append(L.FLUSH_SPLIT)
        out.append(L.FLUSH_DF)
    return out


def tune(kind: str, n: int, k: int, dtype=torch.float64, flushes: Optional[Iterable[int]] = None,
         ariths: Optional[Iterable[int]] = None, walkers: Optional[int] = None, steps: Optional[int] = None,
         delays: Optional[Iterable[int]] = None, tiles: Iterable[int] = (16, 32, 64, 128),
         include_plain: bool = True, use_cache: bool = True) -> Dict:
    """Best {delay, flush, arith, tile_chunks, updates_per_s} for the workload;
    every measured setting is kept under 'trials'.  delay 0 is the plain form
    (left out with include_plain=False)."""
    dev = torch.cuda.get_device_name()
    flushes = list(flushes) if flushes is not None else flush_candidates(kind, n, k, dtype)
    if ariths is None:
        ariths = [L.ARITH_NATIVE] + ([L.ARITH_DF] if dtype == torch.float64 else [])
    ariths = list(ariths)
    key = (f"{dev}|{kind}|n{n}|k{k}|{str(dtype)}|flush{','.join(map(str, flushes))}|"
           f"arith{','.join(map(str, ariths))}|plain{int(include_plain)}")
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except Exception:
            cache = {}
        if key in cache:
            return cache[key]
    walkers = walkers or max(8, min(1024, (1 << 31) // (n * n * 16)))
    delays = list(delays) if delays is not None else candidates(kind, n, k)
    steps_ = steps or max(2 * max(delays) + 4, 24)
    tiles = list(tiles)
    trials = []
    # delay x flush x arithmetic at the default accept tile, then the tiles of the best
    for arith in ariths:
        if include_plain:
            trials.append({"delay": 0, "flush": L.FLUSH_NATIVE, "arith": arith, "tile_chunks": 0,
                           "updates_per_s": _time_chain(kind, n, k, dtype, 0, L.FLUSH_NATIVE, arith, 0, walkers,
                                                        steps_)})
        for K in delays:
            for fl in flushes:
                try:
                    rate = _time_chain(kind, n, k, dtype, K, fl, arith, 0, walkers, steps_)
                except L.LRUError:
                    continue   # combination not built for this shape
                trials.append({"delay": K, "flush": fl, "arith": arith, "tile_chunks": 0, "updates_per_s": rate})
    best = max(trials, key=lambda d: d["updates_per_s"])
    for t in tiles:
        rate = _time_chain(kind, n, k, dtype, best["delay"], best["flush"], best["arith"], t, walkers, steps_)
        trials.append({"delay": best["delay"], "flush": best["flush"], "arith": best["arith"], "tile_chunks": t,
                       "updates_per_s": rate})
    best = max(trials, key=lambda d: d["updates_per_s"])
    res = dict(best)
    res["heuristic_delay"] = heuristic_delay(kind, n, k)
    res["trials"] = trials
    res["walkers"] = walkers
    if use_cache:
        cache[key] = res
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        json.dump(cache, open(CACHE, "w"), indent=1)
    return res


def make_state(kind: str, walkers: int, n: int, k: int = 1, dtype=torch.float64, tuned: Optional[Dict] = None,
               **kw) -> "L.LowRankState":
    """A LowRankState configured with a tune() result (delay, flush, GEMV
    arithmetic, accept tile); tuned=None runs tune() first."""
    tuned = tuned or tune(kind, n, k, dtype)
    return L.LowRankState(kind, walkers, n, k=k, dtype=dtype, delay=tuned["delay"], flush=tuned["flush"],
                          arith=tuned["arith"], tile_chunks=tuned["tile_chunks"], **kw)
