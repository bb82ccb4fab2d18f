#!/usr/bin/env python
"""Throughput of batched low-rank determinant and Pfaffian updates on GB300.

Default workload (the headline; the paper's delayed-update study, Sec. 4.2,
at n = 1024): W = 1024 walkers, each a Slater matrix A = Phi[occ] with Phi
2048 x 1024 N(0, 1/n) (FP64, seeded), rank-1 row replacements (one-hot
U = e_i, dense V = Phi[new] - Phi[old]) accepted every step, and a
from-scratch FP64 refresh of every walker after every 128th step.  One step =
operand formation + propose + accept (+ flush) for all walkers.  Metric:
walker-updates/s of the delayed form (double-float GEMV, flush as an exact
split product on the tensor cores, delay K from the autotuner; the "delayed"
arm) next to the plain FP64 form, with further arms.  The line's roofline is
that of the kernel class with the most time.  The same line carries the
Pfaffian workload's arms (c3, below) under "pf_workload" and, last, a short
"delayed_vs_plain" summary of both.

--config selects another workload of the paper's configurations:
  c1  1 walker, n = 64, Phi 128 x 64 N(0, 1), rank-1 row swaps (latency)
  c2  4096 walkers, n = 512, Phi 1024 x 512 N(0, 1/n), K = 16, refresh every
      128 (--dtype f64 | c128)
  c3  Pfaffian: 1024 walkers, n = 256 on 512 sites, F = G - G^T, rank-2
      row-and-column moves, K = 8, no refresh (--dtype f64 | c128)
  c4  precision form: 64 walkers, n = 2048, two-electron moves (k = 2),
      K = 32, refresh every 64; tensor-core flushes against the FP64 chain
  c5  2048 walkers of uneven n in {128, 256, 512, 1024} and rank k in
      {1, 2, 4, 8}, dense U, V, delayed (K = 4), one persistent launch per
      step replayed from a CUDA graph, and the adjoint (--dtype c128 | c64)

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config ...]
Under torchrun every rank runs its own walkers (weak scaling); rank 0 prints
one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2602_05255_gb300 import multigpu  # noqa: E402

METRIC = "walker-updates/sec at n=1024 (delayed vs plain rank-1, same GPU); roofline fraction"
PF_METRIC = "walker-updates/sec, Pfaffian rank-2 row-and-column moves (delayed vs plain, same GPU); roofline fraction"
RAGGED_METRIC = "walker-updates/sec, walkers of uneven n and rank k in one persistent graph-captured launch"
# profiling classes of the library (lru_profile_read), in order
PROF_CLASSES = ["propose", "accept", "flush", "refresh", "refresh_panel", "refresh_update"]

# the workloads: kind, walkers, n, sites m, rank k, delay K ("tune": from the
# autotuner), refresh period, dtype, arms and the arm the line reports
PRESETS = {
    "headline": {"kind": "det", "walkers": 1024, "n": 1024, "m": 2048, "k": 1, "delay": "tune",
                 "refresh_every": 128, "dtype": "f64", "var": None, "first_rows": False,
                 "arms": "plain,delayed,delayed_fp64gemv,delayed_dfflush,delayed_tf32x3", "main": "delayed"},
    "c1": {"kind": "det", "walkers": 1, "n": 64, "m": 128, "k": 1, "delay": 0, "refresh_every": 0, "dtype": "f64",
           "var": 1.0, "first_rows": True, "arms": "plain", "main": "plain"},
    "c2": {"kind": "det", "walkers": 4096, "n": 512, "m": 1024, "k": 1, "delay": 16, "refresh_every": 128,
           "dtype": "f64", "var": None, "first_rows": False, "arms": "plain,delayed,delayed_fp64gemv",
           "main": "delayed"},
    "c3": {"kind": "pf", "walkers": 1024, "n": 256, "m": 512, "k": 1, "delay": 8, "refresh_every": 0,
           "dtype": "f64", "arms": "plain,plain_dfprop,delayed_dfpass,delayed,delayed_native,delayed_dfflush", "main": "delayed_dfpass"},
    "c4": {"kind": "det", "walkers": 64, "n": 2048, "m": 4096, "k": 2, "delay": 32, "refresh_every": 64,
           "dtype": "f64", "var": None, "first_rows": False,
           "arms": "plain,delayed_fp64gemv,delayed_tf32x3,delayed_bf16x3,delayed_tf32,delayed_bf16",
           "main": "delayed_fp64gemv"},
    "c5": {"kind": "ragged", "walkers": 2048, "ns": (128, 256, 512, 1024), "ks": (1, 2, 4, 8), "delay": 4,
           "dtype": "c128", "refresh_every": 0},
    # Sec. 4.1 Fig. 1 on GB300 (context): direct batched slogdet / slogpf of the
    # updated matrices against the LRU ratio, without and with the inverse update
    "fig1": {"kind": "fig1", "walkers": 1024, "ns": (16, 32, 64, 128, 256, 512, 1024), "dtype": "f64",
             "refresh_every": 0, "delay": 0},
}
FIG1_METRIC = ("speedup at n=1024 of the LRU ratio with the inverse update over the batched direct determinant, "
               "1024 walkers, k=1 (Sec. 4.1 Fig. 1 on GB300)")
# complex dtypes: the arms that apply (FP64-class arithmetic on complex scalars)
COMPLEX_ARMS = {"det": ("plain,delayed_native", "delayed_native"), "pf": ("plain,delayed_native", "delayed_native")}

FLUSH = {"native": 0, "tf32x3": 1, "tf32": 2, "bf16": 3, "bf16x3": 4, "df": 5, "split": 6}
ARITH = {"native": 0, "df": 1}
# determinant arms: name -> (delay: None = the workload's K, GEMV arithmetic, flush)
ARMS = {
    "plain": (0, "native", "native"),               # FP64 Sherman-Morrison-Woodbury step (Eq. det_inv)
    "delayed": (None, "df", "split"),               # double-float GEMV, exact split-product tensor-core flush
    "delayed_fp64gemv": (None, "native", "split"),  # FP64 GEMV, split-product flush
    "delayed_dfflush": (None, "native", "df"),      # FP64 GEMV, double-float flush (FP32 pipe)
    "delayed_native": (None, "native", "native"),   # dtype arithmetic everywhere (FP64 / complex128 flush)
    "delayed_tf32x3": (None, "native", "tf32x3"),   # tensor-core flushes of the precision form
    "delayed_bf16x3": (None, "native", "bf16x3"),
    "delayed_tf32": (None, "native", "tf32"),
    "delayed_bf16": (None, "native", "bf16"),
}
# Pfaffian arms: name -> (delay, arithmetic of the propose's pass over A^{-1}, flush)
PF_ARMS = {
    "plain": (0, "native", "native"),               # exactly skew rank-2 accept (Eq. pf_inv)
    "delayed": (None, "native", "split"),           # split-product flush, lower triangle mirrored (Eq. pf_delayed_Ainv)
    "delayed_native": (None, "native", "native"),   # FP64 skew flush
    "delayed_dfflush": (None, "native", "df"),      # double-float skew flush
    "delayed_df": (None, "df", "df"),               # double-float pass and flush
    "delayed_dfpass": (None, "df", "split"),        # double-float pass, split-product flush
    "plain_dfprop": (0, "df", "native"),
}

# FP64 pipe: 152 SMs x 2 DFMA / clk x 2 flop x 2.07 GHz (the 1.25 TFLOP/s of
# the GB300 datasheet); a DFMA probe measured 1.06 TFLOP/s at 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_SRC = "derived FP64 peak: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz"
# FP32 pipe (single-precision dtypes): 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP32_SRC = "derived FP32 peak: 152 SMs x 128 FFMA/clk x 2 x 2.07 GHz"
# DRAM bytes per walker of one launch of the double-float delayed accept
# (k_accept_delayed_warp_df) at n = 1024, from an ncu capture at 64 walkers:
# one pass over each walker's A_0^{-1}, so a full launch is this times W.
ACCEPT_DF_TRAFFIC_PER_WALKER_N1024 = (548.643328e6 + 4.782592e6) / 64


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=256)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default="headline", choices=list(PRESETS))
    p.add_argument("--workload", default=None, choices=["det", "pf"], help="pf: same as --config c3")
    p.add_argument("--dtype", default=None, choices=["f64", "c128", "c64"])
    p.add_argument("--walkers", type=int, default=None)
    p.add_argument("--n", type=int, default=None)
    p.add_argument("--m", type=int, default=None)
    p.add_argument("--delay", type=int, default=None)
    p.add_argument("--refresh-every", type=int, default=None, help="0: no refresh")
    p.add_argument("--arms", default=None)
    p.add_argument("--no-tune", action="store_true", help="headline: K = 16 instead of the autotuner's")
    p.add_argument("--no-pf", action="store_true", help="headline: leave out the Pfaffian arms")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--seed", type=int, default=6)
    a = p.parse_args(argv)
    if a.workload == "pf":
        a.config = "c3"
    cfg = dict(PRESETS[a.config])
    if a.dtype:
        cfg["dtype"] = a.dtype
    if cfg["kind"] in COMPLEX_ARMS and cfg["dtype"] != "f64":
        cfg["arms"], cfg["main"] = COMPLEX_ARMS[cfg["kind"]]
    for key in ("walkers", "n", "m", "delay", "refresh_every", "arms"):
        v = getattr(a, key)
        if v is not None:
            cfg[key] = v
    if a.no_tune and cfg.get("delay") == "tune":
        cfg["delay"] = 16
    a.cfg = cfg
    return a


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1700.0, "fallback"


def host_threads():
    """Threads the oracle's BLAS/LAPACK calls use on the host cores."""
    try:
        import threadpoolctl
        return int(max(i.get("num_threads", 1) for i in threadpoolctl.threadpool_info()) or 1)
    except Exception:
        return int(os.cpu_count() or 1)


# --------------------------------------------------------------------------
# inputs (seeded, synthetic; numpy PCG64, the same arrays the oracle gets)
# --------------------------------------------------------------------------
def det_inputs(cfg, seed, steps):
    from paper_2602_05255_gb300 import workloads
    W, n, m, k = cfg["walkers"], cfg["n"], cfg["m"], cfg["k"]
    var = 1.0 / n if cfg.get("var") is None else cfg["var"]
    Phi = workloads.orbital_matrix(seed, m, n, var, cfg["dtype"] != "f64")
    occ0 = workloads.initial_occupation(seed + 1, W, m, n, first_rows=cfg.get("first_rows", False))
    if k == 1:
        slot, new = workloads.move_sequence(seed + 2, occ0, m, steps)
    else:
        slot, new = workloads.multi_move_sequence(seed + 2, occ0, m, steps, k)
    return Phi, occ0, slot, new


def pf_inputs(cfg, seed, steps):
    """F = G - G^T (G m x m, N(0, 1/n)), initial positions and the move sequence."""
    from paper_2602_05255_gb300 import workloads
    G = workloads.pairing_generator(seed, cfg["m"], 1.0 / cfg["n"], cfg["dtype"] != "f64")
    F = G - G.T
    pos0 = workloads.initial_occupation(seed + 1, cfg["walkers"], cfg["m"], cfg["n"])
    slot, new = workloads.move_sequence(seed + 2, pos0, cfg["m"], steps)
    return F, pos0, slot, new


def ragged_shapes(cfg, seed):
    from paper_2602_05255_gb300 import workloads
    g = workloads.rng(seed)
    n_w = g.choice(cfg["ns"], cfg["walkers"])
    k_w = g.choice(cfg["ks"], cfg["walkers"])
    return n_w, k_w


def state_bytes(cfg):
    """Bytes of the walkers' A^{-1} state (what every timed pass streams)."""
    if cfg["kind"] == "fig1":
        return cfg["walkers"] * max(cfg["ns"]) ** 2 * scalar_bytes(cfg)
    if cfg["kind"] == "ragged":
        mean_n2 = float(np.mean(np.asarray(cfg["ns"], dtype=np.float64) ** 2))
        return cfg["walkers"] * mean_n2 * scalar_bytes(cfg)
    return cfg["walkers"] * cfg["n"] ** 2 * scalar_bytes(cfg)


def config_of(preset, cfg):
    """The line's config, the same for our arm and the reference arm."""
    K = cfg.get("delay")
    out = {"workload": workload_name(cfg, "autotuned" if K == "tune" else K), "preset": preset,
           "l2": f"inputs larger than L2 (A^-1 state about {state_bytes(cfg) / 2 ** 30:.2f} GiB per GPU)"}
    if cfg.get("refresh_every"):
        out["refresh_timing"] = ("refreshes due inside the timed steps are timed there; the share of a refresh that "
                                 "the steps do not reach (steps/period - floor(steps/period)) is one refresh timed "
                                 "right after the region, scaled by that share")
    return out


def workload_name(cfg, K):
    d = cfg["dtype"].upper()
    if cfg["kind"] == "fig1":
        return (f"det and pf, W={cfg['walkers']} walkers/GPU, n in {list(cfg['ns'])}, rank-1 row moves / row+column "
                f"moves, {d}: direct batched slogdet / slogpf vs LRU ratio vs LRU ratio + inverse update")
    if cfg["kind"] == "det":
        mv = "rank-1 row moves" if cfg["k"] == 1 else f"{cfg['k']}-electron row moves (k={cfg['k']})"
        var = "N(0,1)" if cfg.get("var") else "N(0,1/n)"
        return (f"det {mv}, W={cfg['walkers']} walkers/GPU, n={cfg['n']}, Phi {cfg['m']}x{cfg['n']} {var} {d}, "
                f"K={K}, " + (f"refresh every {cfg['refresh_every']}" if cfg["refresh_every"] else "no refresh"))
    if cfg["kind"] == "pf":
        return (f"pf rank-2 row+column moves, W={cfg['walkers']} walkers/GPU, n={cfg['n']} on {cfg['m']} sites, "
                f"F = G - G^T with G N(0,1/n) {d}, K={K}, "
                + (f"refresh every {cfg['refresh_every']}" if cfg["refresh_every"] else "no refresh"))
    return (f"ragged det, W={cfg['walkers']} walkers/GPU, n in {list(cfg['ns'])}, k in {list(cfg['ks'])}, "
            f"dense backflow-style U, V N(0,1/n) {d}, delayed K={K}, one persistent launch per step (CUDA graph)")


def torch_dtype(torch, cfg):
    return {"f64": torch.float64, "c128": torch.complex128, "c64": torch.complex64}[cfg["dtype"]]


def scalar_bytes(cfg):
    return {"f64": 8, "c128": 16, "c64": 8}[cfg["dtype"]]


def flop_factor(cfg):
    """Real flops per multiply-add of the dtype over a real one (complex: 4)."""
    return 4 if cfg["dtype"] != "f64" else 1


# --------------------------------------------------------------------------
# timing
# --------------------------------------------------------------------------
def refresh_share(steps, every):
    """The part of one refresh that `steps` steps owe the schedule beyond the
    refreshes due inside them: steps/every - floor(steps/every) (0 without a
    refresh period)."""
    return (steps / every - steps // every) if every else 0.0


def timed_steps(torch, st, step, args, dist, dev, refresh=None, every=0):
    """W warm-up steps, then K steps between CUDA events on the launching
    stream (barrier + synchronize on both sides, clocks sampled meanwhile,
    max over ranks); the library's per-class kernel timers run over the same
    region.  With a refresh period `every` that the K steps do not fill
    (K = 20 with a refresh every 128 steps holds no refresh), one refresh of
    every walker (`refresh()`) is timed right after the region, and its share
    K / every - floor(K / every) is added to the time, so the rate carries the
    schedule's refresh cost; the region-only time is returned as well."""
    for s in range(args.warmup):
        step(s, None)
    torch.cuda.synchronize()
    for c in range(len(PROF_CLASSES)):
        st.profile_read(c)
    st.profile(True)
    launches0 = st.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.steps):
        step(args.warmup + i, i)
    e1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = st.launch_count() - launches0
    prof = {name: st.profile_read(c) for c, name in enumerate(PROF_CLASSES)}
    st.profile(False)
    ms = multigpu.max_over_ranks(ms, dist, "cuda")
    amort = None
    frac = refresh_share(args.steps, every) if refresh else 0.0
    if frac > 0:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        r0.record()
        refresh()
        r1.record()
        torch.cuda.synchronize()
        rms = multigpu.max_over_ranks(r0.elapsed_time(r1), dist, "cuda")
        amort = {"refresh_ms": rms, "share": frac, "added_ms": frac * rms, "region_ms": ms,
                 "how": "one refresh of every walker timed after the region (CUDA events), times "
                        "steps/refresh_every - floor(steps/refresh_every)"}
        ms = ms + frac * rms
    return ms, clk, launches, prof, amort


# --------------------------------------------------------------------------
# rooflines (algorithmic bytes and flops per launch; DESIGN tables)
# --------------------------------------------------------------------------
def bound_of(byt, fp64_flop, ms, hbm, fp32=False):
    """Roofline of one launch: HBM bytes against the FP64 pipe (fp32: the
    flops are single precision, against the FP32 pipe), whichever takes longer
    at its peak binds; achieved and frac are against that bound."""
    if not ms:
        return None
    peak, src = (FP32_PEAK_TFLOPS, FP32_SRC) if fp32 else (FP64_PEAK_TFLOPS, FP64_SRC)
    t_hbm, t_fp64 = byt / (hbm * 1e9), fp64_flop / (peak * 1e12)
    out = {"bytes_per_launch": byt, "fp64_flop_per_launch": fp64_flop, "ms_per_launch": ms, "traffic": None,
           "hbm": {"achieved": byt / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s"},
           "time_at_hbm_peak_ms": t_hbm * 1e3, "time_at_fp64_peak_ms": t_fp64 * 1e3}
    out["hbm"]["frac"] = out["hbm"]["achieved"] / hbm
    if fp64_flop and t_fp64 > t_hbm:
        ach = fp64_flop / (ms / 1e3) / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "peak_source": src})
    else:
        out.update({"bound": "hbm", "achieved": out["hbm"]["achieved"], "peak": hbm, "unit": "GB/s",
                    "frac": out["hbm"]["frac"], "peak_source": "HBM of measured (MEASURED_PEAKS.json hbm_gbs)"})
    return out


def accept_roofline(delay, arith, n, W, ms, hbm, pf=False, k=1, s=8, cf=1):
    """Roofline of one accept launch (one walker-update of every walker).

    Algorithmic bytes: plain reads and writes A^{-1} (2 n^2 s per walker);
    delayed reads A_0^{-1} once (n^2 s).  FP64 work of the native GEMV: plain
    n^2 k FMA for y = V A^{-1} plus n^2 k for the rank-k update, delayed n^2 k
    FMA (complex: 4 real FMAs each).  The bound is whichever takes longer at
    its peak (HBM copy bandwidth, FP64 pipe); the double-float GEMV runs on
    the FP32 pipe and is reported against HBM.  Pfaffian row-and-column move
    (B = [x, e_i]), plain form: the exactly skew update A^{-1} + X M^{-1} X^T
    reads the upper triangle and writes both (1.5 n^2 s) with 2 FMA per upper
    element (2 n^2 flop); the delayed Pfaffian accept makes no pass over
    A^{-1}: its GEMV is in the propose, pf_propose_roofline.
    """
    bytes_per = (2 if delay < 2 else 1) * n * n * s * W
    if pf and delay < 2:
        bytes_per = 1.5 * n * n * s * W
    if pf:
        flop_per = 2 * n * n * W * cf
    else:
        flop_per = (4 if delay < 2 else 2) * n * n * k * W * cf
    # FP64-pipe share of the products: all (native), none (double-float)
    fp64_flop = flop_per if arith == "native" else 0.0
    out = bound_of(bytes_per, fp64_flop, ms, hbm)
    if out is None:
        return None
    out["traffic"] = ACCEPT_DF_TRAFFIC_PER_WALKER_N1024 * W if (
        not pf and delay >= 2 and arith == "df" and n == 1024 and k == 1 and s == 8) else None
    return out


def refresh_roofline(prof, n, W, bf16_sustained):
    """Rooflines of the refresh.  Tensor-core form (panel / update classes
    timed): a panel's work is n * 64^2 FMA, 2 * 64 n^2 flop per walker per
    refresh, done as FP64 eliminations of 16-column sub-panels plus their
    K = 16 split-product updates of the other panel columns; it is reported
    as FP64-equivalent throughput against the FP64 pipe.  The full-width
    split-product updates execute 39 BF16 MMA products of n x n x 64 per panel,
    78 n^3 flop per walker, on the tensor pipe (FP64-equivalent work
    2 n^2 (n - 64) flop).  The FP64 Gauss-Jordan form does n^3 FMA = 2 n^3 flop
    per walker."""
    ms, cnt = prof["refresh"]
    if not cnt:
        return None
    per = ms / cnt
    pms, pcnt = prof.get("refresh_panel", (0.0, 0))
    ums, ucnt = prof.get("refresh_update", (0.0, 0))
    if pcnt and ucnt:
        p_ms, u_ms = pms / cnt, ums / cnt          # per refresh
        p_flop = 2.0 * 64 * n * n * W
        u_flop = 78.0 * n ** 3 * W
        u_eq = 2.0 * n * n * (n - 64) * W
        panel = {"kernel": "refresh panels (FP64 sub-panel eliminations + split-product inner updates; "
                           "FP64-equivalent)", "bound": "alu", "unit": "TFLOP/s",
                 "achieved": p_flop / (p_ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                 "frac": p_flop / (p_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS, "traffic": None,
                 "flop_per_refresh": p_flop, "ms_per_refresh": p_ms, "peak_source": FP64_SRC}
        update = {"kernel": "refresh trailing updates (BF16 split products on tcgen05)", "bound": "tensor",
                  "unit": "TFLOP/s", "achieved": u_flop / (u_ms / 1e3) / 1e12, "peak": bf16_sustained,
                  "frac": u_flop / (u_ms / 1e3) / 1e12 / bf16_sustained, "traffic": None,
                  "flop_per_refresh": u_flop, "ms_per_refresh": u_ms,
                  "fp64_equivalent_tflops": u_eq / (u_ms / 1e3) / 1e12,
                  "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops_sustained)"}
        return {"kernel": "refresh (FP64 panels + tensor-core split updates)", "ms_per_launch": per,
                "fp64_equivalent_tflops": 2.0 * n ** 3 * W / (per / 1e3) / 1e12,
                "panel": panel, "update": update}
    ach = 2.0 * n ** 3 * W / (per / 1e3) / 1e12
    return {"kernel": "refresh (Gauss-Jordan inverse, FP64)", "bound": "alu", "achieved": ach,
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
            "flop_per_launch": 2.0 * n ** 3 * W, "ms_per_launch": per, "peak_source": FP64_SRC}


def det_flush_roofline(flush, n, W, kc, ms_per_full, hbm, s=8, cf=1):
    """One full determinant flush of every walker: A_0^{-1} -= P Q^T with Kc =
    K k slot columns (Eq. delayed_Ainv), n^2 Kc FMA per walker, reading and
    writing A_0^{-1} once (2 n^2 s).  FP64 tiles are bound by the FP64 pipe;
    the split product, double-float and TF32 / BF16 flushes keep their
    products off it and are reported against HBM."""
    if not ms_per_full:
        return None
    out = bound_of(2.0 * n * n * s * W, (2.0 * n * n * kc * W * cf) if flush == "native" else 0.0, ms_per_full,
                   hbm)
    out["ms_per_full_flush"] = ms_per_full
    return out


def pf_propose_roofline(n, W, ms, hbm, arith="native", s=8, cf=1):
    """The Pfaffian propose's pass over A^{-1} (A_0^{-1} in the delayed form):
    X = A^{-1} x for the dense column of B = [x, e_i], n^2 FMA and n^2 s bytes
    per walker (the e_i column is a copy of one column; the delayed slot
    corrections are n x 2K).  Bound: the FP64 pipe at n^2 FMA against HBM at
    n^2 s, whichever takes longer; in double-float arithmetic the products run
    on the FP32 pipe and HBM binds."""
    return bound_of(n * n * s * W, (2.0 * n * n * W * cf if arith == "native" else 0.0), ms, hbm)


def pf_flush_roofline(flush, n, W, K, ms_per_full, hbm, s=8, cf=1):
    """One full skew flush of every walker: A_0^{-1} += P Q^T over K steps of
    2 slot columns (Eq. pf_delayed_Ainv), the upper half computed and
    mirrored, n (n + 1) / 2 x 2K FMA per walker, reading the upper half of
    A_0^{-1} and writing both (1.5 n^2 s).  The FP64 flush is bound by the
    FP64 pipe; the double-float and split-product flushes keep their products
    off it and are reported against HBM."""
    if not ms_per_full:
        return None
    flop = 2.0 * (n * (n + 1) / 2) * 2 * K * W * cf
    byt = 1.5 * n * n * s * W
    out = bound_of(byt, flop if flush == "native" else 0.0, ms_per_full, hbm)
    out["flop_per_full_flush"] = flop
    out["bytes_per_full_flush"] = byt
    out["ms_per_full_flush"] = ms_per_full
    out["fp64_equivalent_tflops"] = flop / (ms_per_full / 1e3) / 1e12
    return out


def dominant(cand):
    """The line's roofline: the kernel class with the most time in the timed region."""
    cand = {k: v for k, v in cand.items() if v[1]}
    dom = max(cand, key=lambda k: cand[k][0])
    roof = dict(cand[dom][1])
    roof["kernel"] = roof.get("kernel", dom)
    roof["dominant_kernel_by_time"] = dom
    roof["kernel_ms_in_timed_region"] = {k: v[0] for k, v in cand.items()}
    return roof


# --------------------------------------------------------------------------
# parity samples against exact ratios (fresh LAPACK solves on the host)
# --------------------------------------------------------------------------
def exact_parity_det(Phi, occ0, slot, new, ratios, walkers, steps):
    """Relative error of the GPU ratios of sampled walkers against the exact
    ratio det(I + V A^{-1} U) of every step, A^{-1} U from a fresh LAPACK solve
    of the current matrix."""
    out = []
    k = slot.shape[2] if slot.ndim == 3 else 1
    for w in walkers:
        occ = occ0[w].copy()
        for s in range(steps):
            A = Phi[occ]
            i = np.atleast_1d(slot[s, w])
            nr = np.atleast_1d(new[s, w])
            U = np.zeros((A.shape[0], k), dtype=A.dtype)
            U[i, np.arange(k)] = 1
            V = Phi[nr] - Phi[occ[i]]
            ex = np.linalg.det(np.eye(k, dtype=A.dtype) + V @ np.linalg.solve(A, U))
            out.append(abs(ratios[s, w] - ex) / abs(ex))
            occ[i] = nr
    out = np.array(out)
    return {"walkers": list(walkers), "steps": steps, "max_rel": float(out.max()),
            "median_rel": float(np.median(out)), "p99_rel": float(np.quantile(out, 0.99))}


def exact_parity_pf(F, pos0, slot, new, ratios, walkers, steps):
    """Relative error of the GPU ratios of sampled walkers against the exact
    pf(C^{-1} + B^T A^{-1} B) / pf(C^{-1}) (App. A.2) with A^{-1} B from a
    fresh LAPACK solve; for the row-and-column move B = [x, e_i], C = -J this
    is 1 + x . A^{-1} e_i."""
    out = []
    for w in walkers:
        pos = pos0[w].copy()
        for s in range(steps):
            A = F[np.ix_(pos, pos)]
            i, nr = slot[s, w], new[s, w]
            x = F[nr, pos] - F[pos[i], pos]
            e = np.zeros(len(pos), dtype=A.dtype)
            e[i] = 1
            ex = 1.0 + x @ np.linalg.solve(A, e)
            out.append(abs(ratios[s, w] - ex) / abs(ex))
            pos[i] = nr
    out = np.array(out)
    return {"walkers": list(walkers), "steps": steps, "max_rel": float(out.max()),
            "median_rel": float(np.median(out)), "p99_rel": float(np.quantile(out, 0.99))}


def drift_vs_plain(arm_ratios, arms):
    """Drift of every arm's ratios against the plain FP64 arm (same moves);
    steps within 1e-6 of the median |ratio| (near a node) are counted apart."""
    if "plain" not in arm_ratios:
        return
    ref = arm_ratios["plain"]
    med = ref.abs().median()
    gate = ref.abs() >= 1e-6 * med
    for arm, r in arm_ratios.items():
        if arm == "plain":
            continue
        d = (r - ref).abs()
        relerr = (d / ref.abs())[gate]
        arms[arm]["ratio_err_vs_plain_fp64"] = {
            "max_rel": relerr.max().item(), "median_rel": relerr.median().item(),
            "p99_rel": relerr.double().quantile(0.99).item() if relerr.numel() < 16_000_000 else None,
            "p999_rel": relerr.double().quantile(0.999).item() if relerr.numel() < 16_000_000 else None,
            "max_abs_over_median_abs": (d.max() / med).item(), "near_node_steps": int((~gate).sum().item())}


# --------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and the reference arm)
# --------------------------------------------------------------------------
def cpu_baseline_det(cfg, Phi, occ0, slot, new, budget_s=15.0, max_steps=32):
    from oracle import lru_oracle as O
    n, k = cfg["n"], cfg["k"]
    steps = min(max_steps, slot.shape[0])
    done, tsum, wl = 0, 0.0, 0
    for w in range(occ0.shape[0]):
        occ = occ0[w].copy()
        Ainv = np.linalg.inv(O.slater_matrix(Phi, occ))
        ts = time.perf_counter()
        for s in range(steps):
            i = np.atleast_1d(slot[s, w])
            nr = np.atleast_1d(new[s, w])
            U = O.onehot_matrix(n, i, dtype=Phi.dtype)
            V = Phi[nr] - Phi[occ[i]]
            r, Ainv = O.det_lru(Ainv, U, V, return_update=True)
            occ[i] = nr
        tsum += time.perf_counter() - ts
        done += steps
        wl += 1
        if tsum > budget_s:
            break
    return {"value": done / tsum, "unit": "walker-updates/s", "cores": host_threads(), "kind": "oracle",
            "sample": f"plain {cfg['dtype'].upper()} chain (oracle det_lru, Eq. det_inv) of {wl} walkers x {steps} "
                      f"steps at n={n}, k={k}, {tsum:.1f} s"}


def cpu_baseline_pf(cfg, F, pos0, slot, new, budget_s=15.0, max_steps=32):
    from oracle import lru_oracle as O
    n = cfg["n"]
    steps = min(max_steps, slot.shape[0])
    done, tsum, wl = 0, 0.0, 0
    for w in range(pos0.shape[0]):
        pos = pos0[w].copy()
        Ainv = np.linalg.inv(O.pairing_matrix(F, pos))
        ts = time.perf_counter()
        for s in range(steps):
            B, C = O.pf_row_col_move(F, pos, slot[s, w], new[s, w])
            r, Ainv = O.pf_lru(Ainv, B, C, return_update=True)
            pos[slot[s, w]] = new[s, w]
        tsum += time.perf_counter() - ts
        done += steps
        wl += 1
        if tsum > budget_s:
            break
    return {"value": done / tsum, "unit": "walker-updates/s", "cores": host_threads(), "kind": "oracle",
            "sample": f"plain {cfg['dtype'].upper()} Pfaffian chain (oracle pf_lru, Eq. pf_inv) of {wl} walkers x "
                      f"{steps} steps at n={n}, {tsum:.1f} s"}


def cpu_baseline_ragged(cfg, seed, budget_s=15.0, max_steps=4):
    """The oracle's plain chain (det_lru with dense U, V) on walkers of the
    ragged batch, in the batch's proportions of n and k."""
    from oracle import lru_oracle as O
    from paper_2602_05255_gb300 import workloads
    n_w, k_w = ragged_shapes(cfg, seed)
    g = workloads.rng(seed + 9)
    cplx = cfg["dtype"] != "f64"
    done, tsum, wl = 0, 0.0, 0
    for w in range(len(n_w)):
        n, k = int(n_w[w]), int(k_w[w])
        A = workloads.gaussian(g, (n, n), 1.0 / n, cplx) + 2.5 * np.eye(n)
        Ainv = np.linalg.inv(A)
        ts = time.perf_counter()
        for s in range(max_steps):
            U = workloads.gaussian(g, (n, k), 1.0 / n, cplx)
            V = workloads.gaussian(g, (k, n), 1.0 / n, cplx)
            r, Ainv = O.det_lru(Ainv, U, V, return_update=True)
        tsum += time.perf_counter() - ts
        done += max_steps
        wl += 1
        if tsum > budget_s:
            break
    return {"value": done / tsum, "unit": "walker-updates/s", "cores": host_threads(), "kind": "oracle",
            "sample": f"plain {cfg['dtype'].upper()} chains (oracle det_lru, dense U, V) of the first {wl} walkers "
                      f"of the ragged batch x {max_steps} steps, {tsum:.1f} s"}


def cpu_fig1(cfg, seed, budget_s=15.0, n=128):
    """The same comparison with the oracle on the host cores at one n: its
    from-scratch slogdet (LU, Sec. 2.1's reference values) against its
    Sherman-Morrison step (Eq. det_inv); value = the speedup."""
    from oracle import lru_oracle as O
    from paper_2602_05255_gb300 import workloads
    sub = {"walkers": 16, "n": n, "m": 2 * n, "k": 1, "dtype": "f64", "var": None, "first_rows": False}
    Phi, occ0, slot, new = det_inputs(sub, seed, 4)
    t_d = t_l = 0.0
    done = 0
    t_start = time.perf_counter()
    for w in range(sub["walkers"]):
        occ = occ0[w].copy()
        Ainv = O.inv(O.slater_matrix(Phi, occ))
        for s in range(4):
            U, V = O.det_row_move(Phi, occ, slot[s, w], new[s, w])
            occ2 = occ.copy()
            occ2[slot[s, w]] = new[s, w]
            ts = time.perf_counter()
            O.slogdet(O.slater_matrix(Phi, occ2))
            t_d += time.perf_counter() - ts
            ts = time.perf_counter()
            r, Ainv = O.det_lru(Ainv, U, V, return_update=True)
            t_l += time.perf_counter() - ts
            occ = occ2
            done += 1
        if time.perf_counter() - t_start > budget_s:
            break
    return {"value": t_d / t_l, "unit": "x", "cores": host_threads(), "kind": "oracle",
            "sample": f"oracle slogdet vs det_lru at n={n}, {done} walker-steps"}


# --------------------------------------------------------------------------
# determinant workloads (headline, c1, c2, c4)
# --------------------------------------------------------------------------
def det_state(L, torch, cfg, delay, arith, flush, Phi_d, occ0):
    W, n, k = cfg["walkers"], cfg["n"], cfg["k"]
    tdt = torch_dtype(torch, cfg)
    st = L.LowRankState("det", W, n, k=k, dtype=tdt, delay=delay, flush=FLUSH[flush], arith=ARITH[arith])
    occ_d = torch.tensor(occ0, device="cuda")
    A = st.gather_rows(Phi_d, occ_d)
    st.init(A)
    V = torch.empty(W, k, n, dtype=tdt, device="cuda")
    idx = torch.empty(W, k, dtype=torch.int32, device="cuda")
    ops = (L.Operand(idx=idx, onehot_mask=(1 << k) - 1), L.Operand(dense=V))
    return st, occ_d, A, V, idx, ops


def run_det_arm(L, torch, args, cfg, K, arm, Phi_d, occ0, slot_d, new_d, dist):
    W = cfg["walkers"]
    dev = torch.cuda.current_device()
    delay, arith, flush = ARMS[arm]
    delay = K if delay is None else delay
    st, occ_d, A, V, idx, (U_op, V_op) = det_state(L, torch, cfg, delay, arith, flush, Phi_d, occ0)
    tdt = torch_dtype(torch, cfg)
    ratio = torch.empty(W, dtype=tdt, device="cuda")
    ratios_all = torch.empty(args.steps, W, dtype=tdt, device="cuda")
    status = torch.empty(W, dtype=torch.int32, device="cuda")
    every = cfg["refresh_every"]

    def step(s, timed_idx):
        st.form_row_moves(Phi_d, occ_d, slot_d[s], new_d[s], V, idx)
        st.propose_det(U_op, V_op, ratio if timed_idx is None else ratios_all[timed_idx], status)
        st.accept()
        st.commit_moves(occ_d, slot_d[s], new_d[s])
        if timed_idx is not None and every and (timed_idx + 1) % every == 0:
            st.gather_rows(Phi_d, occ_d, A)
            st.refresh(A, want_drift=False)

    def refresh():
        st.gather_rows(Phi_d, occ_d, A)
        st.refresh(A, want_drift=False)

    ms, clk, launches, prof, amort = timed_steps(torch, st, step, args, dist, dev, refresh, every)
    st.close()
    return ratios_all, ms, clk, launches, prof, (delay, arith, flush), amort


def e2e_det(L, torch, cfg, K, arm, Phi_d, occ0, slot_h, new_h, steps):
    """The metric through the C-ABI with host buffers: each step copies its
    proposals (slot, new row) host->device from pinned memory and reads the
    ratios back, inside the timed region (the line's arm, same refresh
    schedule)."""
    W = cfg["walkers"]
    delay, arith, flush = ARMS[arm]
    delay = K if delay is None else delay
    st, occ_d, A, V, idx, (U_op, V_op) = det_state(L, torch, cfg, delay, arith, flush, Phi_d, occ0)
    tdt = torch_dtype(torch, cfg)
    ratio = torch.empty(W, dtype=tdt, device="cuda")
    status = torch.empty(W, dtype=torch.int32, device="cuda")
    sl_h = torch.from_numpy(np.ascontiguousarray(slot_h)).pin_memory()
    nw_h = torch.from_numpy(np.ascontiguousarray(new_h)).pin_memory()
    r_h = torch.empty(steps, W, dtype=tdt).pin_memory()
    sl_d = torch.empty(sl_h.shape[1:], dtype=torch.int32, device="cuda")
    nw_d = torch.empty(nw_h.shape[1:], dtype=torch.int32, device="cuda")
    every = cfg["refresh_every"]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for s in range(steps):
        sl_d.copy_(sl_h[s], non_blocking=True)
        nw_d.copy_(nw_h[s], non_blocking=True)
        st.form_row_moves(Phi_d, occ_d, sl_d, nw_d, V, idx)
        st.propose_det(U_op, V_op, ratio, status)
        st.accept()
        st.commit_moves(occ_d, sl_d, nw_d)
        r_h[s].copy_(ratio, non_blocking=True)
        if every and (s + 1) % every == 0:
            st.gather_rows(Phi_d, occ_d, A)
            st.refresh(A, want_drift=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    frac = refresh_share(steps, every)
    added = 0.0
    if frac > 0:
        # the schedule's refresh share the steps did not reach, as in the device-timed arm
        e0.record()
        st.gather_rows(Phi_d, occ_d, A)
        st.refresh(A, want_drift=False)
        e1.record()
        torch.cuda.synchronize()
        added = frac * e0.elapsed_time(e1)
    st.close()
    return {"value": W * steps / ((ms + added) / 1e3), "unit": "walker-updates/s",
            "h2d_bytes_per_step": 2 * sl_h[0].numel() * 4, "d2h_bytes_per_step": W * scalar_bytes(cfg),
            "steps": steps, "arm": arm, "refresh_amortised_ms": added}


def tuned_delay(L, torch, cfg, steps):
    """The headline's delay K from the autotuner: the delayed form with its
    double-float GEMV and split-product flush, K among the candidates up to
    min(32, timed steps) (so that the timed region holds a full window)."""
    from paper_2602_05255_gb300 import autotune
    cands = [c for c in autotune.candidates("det", cfg["n"], cfg["k"]) if c <= min(32, max(steps, 4))]
    res = autotune.tune("det", cfg["n"], cfg["k"], torch.float64, flushes=[L.FLUSH_SPLIT], ariths=[L.ARITH_DF],
                        walkers=128, delays=cands, tiles=[], include_plain=False, use_cache=False)
    return res["delay"], {"source": "autotuner (paper_2602_05255_gb300.autotune.tune, 128 walkers)",
                          "candidates": cands, "rates": {str(t["delay"]): t["updates_per_s"] for t in res["trials"]}}


def main_det(args, cfg, torch, L, rank, world, dist):
    W, n, k = cfg["walkers"], cfg["n"], cfg["k"]
    s_b, cf = scalar_bytes(cfg), flop_factor(cfg)
    tune_info = None
    K = cfg["delay"]
    if K == "tune":
        K, tune_info = tuned_delay(L, torch, cfg, args.steps)
    seed = multigpu.shard_seed(args.seed, rank)
    Phi, occ0, slot, new = det_inputs(cfg, seed, args.warmup + args.steps)
    tdt = torch_dtype(torch, cfg)
    Phi_d = torch.tensor(Phi, device="cuda").to(tdt)
    slot_d = torch.tensor(slot, device="cuda")
    new_d = torch.tensor(new, device="cuda")
    hbm, bf16_sus, _ = load_peaks()
    arms, arm_ratios = {}, {}
    order = [a.strip() for a in cfg["arms"].split(",") if a.strip()]
    for arm in order:
        ratios_all, ms, clk, launches, prof, (delay, arith, flush), amort = run_det_arm(
            L, torch, args, cfg, K, arm, Phi_d, occ0, slot_d, new_d, dist)
        arm_ratios[arm] = ratios_all
        upd = W * args.steps * world
        # refresh time of the schedule: timed in the region, plus the amortised share
        ref_ms = prof["refresh"][0] + (amort["added_ms"] if amort else 0.0)
        a = {"value": multigpu.whole_job_rate(W * args.steps, world, ms), "ms_per_step": ms / args.steps,
             "delay_K": delay, "gemv_arith": arith, "flush": flush if delay >= 2 else None,
             "value_excl_refresh": upd / ((ms - ref_ms) / 1e3) if ms > ref_ms else None,
             "refresh_amortised": amort,
             "refreshes_in_timed_region": args.steps // cfg["refresh_every"] if cfg["refresh_every"] else 0,
             "refresh_ms_total": ref_ms, "kernel_ms": {c: v[0] for c, v in prof.items()},
             "kernel_launches_timed": {c: v[1] for c, v in prof.items()}, "gpu_launches": launches, "clocks": clk}
        acc_ms, acc_n = prof["accept"]
        a["accept_roofline"] = accept_roofline(delay, arith, n, W, acc_ms / acc_n if acc_n else None, hbm, k=k,
                                               s=s_b, cf=cf)
        if delay >= 2:
            nfl = (args.warmup + args.steps) // delay - args.warmup // delay
            fl_ms = prof["flush"][0]
            a["flush_roofline"] = det_flush_roofline(flush, n, W, delay * k, fl_ms / nfl if nfl else None, hbm,
                                                     s=s_b, cf=cf)
            a["full_flushes_in_timed_region"] = nfl
        if cfg["dtype"] == "f64":
            a["refresh_roofline"] = refresh_roofline(prof, n, W, bf16_sus)
        arms[arm] = a
    drift_vs_plain(arm_ratios, arms)
    if rank == 0:
        psteps = min(args.steps, 64 if n <= 512 else (32 if n <= 1024 else 8))
        occ_t = occ0.copy()                      # occupation at the start of the timed region
        for s_ in range(args.warmup):
            rows = np.arange(W)[:, None] if slot.ndim == 3 else np.arange(W)
            occ_t[rows, slot[s_]] = new[s_]
        for arm, r in arm_ratios.items():
            arms[arm]["parity_vs_exact"] = exact_parity_det(
                Phi, occ_t, slot[args.warmup:], new[args.warmup:], r[:psteps].cpu().numpy(),
                sorted({0, W // 2}), psteps)
    main_arm = cfg["main"] if cfg["main"] in arms else order[0]
    head = arms[main_arm]
    km = head["kernel_ms"]
    cand = {"accept": (km.get("accept", 0.0), head["accept_roofline"])}
    if head.get("flush_roofline"):
        cand["flush"] = (km.get("flush", 0.0), head["flush_roofline"])
    rr = head.get("refresh_roofline")
    if rr and "panel" in rr:
        cand["refresh_panel"] = (km.get("refresh_panel", 0.0), rr["panel"])
        cand["refresh_update"] = (km.get("refresh_update", 0.0), rr["update"])
    elif rr:
        cand["refresh"] = (km.get("refresh", 0.0), rr)
    roof = dominant(cand)
    line = {
        "metric": METRIC if args.config == "headline" else
        f"walker-updates/sec, {args.config}: {workload_name(cfg, cfg.get('delay'))}",
        "value": head["value"], "unit": "walker-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": cfg["dtype"], "data": "synthetic",
        "config": config_of(args.config, cfg),
        "run": {"arm": main_arm, "delay_K": K, "walkers_per_gpu": W, "n": n, "m": cfg["m"], "k": k},
        "roofline": roof, "arms": arms, "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
    }
    if tune_info:
        line["run"]["delay_K_tuning"] = tune_info
    if rank == 0 and not args.no_e2e:
        line["e2e"] = e2e_det(L, torch, cfg, K, main_arm, Phi_d, occ0, slot[args.warmup:args.warmup + args.steps],
                              new[args.warmup:args.warmup + args.steps], args.steps)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_det(cfg, Phi, occ0, slot, new)
    return line


# --------------------------------------------------------------------------
# Pfaffian workload (c3; Sec. 3): rank-2 row-and-column moves
# --------------------------------------------------------------------------
def pf_state(L, torch, cfg, delay, arith, flush, F_d, pos0):
    """A Pfaffian handle initialised from F[pos][:, pos], with its move buffers."""
    W, n = cfg["walkers"], cfg["n"]
    tdt = torch_dtype(torch, cfg)
    st = L.LowRankState("pf", W, n, k=1, dtype=tdt, delay=delay, flush=FLUSH[flush], arith=ARITH[arith])
    pos_d = torch.tensor(pos0, device="cuda")
    A = st.gather_pairs(F_d, pos_d)
    st.init(A)
    B = torch.empty(W, 2, n, dtype=tdt, device="cuda")
    idx = torch.empty(W, 2, dtype=torch.int32, device="cuda")
    B_op = L.Operand(dense=B, idx=idx, onehot_mask=0b10)     # B = [x, e_i], C = -J
    return st, pos_d, A, B, idx, B_op


def run_pf_arm(L, torch, args, cfg, arm, F_d, pos0, slot_d, new_d, dist):
    W = cfg["walkers"]
    dev = torch.cuda.current_device()
    delay, arith, flush = PF_ARMS[arm]
    delay = cfg["delay"] if delay is None else delay
    st, pos_d, A, B, idx, B_op = pf_state(L, torch, cfg, delay, arith, flush, F_d, pos0)
    tdt = torch_dtype(torch, cfg)
    ratio = torch.empty(W, dtype=tdt, device="cuda")
    ratios_all = torch.empty(args.steps, W, dtype=tdt, device="cuda")
    status = torch.empty(W, dtype=torch.int32, device="cuda")
    every = cfg["refresh_every"]

    def step(s, timed_idx):
        st.form_pf_moves(F_d, pos_d, slot_d[s], new_d[s], B, idx)
        st.propose_pf(B_op, None, ratio if timed_idx is None else ratios_all[timed_idx], status)
        st.accept()
        st.commit_moves(pos_d, slot_d[s], new_d[s])
        if timed_idx is not None and every and (timed_idx + 1) % every == 0:
            st.gather_pairs(F_d, pos_d, A)
            st.refresh(A, want_drift=False)

    def refresh():
        st.gather_pairs(F_d, pos_d, A)
        st.refresh(A, want_drift=False)

    ms, clk, launches, prof, amort = timed_steps(torch, st, step, args, dist, dev, refresh, every)
    st.close()
    return ratios_all, ms, clk, launches, prof, (delay, arith, flush), amort


def e2e_pf(L, torch, cfg, arm, F_d, pos0, slot_h, new_h, steps):
    """The Pfaffian metric through the C-ABI with host buffers: each step
    copies its moves host->device from pinned memory and reads the ratios
    back inside the timed region (the line's arm)."""
    W = cfg["walkers"]
    delay, arith, flush = PF_ARMS[arm]
    delay = cfg["delay"] if delay is None else delay
    st, pos_d, A, B, idx, B_op = pf_state(L, torch, cfg, delay, arith, flush, F_d, pos0)
    tdt = torch_dtype(torch, cfg)
    ratio = torch.empty(W, dtype=tdt, device="cuda")
    status = torch.empty(W, dtype=torch.int32, device="cuda")
    sl_h = torch.from_numpy(np.ascontiguousarray(slot_h)).pin_memory()
    nw_h = torch.from_numpy(np.ascontiguousarray(new_h)).pin_memory()
    r_h = torch.empty(steps, W, dtype=tdt).pin_memory()
    sl_d = torch.empty(W, dtype=torch.int32, device="cuda")
    nw_d = torch.empty(W, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for s in range(steps):
        sl_d.copy_(sl_h[s], non_blocking=True)
        nw_d.copy_(nw_h[s], non_blocking=True)
        st.form_pf_moves(F_d, pos_d, sl_d, nw_d, B, idx)
        st.propose_pf(B_op, None, ratio, status)
        st.accept()
        st.commit_moves(pos_d, sl_d, nw_d)
        r_h[s].copy_(ratio, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st.close()
    return {"value": W * steps / (ms / 1e3), "unit": "walker-updates/s", "h2d_bytes_per_step": 2 * W * 4,
            "d2h_bytes_per_step": W * scalar_bytes(cfg), "steps": steps, "arm": arm}


def main_pf(args, cfg, torch, L, rank, world, dist):
    W, n, K = cfg["walkers"], cfg["n"], cfg["delay"]
    s_b, cf = scalar_bytes(cfg), flop_factor(cfg)
    seed = multigpu.shard_seed(args.seed, rank)
    F, pos0, slot, new = pf_inputs(cfg, seed, args.warmup + args.steps)
    F_d = torch.tensor(F, device="cuda").to(torch_dtype(torch, cfg))
    slot_d = torch.tensor(slot, device="cuda")
    new_d = torch.tensor(new, device="cuda")
    hbm, _, _ = load_peaks()
    arms, arm_ratios = {}, {}
    order = [a.strip() for a in cfg["arms"].split(",") if a.strip()]
    for arm in order:
        ratios_all, ms, clk, launches, prof, (delay, arith, flush), amort = run_pf_arm(
            L, torch, args, cfg, arm, F_d, pos0, slot_d, new_d, dist)
        arm_ratios[arm] = ratios_all
        acc_ms, acc_n = prof["accept"]
        pro_ms, pro_n = prof["propose"]
        a = {"value": multigpu.whole_job_rate(W * args.steps, world, ms), "ms_per_step": ms / args.steps,
             "delay_K": delay, "propose_arith": arith, "flush": flush if delay >= 2 else None,
             "kernel_ms": {c: v[0] for c, v in prof.items()},
             "kernel_launches_timed": {c: v[1] for c, v in prof.items()},
             "gpu_launches": launches, "clocks": clk, "refresh_amortised": amort,
             "propose_roofline": pf_propose_roofline(n, W, pro_ms / pro_n if pro_n else None, hbm, arith, s_b, cf)}
        if delay < 2:
            a["accept_roofline"] = accept_roofline(delay, "native", n, W, acc_ms / acc_n if acc_n else None, hbm,
                                                   pf=True, s=s_b, cf=cf)
        else:
            nfl = (args.warmup + args.steps) // delay - args.warmup // delay
            a["flush_roofline"] = pf_flush_roofline(flush, n, W, delay, prof["flush"][0] / nfl if nfl else None,
                                                    hbm, s_b, cf)
        arms[arm] = a
    drift_vs_plain(arm_ratios, arms)
    if rank == 0:
        psteps = min(args.steps, 64)
        pos_t = pos0.copy()                      # positions at the start of the timed region
        for s_ in range(args.warmup):
            pos_t[np.arange(W), slot[s_]] = new[s_]
        for arm, r in arm_ratios.items():
            arms[arm]["parity_vs_exact"] = exact_parity_pf(
                F, pos_t, slot[args.warmup:], new[args.warmup:], r[:psteps].cpu().numpy(), [0, W // 2], psteps)
    main_arm = cfg["main"] if cfg["main"] in arms else order[0]
    head = arms[main_arm]
    km = head["kernel_ms"]
    cand = {"propose": (km.get("propose", 0.0), head["propose_roofline"])}
    if head.get("accept_roofline"):
        cand["accept"] = (km.get("accept", 0.0), head["accept_roofline"])
    if head.get("flush_roofline"):
        cand["flush"] = (km.get("flush", 0.0), head["flush_roofline"])
    line = {
        "metric": PF_METRIC, "value": head["value"], "unit": "walker-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": cfg["dtype"], "data": "synthetic",
        "config": config_of("c3", cfg),
        "run": {"arm": main_arm, "delay_K": K, "walkers_per_gpu": W, "n": n, "m": cfg["m"]},
        "roofline": dominant(cand), "arms": arms, "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
    }
    if rank == 0 and not args.no_e2e:
        line["e2e"] = e2e_pf(L, torch, cfg, main_arm, F_d, pos0, slot[args.warmup:args.warmup + args.steps],
                             new[args.warmup:args.warmup + args.steps], args.steps)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_pf(cfg, F, pos0, slot, new)
    return line


# --------------------------------------------------------------------------
# c5: walkers of uneven n and k in one persistent launch, and the adjoint
# --------------------------------------------------------------------------
def main_ragged(args, cfg, torch, L, rank, world, dist):
    W, K = cfg["walkers"], cfg["delay"]
    tdt = torch_dtype(torch, cfg)
    s_b, cf = scalar_bytes(cfg), flop_factor(cfg)
    seed = multigpu.shard_seed(args.seed, rank)
    n_w, k_w = ragged_shapes(cfg, seed)
    kmax = int(max(cfg["ks"]))
    offs = np.concatenate([[0], np.cumsum(n_w)]).astype(np.int64)
    moffs = np.concatenate([[0], np.cumsum(n_w.astype(np.int64) ** 2)])
    st = L.LowRankState("det", W, [int(x) for x in n_w], k=kmax, dtype=tdt, delay=K,
                        k_per_walker=[int(x) for x in k_w])
    gen = torch.Generator(device="cuda").manual_seed(seed)
    # A_w = 2.5 I + N(0, 1/n) (complex parts N(0, 1/2n)), built on the device
    A = torch.empty(int(moffs[-1]), dtype=tdt, device="cuda")
    for w in range(W):
        nn = int(n_w[w])
        blk = torch.randn(nn, nn, dtype=tdt, device="cuda", generator=gen) / math.sqrt(nn)
        blk.diagonal().add_(2.5)
        A[moffs[w]:moffs[w + 1]] = blk.reshape(-1)
    st.init(A)
    del A

    def operands():
        U = torch.zeros(int(offs[-1]) * kmax, dtype=tdt, device="cuda")
        V = torch.zeros_like(U)
        for w in range(W):
            nn, kk = int(n_w[w]), int(k_w[w])
            b = int(offs[w]) * kmax
            U[b: b + kk * nn] = torch.randn(kk * nn, dtype=tdt, device="cuda", generator=gen) * (0.3 / math.sqrt(nn))
            V[b: b + kk * nn] = torch.randn(kk * nn, dtype=tdt, device="cuda", generator=gen) * (0.3 / math.sqrt(nn))
        return U, V

    sets = [operands() for _ in range(2)]
    ratio = torch.empty(W, dtype=tdt, device="cuda")
    status = torch.empty(W, dtype=torch.int32, device="cuda")
    acc = torch.empty(W, dtype=torch.uint8, device="cuda")

    def launch(i):
        U, V = sets[i]
        st.step_persistent(L.Operand(dense=U), L.Operand(dense=V), accept=True, ratio=ratio, status=status, acc=acc)

    launch(0)                              # one eager call before capturing
    torch.cuda.synchronize()
    graphs = []
    for i in range(len(sets)):
        g_ = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_):
            launch(i)
        graphs.append(g_)

    def step(s, timed_idx):
        graphs[s % len(graphs)].replay()

    dev = torch.cuda.current_device()
    ms, clk, launches, prof, _ = timed_steps(torch, st, step, args, dist, dev)
    launches = args.steps                  # one persistent kernel per replay (the memset is a copy engine op)
    st.check_device_error()
    # algorithmic work per step: the propose's X = A_0^{-1} U (n^2 s read, n^2 k
    # FMA), the delayed accept's GEMV (the same again) and the flush amortised
    # over K steps (2 n^2 s and n^2 K k FMA per full flush)
    n2 = n_w.astype(np.float64) ** 2
    byt = float(np.sum(2 * n2 * s_b + 2 * n2 * s_b / K))
    flop = float(np.sum(2 * 2 * n2 * k_w * cf + 2 * n2 * k_w * cf))
    hbm, _, _ = load_peaks()
    roof = bound_of(byt, flop, ms / args.steps, hbm, fp32=cfg["dtype"] == "c64")
    roof["kernel"] = "persistent step (propose + accept + flush, one launch)"
    # the adjoint: propose-only launch + lru_backward_det (d log r / d(U, V, A))
    U, V = sets[0]
    gvec = torch.randn(W, dtype=tdt, device="cuda", generator=gen)
    st.step_persistent(L.Operand(dense=U), L.Operand(dense=V), accept=False, ratio=ratio, status=status, acc=acc)
    st.backward_det(gvec)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record()
    for _ in range(reps):
        st.backward_det(gvec)
    e1.record()
    torch.cuda.synchronize()
    bw_ms = e0.elapsed_time(e1) / reps
    line = {
        "metric": RAGGED_METRIC, "value": multigpu.whole_job_rate(W * args.steps, world, ms), "unit": "walker-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": cfg["dtype"], "data": "synthetic",
        "config": config_of("c5", cfg),
        "run": {"delay_K": K, "walkers_per_gpu": W,
                "n_counts": {str(x): int((n_w == x).sum()) for x in cfg["ns"]},
                "k_counts": {str(x): int((k_w == x).sum()) for x in cfg["ks"]}},
        "roofline": roof, "gpu_launches": launches, "clocks": clk,
        "adjoint": {"ms_per_backward": bw_ms, "walker_gradients_per_s": W / (bw_ms / 1e3),
                    "of": "d log r / d(U, V, A) of every walker (lru_backward_det)"},
    }
    if rank == 0 and not args.no_e2e:
        # the same steps through the C-ABI with host buffers: U, V copied in from
        # pinned memory every step, ratios and decisions read back
        Uh = [x[0].cpu().pin_memory() for x in sets]
        Vh = [x[1].cpu().pin_memory() for x in sets]
        Ud, Vd = torch.empty_like(sets[0][0]), torch.empty_like(sets[0][1])
        r_h = torch.empty(args.steps, W, dtype=tdt).pin_memory()
        torch.cuda.synchronize()
        e0.record()
        for s in range(args.steps):
            Ud.copy_(Uh[s % 2], non_blocking=True)
            Vd.copy_(Vh[s % 2], non_blocking=True)
            st.step_persistent(L.Operand(dense=Ud), L.Operand(dense=Vd), accept=True, ratio=ratio, status=status,
                               acc=acc)
            r_h[s].copy_(ratio, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1)
        line["e2e"] = {"value": W * args.steps / (ems / 1e3), "unit": "walker-updates/s",
                       "h2d_bytes_per_step": 2 * Ud.numel() * Ud.element_size(),
                       "d2h_bytes_per_step": W * ratio.element_size(), "steps": args.steps}
    st.close()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_ragged(cfg, seed)
    return line


# --------------------------------------------------------------------------
# fig1: the paper's Fig. 1 scan on GB300 (context, not a target)
# --------------------------------------------------------------------------
def main_fig1(args, cfg, torch, L, rank, world, dist):
    """Per n: the time of one step of W walkers for (a) the direct batched
    slogdet / slogpf of the updated matrices (O(n^3) per walker), (b) the LRU
    ratio alone (propose), (c) the LRU ratio with the inverse update (propose
    + accept, plain form).  Each at warm state, CUDA events, median of a few
    repetitions."""
    W = cfg["walkers"]
    reps = max(3, min(args.steps, 20))
    ev = lambda: torch.cuda.Event(enable_timing=True)
    table = []
    hbm, _, _ = load_peaks()
    for n in cfg["ns"]:
        row = {"n": n}
        for kind in ("det", "pf"):
            sub = {"walkers": W, "n": n, "m": 2 * n, "k": 1, "dtype": "f64", "var": None, "first_rows": False,
                   "delay": 0, "refresh_every": 0}
            if kind == "det":
                Phi, occ0, slot, new = det_inputs(sub, args.seed + n, reps + 2)
                src = torch.tensor(Phi, device="cuda")
            else:
                F, occ0, slot, new = pf_inputs(sub, args.seed + n, reps + 2)
                src = torch.tensor(F, device="cuda")
            st = L.LowRankState(kind, W, n, k=1, dtype=torch.float64)
            occ_d = torch.tensor(occ0, device="cuda")
            A = st.gather_rows(src, occ_d) if kind == "det" else st.gather_pairs(src, occ_d)
            st.init(A)
            slot_d, new_d = torch.tensor(slot, device="cuda"), torch.tensor(new, device="cuda")
            times = {"direct": [], "ratio": [], "ratio_and_inverse": []}
            for s in range(reps):
                # (a) direct: the updated matrices from scratch
                e0, e1 = ev(), ev()
                occ2 = occ_d.clone()
                occ2[torch.arange(W, device="cuda"), slot_d[s].long()] = new_d[s]
                e0.record()
                A2 = st.gather_rows(src, occ2, A) if kind == "det" else st.gather_pairs(src, occ2, A)
                (L.slogdet_batched if kind == "det" else L.slogpf_batched)(A2.view(W, n, n))
                e1.record()
                torch.cuda.synchronize()
                times["direct"].append(e0.elapsed_time(e1))
                # (b) ratio only and (c) ratio + inverse update
                for key, do_accept in (("ratio", False), ("ratio_and_inverse", True)):
                    e0, e1 = ev(), ev()
                    e0.record()
                    if kind == "det":
                        V, idx = st.form_row_moves(src, occ_d, slot_d[s], new_d[s])
                        st.propose_det(L.Operand(idx=idx, onehot_mask=1), L.Operand(dense=V))
                    else:
                        B, idx = st.form_pf_moves(src, occ_d, slot_d[s], new_d[s])
                        st.propose_pf(L.Operand(dense=B, idx=idx, onehot_mask=0b10))
                    if do_accept:
                        st.accept()
                        st.commit_moves(occ_d, slot_d[s], new_d[s])
                    e1.record()
                    torch.cuda.synchronize()
                    times[key].append(e0.elapsed_time(e1))
            st.close()
            med = {k: float(np.median(v[1:] if len(v) > 1 else v)) for k, v in times.items()}
            row[kind] = {"ms_per_step": med, "speedup_ratio_vs_direct": med["direct"] / med["ratio"],
                         "speedup_ratio_and_inverse_vs_direct": med["direct"] / med["ratio_and_inverse"]}
        table.append(row)
    last = table[-1]
    n = last["n"]
    d_ms = last["det"]["ms_per_step"]["direct"]
    # the direct determinant kernel at the largest n: Gauss-Jordan, n^3 FMA per walker, against the FP64 pipe
    roof = bound_of(n * n * 8.0 * W, 2.0 * n ** 3 * W, d_ms, hbm)
    roof["kernel"] = "direct batched slogdet (Gauss-Jordan, FP64), the O(n^3) side of the comparison"
    line = {"metric": FIG1_METRIC, "value": last["det"]["speedup_ratio_and_inverse_vs_direct"], "unit": "x",
            "n_gpus": world, "steps": reps, "warmup": 1, "ms_per_step": last["det"]["ms_per_step"]["ratio_and_inverse"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of("fig1", cfg), "roofline": roof, "table": table, "gpu_launches": None,
            "paper_context": "A100-80GB, JAX: about 200x (det) and 1000x (pf) at n = 1024, 1024 matrices (Sec. 4.1)"}
    return line


# --------------------------------------------------------------------------
def summary(line):
    """The line's arm against the plain arm (and the same for its Pfaffian
    arms), short enough to survive a truncated log tail."""
    out = {}
    for key, part in (("det", line), ("pf", line.get("pf_workload"))):
        arms = (part or {}).get("arms")
        arm = ((part or {}).get("run") or {}).get("arm")
        if not arms or "plain" not in arms or arm not in arms or arm == "plain":
            continue
        out[key] = {"plain": round(arms["plain"]["value"]), arm: round(arms[arm]["value"]),
                    "ratio": round(arms[arm]["value"] / arms["plain"]["value"], 3),
                    "max_err_vs_exact": arms[arm].get("parity_vs_exact", {}).get("max_rel")}
    return out


def main():
    args = parse()
    rank, world, local = multigpu.rank_env()
    cfg = args.cfg
    if args.impl == "reference":
        if rank != 0:
            return 0
        return reference_arm(args)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2602_05255_gb300 import lrugb as L
    if cfg["kind"] == "det":
        line = main_det(args, cfg, torch, L, rank, world, dist)
        if args.config == "headline" and not args.no_pf:
            # the Pfaffian workload (c3) in the same run, at the same steps
            pcfg = dict(PRESETS["c3"])
            pcfg["arms"] = "plain,delayed_dfpass,delayed"
            pargs = argparse.Namespace(**vars(args))
            pargs.no_e2e, pargs.no_cpu_baseline = True, True
            pl = main_pf(pargs, pcfg, torch, L, rank, world, dist)
            line["pf_workload"] = {k: pl[k] for k in ("metric", "value", "ms_per_step", "config", "run",
                                                      "roofline", "arms", "gpu_launches")}
    elif cfg["kind"] == "pf":
        line = main_pf(args, cfg, torch, L, rank, world, dist)
    elif cfg["kind"] == "fig1":
        line = main_fig1(args, cfg, torch, L, rank, world, dist)
    else:
        line = main_ragged(args, cfg, torch, L, rank, world, dist)
    line["delayed_vs_plain"] = summary(line)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def reference_arm(args):
    """The oracle as it stands on the host cores (there is no reference code),
    on a bounded sample of the same workload and config: the plain FP64 (or
    complex) chain of as many walkers as fit the time budget."""
    cfg = args.cfg
    budget = max(5.0, min(60.0, 2.0 * args.steps))
    nsteps = max(4, min(args.steps, 16))
    t0 = time.perf_counter()
    if cfg["kind"] == "pf":
        F, pos0, slot, new = pf_inputs(cfg, args.seed, nsteps)
        cb = cpu_baseline_pf(cfg, F, pos0, slot, new, budget_s=budget, max_steps=nsteps)
        metric = PF_METRIC
    elif cfg["kind"] == "det":
        Phi, occ0, slot, new = det_inputs(cfg, args.seed, nsteps)
        cb = cpu_baseline_det(cfg, Phi, occ0, slot, new, budget_s=budget, max_steps=nsteps)
        metric = METRIC if args.config == "headline" else None
    elif cfg["kind"] == "fig1":
        cb = cpu_fig1(cfg, args.seed, budget_s=budget)
        metric = FIG1_METRIC
    else:
        cb = cpu_baseline_ragged(cfg, args.seed, budget_s=budget)
        metric = RAGGED_METRIC
    conf = config_of(args.config, cfg)
    if metric is None:
        metric = f"walker-updates/sec, {args.config}: {workload_name(cfg, cfg.get('delay'))}"
    el = time.perf_counter() - t0
    line = {"impl": "reference", "metric": metric, "value": cb["value"], "unit": "walker-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * cfg["walkers"] / cb["value"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": cfg["dtype"], "data": "synthetic",
            "config": conf,
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "walker-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": el}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
