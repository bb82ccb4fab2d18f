"""The roofline arithmetic of bench.py, checked on the CPU against the
per-unit bytes and flops stated for each kernel (one walker-update of every
walker per accept or propose launch; one full flush of every walker)."""
import math
import os
import sys

import pytest

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

HBM = 6784.5
FP64 = bench.FP64_PEAK_TFLOPS


def test_fp64_peak_from_unit_counts():
    # 152 SMs x 2 DFMA per clock x 2 flop x 2.07 GHz
    assert math.isclose(FP64, 1.25856, rel_tol=1e-12)


def test_det_accept_plain_and_delayed():
    n, W = 1024, 1024
    ms = 4.0
    plain = bench.accept_roofline(0, "native", n, W, ms, HBM)
    assert plain["bytes_per_launch"] == 2 * n * n * 8 * W          # read + write A^{-1}
    assert plain["fp64_flop_per_launch"] == 4 * n * n * W          # GEMV + rank-1 update
    assert plain["bound"] == "alu"                                 # 3.4 ms at FP64 peak > 2.5 ms at HBM
    assert math.isclose(plain["achieved"], 4 * n * n * W / (ms / 1e3) / 1e12)
    assert math.isclose(plain["frac"], plain["achieved"] / FP64)
    assert math.isclose(plain["hbm"]["frac"], 2 * n * n * 8 * W / (ms / 1e3) / 1e9 / HBM)
    dl = bench.accept_roofline(16, "native", n, W, 1.9, HBM)
    assert dl["bytes_per_launch"] == n * n * 8 * W                 # one pass over A_0^{-1}
    assert dl["fp64_flop_per_launch"] == 2 * n * n * W
    assert dl["bound"] == "alu" and dl["traffic"] is None
    df = bench.accept_roofline(16, "df", n, W, 1.5, HBM)
    assert df["bound"] == "hbm" and df["fp64_flop_per_launch"] == 0
    # the headline accept's DRAM traffic is scaled from the 64-walker capture
    assert math.isclose(df["traffic"], bench.ACCEPT_DF_TRAFFIC_PER_WALKER_N1024 * W)
    # complex128: 16-byte scalars, four real FMAs per complex one
    c = bench.accept_roofline(16, "native", 512, 4096, 1.0, HBM, s=16, cf=4)
    assert c["bytes_per_launch"] == 512 * 512 * 16 * 4096 and c["fp64_flop_per_launch"] == 4 * 2 * 512 * 512 * 4096


def test_pf_accept_propose_and_flush():
    n, W, K = 256, 1024, 8
    acc = bench.accept_roofline(0, "native", n, W, 0.32, HBM, pf=True)
    # exactly skew rank-2 update: 2 FMA per upper element, read the upper half, write both
    assert acc["fp64_flop_per_launch"] == 2 * n * n * W
    assert acc["bytes_per_launch"] == 1.5 * n * n * 8 * W
    assert acc["bound"] == "hbm"                                   # 0.118 ms at HBM > 0.107 ms at FP64 peak
    assert acc["traffic"] is None
    pro = bench.pf_propose_roofline(n, W, 0.18, HBM)
    assert pro["bytes_per_launch"] == n * n * 8 * W and pro["fp64_flop_per_launch"] == 2 * n * n * W
    assert pro["bound"] == "alu"                                   # 0.107 ms at FP64 peak > 0.079 ms at HBM
    prd = bench.pf_propose_roofline(n, W, 0.09, HBM, "df")        # double-float pass: FP32 pipe
    assert prd["bound"] == "hbm" and prd["fp64_flop_per_launch"] == 0
    assert bench.pf_propose_roofline(n, W, None, HBM) is None
    fl = bench.pf_flush_roofline("native", n, W, K, 2.66, HBM)
    # upper half of A_0^{-1} (mirrored), 2K slot columns per element
    assert math.isclose(fl["flop_per_full_flush"], 2 * (n * (n + 1) / 2) * 2 * K * W)
    assert fl["bytes_per_full_flush"] == 1.5 * n * n * 8 * W
    assert fl["bound"] == "alu" and math.isclose(fl["frac"], fl["achieved"] / FP64)
    fd = bench.pf_flush_roofline("df", n, W, K, 2.05, HBM)
    assert fd["bound"] == "hbm" and math.isclose(fd["frac"], fd["hbm"]["frac"])


def test_refresh_roofline_split_classes():
    n, W = 1024, 1024
    prof = {"refresh": (577.0, 2), "refresh_panel": (285.4, 2), "refresh_update": (278.2, 2)}
    r = bench.refresh_roofline(prof, n, W, 1687.2)
    p, u = r["panel"], r["update"]
    assert math.isclose(p["flop_per_refresh"], 2 * 64 * n * n * W)
    assert math.isclose(u["flop_per_refresh"], 78 * n ** 3 * W)     # 39 BF16 slice products of n x n x 64 per panel
    assert math.isclose(p["ms_per_refresh"], 142.7) and math.isclose(u["ms_per_refresh"], 139.1)
    assert math.isclose(u["fp64_equivalent_tflops"], 2 * n * n * (n - 64) * W / 0.1391 / 1e12)
    assert math.isclose(r["ms_per_launch"], 288.5)
    # the FP64 Gauss-Jordan form: n^3 FMA per walker
    g = bench.refresh_roofline({"refresh": (2300.0, 1)}, n, W, 1687.2)
    assert g["bound"] == "alu" and math.isclose(g["achieved"], 2 * n ** 3 * W / 2.3 / 1e12)
    assert bench.refresh_roofline({"refresh": (0.0, 0)}, n, W, 1687.2) is None


def test_drift_vs_plain_gates_near_nodes():
    ref = torch.tensor([[1.0, 2.0, 1e-9], [4.0, -1.0, 3.0]], dtype=torch.float64)
    other = ref.clone()
    other[0, 0] = 1.0 + 1e-8
    other[0, 2] = 5e-9                    # near a node: counted apart, not in the relative error
    arms = {"plain": {}, "delayed": {}}
    bench.drift_vs_plain({"plain": ref, "delayed": other}, arms)
    d = arms["delayed"]["ratio_err_vs_plain_fp64"]
    assert d["near_node_steps"] == 1
    assert math.isclose(d["max_rel"], 1e-8, rel_tol=1e-6)
    assert "ratio_err_vs_plain_fp64" not in arms["plain"]


def test_refresh_share_of_a_short_window():
    # 20 steps of a schedule that refreshes every 128 steps owe 20/128 of a
    # refresh; 256 steps hold both refreshes themselves; 300 steps hold two and
    # owe 44/128 of a third; no period, no share
    assert math.isclose(bench.refresh_share(20, 128), 20 / 128)
    assert bench.refresh_share(256, 128) == 0.0
    assert math.isclose(bench.refresh_share(300, 128), 44 / 128)
    assert bench.refresh_share(64, 0) == 0.0
