"""The benchmark's roofline arithmetic on the CPU.

The counts the JSON line reports are fixed by the workload: the benchmark performs 24 complex
64 x 64 products per pulse-step on the survey's count (K*d = 12 x 2 digit operators, 8N^3 flop
each, 50.3 MFLOP), the level table performs 12, and split FP16 runs 3 fp16 products per complex
product. The operand stream reads one 32 KB plane per product. GRAPE at N=256, K=16, M=1000
takes 2 products per digit factor: 8.6 TFLOP per iteration. These tests recompute the reported
figures from those counts for given times.
"""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"bf16_tflops_sustained": 1699.6, "bf16_tflops": 1908.8, "hbm_gbs": 6783.5}


def test_benchmark_chain_roofline_counts():
    B, M, N, K, d, t = 256, 2000, 64, 12, 2, 0.0330
    r = bench.chain_roofline(PEAKS, {}, B, M, N, K, d, K, t, "fp16x3", "chain_tc")
    per_step = K * d * 8 * N ** 3
    assert per_step == 50_331_648                                   # 50.3 MFLOP per pulse-step
    alg = B * M * per_step
    assert math.isclose(r["achieved"], alg / t / 1e12, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / 1699.6, rel_tol=1e-12)
    assert math.isclose(r["frac_of_burst"], r["achieved"] / 1908.8, rel_tol=1e-12)
    assert 0.45 < r["frac"] < 0.47                                  # the reported 0.46 at 33.0 ms
    assert math.isclose(r["method_products"]["achieved"], r["achieved"] / 2, rel_tol=1e-12)
    assert math.isclose(r["hardware_fp16"]["achieved"], 1.5 * r["achieved"], rel_tol=1e-12)
    s = r["hbm_operand_stream"]
    assert s["bytes_per_launch"] == B * M * K * 32768 == 201_326_592_000
    assert math.isclose(s["frac"], s["bytes_per_launch"] / t / 1e9 / 6783.5, rel_tol=1e-12)
    assert 0.89 < s["frac"] < 0.91                                  # the reported 0.90 of HBM
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["traffic"] is None


def test_other_precisions_use_their_own_pipes():
    r32 = bench.chain_roofline(PEAKS, {"sm_max_mhz": 2070.0}, 4, 10, 64, 12, 2, 24, 1e-3, "fp32", "chain")
    assert r32["bound"] == "alu" and math.isclose(r32["peak"], 152 * 128 * 2 * 2.07e9 / 1e12, rel_tol=1e-12)
    r64 = bench.chain_roofline(PEAKS, {}, 4, 10, 64, 12, 2, 24, 1e-3, "fp64", "chain")
    assert r64["peak"] == 1.25 and math.isclose(r64["frac"], r64["achieved"] / 1.25, rel_tol=1e-12)


def test_grape_flop_counts():
    class W:
        N, K, M, digits = 256, 16, 1000, 2
    ms = 15.04                                                      # 66.5 iterations/s
    gflop = 2 * W.M * W.K * 8.0 * W.N ** 3                         # level table: 2 products per factor
    gres = {"fp16x3": {"ms_per_iter": ms, "iters_per_s": 1e3 / ms}}
    g = bench.grape_summary(gres, gflop, 0.8, W, PEAKS)
    alg = g["flop_counts"]["algorithmic"]
    assert math.isclose(alg["tflop_per_iteration"], 2 * 1000 * 32 * 8 * 256 ** 3 / 1e12, rel_tol=1e-12)
    assert 8.58 < alg["tflop_per_iteration"] < 8.60                 # 8.6 TFLOP per iteration
    assert math.isclose(g["flop_counts"]["method_level_table"]["tflop_per_iteration"], 4.294967296, rel_tol=1e-12)
    assert math.isclose(g["flop_counts"]["hardware_fp16"]["tflop_per_iteration"], 3 * 4.294967296, rel_tol=1e-12)
    assert math.isclose(g["roofline"]["frac_of_sustained"], alg["tflop_per_iteration"] / (ms / 1e3) / 1699.6,
                        rel_tol=1e-12)
    assert 0.33 < g["roofline"]["frac_of_sustained"] < 0.34          # the reported 0.336
