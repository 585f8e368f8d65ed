#!/usr/bin/env python3
"""Benchmark: REDO propagation throughput on the batched N=64 workload.

Workload (one "step"): B=256 independent pulses on a 6-qubit NMR-like system
(N=64, K=12 per-qubit x/y controls), M=2000 piecewise-constant steps of 1 us,
coefficients uniform on [-Omega, Omega] with 4096 levels (base 64, 2 digits).
A step quantizes the coefficients, forms every pulse's REDO propagator
U = U_M ... U_1 from the discrete-operator table and reduces its fidelity
against a Haar-random target.  The table is built once, outside the timed
region (it is the one-time process of the method).

Reports one JSON line (rank 0).  ``--impl reference`` times the CPU FP64
oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "REDO prop steps/s & GRAPE iters/s vs FP64 plain REDO, same GB300, |ΔF|≤1e-6"
UNIT = "pulse-steps/s"
B_FULL, M_FULL, N_QUBITS = 256, 2000, 6
MAIN_PREC = os.environ.get("REDO_BENCH_PREC", "fp16x3")
REUNIT = 64          # re-unitarisation period (steps) of the reduced-precision forms


def _workload_config(extra=None):
    cfg = {"workload": "batched REDO propagation: N=64 (6 qubits), K=12 x/y controls, B=256 pulses, "
                       "M=2000 steps of 1 us, 4096 levels (b=64, d=2), fidelity vs Haar target",
           "B": B_FULL, "M": M_FULL, "N": 64, "K": 12, "levels": 4096, "base": 64, "digits": 2,
           "seed": 1}
    if extra:
        cfg.update(extra)
    return cfg


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.gpu_index = gpu_index
        # raw samples go to REDO_CLOCKS_DIR (default: the system temporary directory); the JSON
        # line carries their summary
        out_dir = os.environ.get("REDO_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                                 parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle (CPU)

def _oracle_worker(args):
    seed_pulse, M_sample = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import redo_oracle as O
    from paper_1707_02162_gb300 import inputs
    w = inputs.config(1, B=1, M=M_sample, seed=1)
    rng = np.random.default_rng(1000 + seed_pulse)
    u = rng.uniform(w.lo[0], w.hi[0], size=(1, M_sample, w.K))
    T, D = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits)
    t0 = time.perf_counter()
    q, _, _ = O.quantize(u, w.lo, w.hi, w.levels)
    dig = O.level_digits(q, w.base, w.digits)
    U = O.propagate(T, D, dig[0])
    F = O.fidelity(w.target, U)
    dt = time.perf_counter() - t0
    return dt, M_sample, F


def _oracle_parity_worker(pulse):
    """The oracle's propagator of one whole pulse of the benchmark workload (all M steps)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import redo_oracle as O
    from paper_1707_02162_gb300 import inputs
    w = inputs.config(1, B=B_FULL, M=M_FULL, seed=1)
    T, D = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits, method="eig")
    q, _, _ = O.quantize(w.u[pulse:pulse + 1], w.lo, w.hi, w.levels)
    U = O.propagate(T, D, O.level_digits(q, w.base, w.digits)[0])
    return pulse, U, O.fidelity(w.target, U)


def oracle_parity(pulses):
    """Oracle propagators of the given pulses, one spawn worker each (the CPU leg of the run)."""
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(len(pulses)) as pool:
            res = pool.map(_oracle_parity_worker, list(pulses))
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {p: (U, F) for p, U, F in res}


def oracle_throughput(cores=None, M_sample=600):
    """Oracle pulse-steps/s over `cores` spawn workers, one pulse of M_sample steps each."""
    cores = cores or os.cpu_count() or 1
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            res = pool.map(_oracle_worker, [(i, M_sample) for i in range(cores)])
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    elapsed = max(r[0] for r in res)
    steps = sum(r[1] for r in res)
    return {"value": steps / elapsed, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} pulses x {M_sample} steps of the same N=64, K=12 system (one pulse per worker "
                      f"process, numpy FP64 oracle, single-threaded BLAS); quantize + product chain + fidelity; "
                      f"wall {elapsed:.2f} s"}


# ----------------------------------------------------------------------------- GPU arm

def _dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def chain_roofline(peaks, clk, B, M, N, K, digits, prods_per_step, avg_s, prec, kernel):
    """Roofline of one chain-kernel launch over B pulses x M steps.

    The algorithmic count is the method's as the survey of the paper states it: K*digits complex
    N x N products per pulse-step (the digit operators of Eq. exp2prod), 8N^3 flop each.  With the
    level table the call performs K products per pulse-step (process 3 applied to every level),
    and the split-FP16 form runs 3 fp16 products per complex product; both are reported beside it.
    """
    n3 = 8.0 * N ** 3
    alg_flop = B * M * K * digits * n3
    method_flop = B * M * prods_per_step * n3
    alg_tf = alg_flop / avg_s / 1e12
    out = {"kernel": kernel, "launch_ms": avg_s * 1e3,
           "algorithmic_per_launch": (f"{alg_flop:.4g} flop: B*M*{K * digits} complex {N}x{N} products "
                                      f"(K*d digit operators per pulse-step), 8N^3 each"),
           "traffic": None}
    if prec == "fp16x3":
        sus = peaks.get("bf16_tflops_sustained", 1699.6)
        burst = peaks.get("bf16_tflops", 1908.8)
        op_bytes = B * M * prods_per_step * 32768.0            # one 32 KB split-FP16 operand per product
        out.update({"bound": "tensor", "unit": "TFLOP/s", "achieved": alg_tf, "peak": sus,
                    "peak_source": "measured dense bf16, sustained (of measured; fp16 has the same nominal rate)",
                    "frac": alg_tf / sus, "frac_of_burst": alg_tf / burst,
                    "method_products": {"what": f"{prods_per_step} complex products per pulse-step as performed",
                                        "achieved": method_flop / avg_s / 1e12,
                                        "frac": method_flop / avg_s / 1e12 / sus},
                    "hardware_fp16": {"what": "3 fp16 products per complex product (split operands)",
                                      "achieved": 3 * method_flop / avg_s / 1e12,
                                      "frac": 3 * method_flop / avg_s / 1e12 / sus},
                    "hbm_operand_stream": {"bytes_per_launch": op_bytes, "achieved_gbs": op_bytes / avg_s / 1e9,
                                           "peak_gbs": peaks.get("hbm_gbs", 6783.5),
                                           "frac": op_bytes / avg_s / 1e9 / peaks.get("hbm_gbs", 6783.5)}})
    elif prec == "fp32":
        clk_max = (clk.get("sm_max_mhz") or 2070.0) * 1e6
        peak = 152 * 128 * 2 * clk_max / 1e12
        out.update({"bound": "alu", "unit": "TFLOP/s", "achieved": alg_tf, "peak": peak, "frac": alg_tf / peak,
                    "peak_source": "FP32 FMA pipe: 152 SMs x 128 lanes x 2 flop x max SM clock"})
    else:
        out.update({"bound": "alu", "unit": "TFLOP/s", "achieved": alg_tf, "peak": 1.25, "frac": alg_tf / 1.25,
                    "peak_source": "nominal GB300 FP64"})
    return out


def grape_summary(gres, gflop, gbuild, gw, peaks):
    """GRAPE iterations/s on the N=256 workload with the three flop counts side by side."""
    ms = gres["fp16x3"]["ms_per_iter"]
    sus = peaks.get("bf16_tflops_sustained", 1699.6)
    n3 = 8.0 * gw.N ** 3
    survey = 2 * gw.M * gw.K * gw.digits * n3            # 2 products per digit factor (forward, costate)
    counts = {"algorithmic": (survey, "2 complex products per digit factor per step (K*d = "
                                      f"{gw.K * gw.digits} factors), 8N^3 each"),
              "method_level_table": (gflop, f"2 complex products per level factor ({gw.K} per step)"),
              "hardware_fp16": (3 * gflop, "x3 fp16 products per complex product")}
    flops = {k: {"tflop_per_iteration": v / 1e12, "achieved_tflops": v / (ms / 1e3) / 1e12,
                 "frac_of_sustained": v / (ms / 1e3) / 1e12 / sus, "what": what}
             for k, (v, what) in counts.items()}
    return {"metric": "GRAPE iters/s", "value": gres["fp16x3"]["iters_per_s"], "unit": "iterations/s",
            "workload": "GRAPE gradient + update, N=256 (8 qubits), K=16, M=1000, dt=2 us, Haar target, "
                        "checkpoints every 32 steps, level table (one operator per control level)",
            "fp64_plain_redo": gres.get("fp64"),
            "speedup_vs_fp64": (gres["fp16x3"]["iters_per_s"] / gres["fp64"]["iters_per_s"]
                                if "fp64" in gres else None),
            "roofline": dict(flops["algorithmic"], bound="tensor", peak=sus, unit="TFLOP/s",
                             peak_source="measured dense bf16, sustained (of measured)"),
            "flop_counts": flops, "phase_ms": gres["fp16x3"].get("phase_ms"), "table_build_s": gbuild}


def precision_table(forms, oracle):
    """max |U - U_oracle| and |F - F_oracle| of every precision form on the sampled pulses."""
    table = {}
    for prec, val in forms.items():
        if prec == "pulses":
            continue
        Ug, Fg, reunit = val
        dU = max(float(np.abs(Ug[i] - oracle[p][0]).max()) for i, p in enumerate(forms["pulses"]))
        dF = max(abs(float(Fg[i]) - oracle[p][1]) for i, p in enumerate(forms["pulses"]))
        table[prec] = {"max_abs_dU": dU, "max_abs_dF": dF, "reunit_every": reunit}
    table["tf32"] = "not offered: a TF32 chain emulated on this system misses the entry budget by ~30x"
    table["pulses"] = forms["pulses"]
    table["what"] = ("error of each product-chain form against the CPU FP64 oracle's chain, whole pulses of "
                     "the timed workload (all 2000 steps)")
    return table


def plain_measure(redo, inputs, torch, reps=5):
    """Plain REDO on the 3-qubit system (N=8, K=2 global x/y, M=1000, FP64): one pulse (latency)
    and 4096 replica pulses (throughput), with the FP32 form beside each."""
    res = {}
    for B in (1, 4096):
        w = inputs.config(0, B=B)
        t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
        u = torch.tensor(w.u, device="cuda")
        target = torch.as_tensor(w.target, device="cuda")
        q = torch.empty(u.shape, dtype=torch.int32, device="cuda")
        U = torch.empty((B, w.N, w.N), dtype=torch.complex128, device="cuda")
        F = torch.empty(B, dtype=torch.float64, device="cuda")
        tau = torch.empty(B, dtype=torch.complex128, device="cuda")
        for prec in ("fp64", "fp32"):
            ws = t.workspace(B, w.M, prec)

            def it():
                redo.redo_quantize(t.handle, u, q)
                redo.redo_propagate(t.handle, q, prec, U, target, F, tau, ws)
            it()
            ms = _events_time(it, reps)
            # 4 complex 8x8 products per pulse-step: K*d = 4 digit operators, the drift folded in
            flop = B * w.M * w.K * w.digits * 8.0 * w.N ** 3
            peak = 1.25 if prec == "fp64" else 152 * 128 * 2 * 2.07e9 / 1e12
            res[f"B{B}_{prec}"] = {"pulse_steps_per_s": B * w.M / (ms / 1e3), "ms_per_call": ms,
                                   "roofline": {"bound": "alu", "unit": "TFLOP/s",
                                                "achieved": flop / (ms / 1e3) / 1e12, "peak": peak,
                                                "frac": flop / (ms / 1e3) / 1e12 / peak,
                                                "peak_source": ("nominal GB300 FP64" if prec == "fp64" else
                                                                "FP32 FMA pipe: 152 x 128 lanes x 2 x 2.07 GHz"),
                                                "timed": "whole call (quantize, chain, combine, fidelity)"}}
        t.close()
    return {"metric": "REDO prop steps/s, plain REDO FP64 (N=8)", "unit": "pulse-steps/s",
            "workload": "3 qubits (N=8), K=2 global x/y controls, M=1000 steps of 1 us, 4096 levels, "
                        "FP64, Haar target; B=1 and 4096 replica pulses",
            "value": res["B1_fp64"]["pulse_steps_per_s"], "replicas_4096_fp64": res["B4096_fp64"]["pulse_steps_per_s"],
            "results": res}


def ensemble_measure(redo, inputs, torch, peaks, M=2000):
    """Noisy-drive ensemble: 10-qubit ZZ chain (N=1024), global x drive Omega(1 + xi(t)) with OU
    noise, 64 realisations x M steps: <Z_1>(t) from |0...0> plus every final propagator in split
    FP16, and <Z_1>(t) in FP64 (state only) for its error.  Primary: the level table (each of the
    4096 levels' operators evaluated once, process 3: one product per step); beside it the digit
    table (two products per step)."""
    w = inputs.config(3, M=M)
    steps = w.B * M
    alg = steps * w.K * w.digits * 8.0 * w.N ** 3          # 2 complex 1024x1024 products per realisation-step
    sus = peaks.get("bf16_tflops_sustained", 1699.6)
    res = {}
    for levels in (True, False):
        t0 = time.time()
        t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=False, fp16x3=True, levels=levels)
        torch.cuda.synchronize()
        build_s = time.time() - t0
        q = t.quantize(w.u)
        psi0 = torch.as_tensor(w.psi0, device="cuda")
        obs = torch.as_tensor(w.obs_diag, device="cuda")
        ex16 = torch.empty((w.B, M + 1), dtype=torch.float64, device="cuda")
        ex64 = torch.empty((w.B, M + 1), dtype=torch.float64, device="cuda")
        Uf = torch.empty((w.B, w.N, w.N), dtype=torch.complex128, device="cuda")
        ws16 = torch.empty(max(redo.redo_simulate_workspace(t.handle, w.B, M, "fp16x3", 0, True), 256),
                           dtype=torch.uint8, device="cuda")
        ws64 = torch.empty(max(redo.redo_simulate_workspace(t.handle, w.B, M, "fp64", 0, False), 256),
                           dtype=torch.uint8, device="cuda")
        run16 = lambda: redo.redo_simulate(t.handle, q, "fp16x3", 0, psi0, obs, ex16, Uf, ws16)
        run64 = lambda: redo.redo_simulate(t.handle, q, "fp64", 0, psi0, obs, ex64, None, ws64)
        run16()
        ms16 = _events_time(run16, 1)
        ms64 = _events_time(run64, 1)
        res["level_table" if levels else "digit_table"] = {
            "realisation_steps_per_s": steps / (ms16 / 1e3), "ms_per_call": ms16,
            "products_per_step": w.K * (1 if levels else w.digits),
            "fp64_state_only": {"realisation_steps_per_s": steps / (ms64 / 1e3), "ms_per_call": ms64},
            "max_abs_dZ1_fp16x3_vs_fp64": float((ex16 - ex64).abs().max()),
            "tensor_frac_algorithmic": alg / (ms16 / 1e3) / 1e12 / sus,
            "table_build_s": build_s}
        t.close()
        del ws16, ws64, Uf
    lv = res["level_table"]
    return {"metric": "REDO prop steps/s (noisy-drive ensemble, propagators + <Z_1>(t))", "unit": "realisation-steps/s",
            "workload": "10-qubit ZZ chain (N=1024), K=1 global x drive Omega(1+xi), OU sigma=0.1 tau=50 us, "
                        f"64 realisations x {M} steps of 1 us, 4096 levels",
            "value": lv["realisation_steps_per_s"], "ms_per_call": lv["ms_per_call"],
            "precision": "fp16x3 products, fp32 state path", "results": res,
            "roofline": {"bound": "tensor", "unit": "TFLOP/s", "peak": sus,
                         "peak_source": "measured dense bf16, sustained (of measured)",
                         "achieved": alg / (lv["ms_per_call"] / 1e3) / 1e12,
                         "frac": alg / (lv["ms_per_call"] / 1e3) / 1e12 / sus, "timed": "whole call",
                         "algorithmic_per_call": f"{alg:.4g} flop (2 complex digit-operator products of 8N^3 per "
                                                 "realisation-step)"}}


def run_gpu(args):
    import torch
    world, rank, local = _dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1707_02162_gb300 import build as _b
    _b.build()
    from paper_1707_02162_gb300 import inputs, redo
    import json as _json
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = _json.load(open(pk))

    # Each rank runs an independent replica batch (weak scaling, no collective on the data path).
    from paper_1707_02162_gb300.replicas import aggregate_throughput, replica_seed
    w = inputs.config(1, seed=1, B=args.B, M=args.M)
    if rank:
        w.u = np.random.default_rng(replica_seed(1, rank)).uniform(w.lo[0], w.hi[0], size=w.u.shape)
    dev = torch.device("cuda", local)
    table = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True,
                       fp16x3=(MAIN_PREC == "fp16x3"), levels=args.levels)
    prods_per_step = w.K * (1 if args.levels else w.digits)
    u_host = torch.from_numpy(w.u).pin_memory()
    u_dev = u_host.to(dev)
    target = torch.as_tensor(w.target, device=dev)
    B, M, N = w.B, w.M, w.N
    q = torch.empty(u_dev.shape, dtype=torch.int32, device=dev)
    U = torch.empty((B, N, N), dtype=torch.complex128, device=dev)
    F = torch.empty(B, dtype=torch.float64, device=dev)
    tau = torch.empty(B, dtype=torch.complex128, device=dev)
    status = redo.new_status(dev)
    reunit_main = 0 if MAIN_PREC == "fp64" else REUNIT
    ws = table.workspace(B, M, MAIN_PREC, reunit_main)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)      # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step(prec=MAIN_PREC, qq=q, UU=U, FF=F, tt=tau, uu=u_dev, wsp=ws, reunit=reunit_main):
        redo.redo_quantize(table.handle, uu, qq, status)
        redo.redo_propagate(table.handle, qq, prec, UU, target, FF, tt, wsp, status, reunit_every=reunit)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    redo.redo_profile_read()
    redo.redo_profile_enable(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    for i in range(args.steps):
        flush.zero_()                               # L2 flushed between timed steps (outside the events)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    redo.redo_profile_enable(False)
    prof = redo.redo_profile_read()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, total_s = aggregate_throughput(float(B * M * args.steps), sum(step_ms) / 1e3)
    ms_per_step = total_s * 1e3 / args.steps

    st = status.cpu().numpy()
    # parity guard on the measured run: F of two pulses against FP64 GPU path is checked in tests;
    # here we only refuse to report if the device flagged a timeout or a bad index.
    assert st[2] == 0 and st[3] == 0, f"device status {st}"

    # ---- roofline of the dominant kernel (the chain kernel)
    seg_ms, seg_n = prof.get("chain_segments", (0.0, 0))
    tc_ms, tc_n = prof.get("chain_tc", (0.0, 0))
    if tc_n:
        dom_ms, dom_n, dom_name = tc_ms, tc_n, "chain_tc"
    else:
        dom_ms, dom_n, dom_name = seg_ms, seg_n, "chain_segments"
    avg_s = (dom_ms / max(dom_n, 1)) / 1e3
    roof = chain_roofline(peaks, clk, B, M, N, w.K, w.digits, prods_per_step, avg_s, MAIN_PREC, dom_name)

    # ---- end to end through the C ABI with host buffers (right after the timed steps, before the
    # FP64 comparison arm, so that both see the same clocks)
    e2e = None
    if not args.skip_e2e:
        U_host = torch.empty((B, N, N), dtype=torch.complex128).pin_memory()
        F_host = torch.empty(B, dtype=torch.float64).pin_memory()
        step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        reps = max(1, args.steps)
        for _ in range(reps):
            u_dev.copy_(u_host, non_blocking=True)
            step()
            U_host.copy_(U, non_blocking=True)
            F_host.copy_(F, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        e_ms = a.elapsed_time(b) / reps
        e2e = {"value": world * B * M / (e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(u_host.numel() * 8),
               "d2h_bytes_per_step": int(U_host.numel() * 16 + F_host.numel() * 8)}

    # ---- FP64 plain REDO on the same GPU (subset of pulses, same steps)
    fp64 = None
    if rank == 0 and not args.skip_fp64:
        Bs = 16
        qs = q[:Bs].contiguous()
        Us = torch.empty((Bs, N, N), dtype=torch.complex128, device=dev)
        Fs = torch.empty(Bs, dtype=torch.float64, device=dev)
        ts = torch.empty(Bs, dtype=torch.complex128, device=dev)
        ws64 = table.workspace(Bs, M, "fp64")
        us = u_dev[:Bs].contiguous()
        step("fp64", qs, Us, Fs, ts, us, ws64, 0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        a.record(stream)
        for _ in range(reps):
            step("fp64", qs, Us, Fs, ts, us, ws64, 0)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b) / reps
        fp64_val = Bs * M / (ms64 / 1e3)
        dF = float((Fs - F[:Bs]).abs().max().item())
        dU = float((Us - U[:Bs]).abs().max().item())
        fp64 = {"value": fp64_val, "unit": UNIT, "sample": f"{Bs} of the {B} pulses, all {M} steps",
                "speedup_of_main": value / world / fp64_val,
                "main_vs_fp64_max_abs_dF": dF, "main_vs_fp64_max_abs_dU": dU}

    grape = None
    if rank == 0 and not args.skip_grape:
        gres, gflop, gbuild, gw = grape_measure(redo, inputs, torch, 3, levels=True, with_fp32=False,
                                                with_fp64=not args.skip_fp64)
        grape = grape_summary(gres, gflop, gbuild, gw, peaks)

    # ---- each precision form on sampled pulses, for their error against the oracle (CPU leg)
    forms = None
    if rank == 0 and not args.skip_cpu and (B, M) == (B_FULL, M_FULL):
        picks = [0, 131]
        forms = {"pulses": picks, MAIN_PREC: (U[picks].cpu().numpy(), F[picks].cpu().numpy(), reunit_main)}
        qp = q[picks].contiguous()
        for prec, reunit in (("fp64", 0), ("fp32", REUNIT)):
            if prec == MAIN_PREC:
                continue
            Up = torch.empty((len(picks), N, N), dtype=torch.complex128, device=dev)
            Fp = torch.empty(len(picks), dtype=torch.float64, device=dev)
            redo.redo_propagate(table.handle, qp, prec, Up, target, Fp, None,
                                table.workspace(len(picks), M, prec, reunit), status, reunit_every=reunit)
            forms[prec] = (Up.cpu().numpy(), Fp.cpu().numpy(), reunit)

    plain = ensemble = None
    if rank == 0 and not args.skip_extra:
        plain = plain_measure(redo, inputs, torch)
        ensemble = ensemble_measure(redo, inputs, torch, peaks)

    launches = sum(n for _, n in prof.values())
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "fp16x3": "f16x3 (f32 accumulate)"}[MAIN_PREC],
           "data": "synthetic (seeded NMR-like Hamiltonian, uniform random controls, Haar target)",
           "config": _workload_config({"precision": MAIN_PREC, "B": B, "M": M, "reunit_every": reunit_main,
                                       "table": ("level table (process 3): K products per step" if args.levels
                                                 else "digit table: K*d products per step"),
                                       "l2": "flushed between timed steps (256 MB write outside the events)"}),
           "roofline": roof, "e2e": e2e, "gpu_launches": int(launches),
           "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
           "fp64_plain_redo": fp64, "grape": grape, "plain_n8": plain, "ensemble_n1024": ensemble,
           "clocks": clk}
    if rank == 0 and not args.skip_cpu:
        out["cpu_baseline"] = oracle_throughput()
        if forms is not None:
            out["precision_vs_oracle"] = precision_table(forms, oracle_parity(sorted(forms["pulses"])))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        emit(out, args)


def emit(out: dict, args) -> None:
    """Print the run's JSON line; with ``--jsonl PATH`` also append it to that file."""
    line = json.dumps(out)
    print(line)
    if getattr(args, "jsonl", None):
        with open(args.jsonl, "a") as f:
            f.write(line + "\n")


def run_reference(args):
    world, rank, _ = _dist_env()
    if rank != 0:
        return
    per = []
    info = None
    for i in range(args.warmup + args.steps):
        r = oracle_throughput(M_sample=200)
        if i >= args.warmup:
            per.append(r["value"])
            info = r
    value = statistics.median(per)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": B_FULL * M_FULL / value * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded NMR-like Hamiltonian, uniform random controls, Haar target)",
           "config": _workload_config({"precision": "fp64 (CPU oracle)",
                                       "sample": "each step times a bounded sample; ms_per_step is extrapolated "
                                                 "to the full workload"}),
           "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": info["cores"],
                            "sample": info["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(out, args)


# ----------------------------------------------------------------------------- other workloads
# One JSON line each; the driver's default run is the batched-propagation line above.

def _peaks() -> dict:
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(pk)) if os.path.exists(pk) else {}


def _events_time(fn, reps):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def grape_measure(redo, inputs, torch, steps, levels=False, with_fp32=True, with_fp64=True, M=None):
    """GRAPE iterations/s on the 8-qubit (N=256), K=16, M=1000, dt=2 us workload, B=1, checkpoints
    every 32 steps: split FP16 on tensor cores, optionally FP32 SIMT and FP64 plain REDO."""
    w = inputs.config(2, M=M)
    t0 = time.time()
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=True, levels=levels)
    build_s = time.time() - t0
    u = torch.tensor(w.u, device="cuda")
    target = torch.as_tensor(w.target, device="cuda")
    q = torch.empty(u.shape, dtype=torch.int32, device="cuda")
    F = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty(u.shape, dtype=torch.float64, device="cuda")
    res = {}
    precs = [("fp16x3", steps)] + ([("fp32", steps)] if with_fp32 else []) + ([("fp64", 1)] if with_fp64 else [])
    for prec, reps in precs:
        ws = torch.empty(redo.redo_fidelity_grad_workspace(t.handle, 1, w.M, prec, 32), dtype=torch.uint8,
                         device="cuda")

        def it():
            redo.redo_quantize(t.handle, u, q)
            redo.redo_fidelity_grad(t.handle, q, target, prec, 32, F, g, ws)
            redo.redo_grape_step(t.handle, u, g, 1e9)
        it()
        ms = _events_time(it, reps)
        res[prec] = {"iters_per_s": 1e3 / ms, "ms_per_iter": ms, "timed_iterations": reps}
        if prec == "fp16x3":
            # one more iteration with the library's phase events (outside the timed ones)
            redo.redo_profile_read()
            redo.redo_profile_enable(True)
            it()
            redo.redo_profile_enable(False)
            res[prec]["phase_ms"] = {k: round(v[0], 3) for k, v in redo.redo_profile_read().items()}
        del ws
    t.close()
    # two complex products per factor: the forward sweep (every state kept) and the costate sweep
    flop = 2 * w.M * w.K * (1 if levels else w.digits) * 8.0 * w.N ** 3
    return res, flop, build_s, w


def run_workload(args):
    import torch
    torch.cuda.set_device(0)
    from paper_1707_02162_gb300 import build as _b
    _b.build()
    from paper_1707_02162_gb300 import inputs, redo
    out = {"workload": args.workload, "n_gpus": 1, "data": "synthetic"}
    if args.workload == "grape":
        res, flop, build_s, w = grape_measure(redo, inputs, torch, args.steps, levels=args.levels,
                                              with_fp32=not args.skip_fp64, with_fp64=not args.skip_fp64,
                                              M=args.M if args.M != M_FULL else None)
        out.update({"metric": "GRAPE iters/s", "unit": "iterations/s", "value": res["fp16x3"]["iters_per_s"],
                    "precision": "fp16x3 (tcgen05 lockstep chains, FP32 accumulate)", "fp32_simt": res.get("fp32"),
                    "fp64_plain_redo": res.get("fp64"),
                    "speedup_vs_fp64": (res["fp16x3"]["iters_per_s"] / res["fp64"]["iters_per_s"]
                                        if "fp64" in res else None),
                    "phase_ms": res["fp16x3"].get("phase_ms"),
                    "algorithmic_flop_per_iter": flop,
                    "achieved_tensor_tflops_fp16x3": 3 * flop / (res["fp16x3"]["ms_per_iter"] / 1e3) / 1e12,
                    "achieved_tflops_fp32": (flop / (res["fp32"]["ms_per_iter"] / 1e3) / 1e12
                                             if "fp32" in res else None),
                    "table_build_s": build_s,
                    "config": {"N": w.N, "K": w.K, "M": w.M, "dt": w.dt, "checkpoint_every": 32, "B": 1,
                               "table": "level table" if args.levels else "digit table"}})
    elif args.workload == "sim":
        # 10-qubit ZZ chain (N=1024), global X drive with OU noise, 64 realisations; M_sample steps timed
        Ms = args.M if args.M != M_FULL else 40
        w = inputs.config(3, M=Ms, B=args.B if args.B != B_FULL else None, n_qubits=args.nq)
        t0 = time.time()
        t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=True)
        build_s = time.time() - t0
        q = t.quantize(w.u)
        psi0 = torch.as_tensor(w.psi0, device="cuda")
        obs = torch.as_tensor(w.obs_diag, device="cuda")
        ex = torch.empty((w.B, Ms + 1), dtype=torch.float64, device="cuda")
        Uf = torch.empty((w.B, w.N, w.N), dtype=torch.complex128, device="cuda")
        res = {}
        for prec, want in (("fp16x3", True), ("fp32", False), ("fp32", True), ("fp64", False)):
            nb = redo.redo_simulate_workspace(t.handle, w.B, Ms, prec, 0, want)
            ws = torch.empty(max(nb, 256), dtype=torch.uint8, device="cuda")

            def it():
                redo.redo_simulate(t.handle, q, prec, 0, psi0, obs, ex, Uf if want else None, ws)
            it()
            ms = _events_time(it, 1)
            res[f"{prec}{'_with_U' if want else '_state_only'}"] = {
                "realisation_steps_per_s": w.B * Ms / (ms / 1e3), "ms": ms}
        flop_step = 3 * w.K * w.digits * 8.0 * w.N ** 3
        out.update({"metric": "REDO prop steps/s (noisy-drive ensemble)", "unit": "realisation-steps/s",
                    "value": res["fp16x3_with_U"]["realisation_steps_per_s"], "results": res,
                    "achieved_tensor_tflops_fp16x3": flop_step * res["fp16x3_with_U"]["realisation_steps_per_s"] / 1e12,
                    "tensor_frac_of_sustained": (flop_step * res["fp16x3_with_U"]["realisation_steps_per_s"] / 1e12
                                                 / _peaks().get("bf16_tflops_sustained", 1709.6)),
                    "sample": f"{Ms} of the 2000 steps, all 64 realisations", "table_build_s": build_s,
                    "config": {"N": w.N, "K": w.K, "B": w.B, "M_timed": Ms}})
    elif args.workload == "freeze":
        # Section IV noisy exotic freezing: 3-spin Ising chain, Q(omega, lambda) over 500 omegas in
        # [1, 25] rad/s x 1000 lambdas in [0, 1], 10^4 steps on [0, 20 pi], coefficient grid b=100, d=2.
        # The drive h0{(1-lambda) cos(omega t_n) + lambda eta_n} is synthesised on the device
        # (eta_n uniform on [-1, 1] from a seeded Philox generator), pulses omega-major.
        n_om = args.B if args.B != B_FULL else 500
        n_la = 1000
        M = args.M if args.M != M_FULL else 10000
        h0, Tw = inputs.FREEZE_H0_AMP, inputs.FREEZE_T
        H0, Hk, rho, obs = inputs.freezing_system(3, h0, basis="x")
        t = redo.Table(H0, Hk, Tw / M, np.array([-h0]), np.array([h0]), 100, 2, fp32=True)
        rho_d = torch.as_tensor(rho, device="cuda")
        obs_d = torch.as_tensor(obs, device="cuda")
        oms = torch.linspace(1.0, 25.0, n_om, dtype=torch.float64, device="cuda")
        las = torch.linspace(0.0, 1.0, n_la, dtype=torch.float64, device="cuda")
        tn = (torch.arange(M, dtype=torch.float64, device="cuda") + 0.5) * (Tw / M)
        gen = torch.Generator(device="cuda").manual_seed(5)
        chunk_om = max(1, min(n_om, 100))      # 100 000 pulses per launch: ten waves of CTAs
        Qmap = torch.empty((n_om, n_la), dtype=torch.float64, device="cuda")
        kern_ms = 0.0
        ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.time()
        for i0 in range(0, n_om, chunk_om):
            om = oms[i0:i0 + chunk_om]
            Bc = om.numel() * n_la
            eta = torch.rand((Bc, M), dtype=torch.float64, device="cuda", generator=gen) * 2.0 - 1.0
            la = las.repeat(om.numel())[:, None]
            u = (h0 * ((1.0 - la) * torch.cos(om.repeat_interleave(n_la)[:, None] * tn[None, :]) + la * eta))[:, :, None]
            del eta
            q = torch.empty(u.shape, dtype=torch.int32, device="cuda")
            mean = torch.empty(Bc, dtype=torch.float64, device="cuda")
            ev_a.record()
            redo.redo_quantize(t.handle, u.contiguous(), q)
            redo.redo_expect_diag(t.handle, q, "fp32", rho_d, obs_d, None, mean)
            ev_b.record()
            torch.cuda.synchronize()
            kern_ms += ev_a.elapsed_time(ev_b)
            Qmap[i0:i0 + om.numel()] = (mean / float(np.sum(rho * obs))).reshape(om.numel(), n_la)
            del u, q
        wall = time.time() - t0
        # same-GPU FP64 on the first omega's 1000 pulses (context for the FP32 map)
        om = oms[:1]
        eta = torch.rand((n_la, M), dtype=torch.float64, device="cuda", generator=gen) * 2.0 - 1.0
        u = (h0 * ((1.0 - las[:, None]) * torch.cos(om[0] * tn[None, :]) + las[:, None] * eta))[:, :, None].contiguous()
        q = torch.empty(u.shape, dtype=torch.int32, device="cuda")
        redo.redo_quantize(t.handle, u, q)
        mean64 = torch.empty(n_la, dtype=torch.float64, device="cuda")
        ev_a.record()
        redo.redo_expect_diag(t.handle, q, "fp64", rho_d, obs_d, None, mean64)
        ev_b.record()
        torch.cuda.synchronize()
        fp64_rate = n_la * M / (ev_a.elapsed_time(ev_b) / 1e3)
        mean32 = torch.empty(n_la, dtype=torch.float64, device="cuda")
        redo.redo_expect_diag(t.handle, q, "fp32", rho_d, obs_d, None, mean32)
        fp32_vs_fp64 = float((mean32 - mean64).abs().max() / float(np.sum(rho * obs)))
        Q0 = Qmap[:, 0].cpu().numpy()
        omh = oms.cpu().numpy()
        from scipy.special import jn_zeros
        roots = [2 * h0 / z for z in jn_zeros(0, 4)]
        peaks = {}
        for r in roots:
            sel = np.abs(omh - r) < 0.4
            if sel.any():
                peaks[f"{r:.3f}"] = {"omega_at_max_Q": float(omh[sel][np.argmax(Q0[sel])]), "max_Q": float(Q0[sel].max())}
        steps = n_om * n_la * M
        out.update({"metric": "noisy exotic freezing Q(omega, lambda) map: pulse-steps/s", "unit": "pulse-steps/s",
                    "value": steps / (kern_ms / 1e3), "kernel_ms": kern_ms, "wall_s_with_drive_synthesis": wall,
                    "precision": "fp32 chains, fp64 reductions", "pulses": n_om * n_la, "steps": M,
                    "fp64_same_gpu": {"pulse_steps_per_s": fp64_rate, "sample": f"{n_la} pulses x {M} steps",
                                      "max_abs_dQ_fp32_vs_fp64": fp32_vs_fp64},
                    "lambda0_peaks_vs_bessel_roots": peaks,
                    "Q_mean_lambda1": float(Qmap[:, -1].mean()), "Q_mean_lambda0": float(Q0.mean()),
                    "config": {"N": 8, "K": 1, "h0": h0, "J": h0 / 20, "omegas": [1.0, 25.0, n_om],
                               "lambdas": [0.0, 1.0, n_la], "T": Tw, "base": 100, "digits": 2}})
    elif args.workload == "state":
        # state-to-state GRAPE on the 8-qubit GRAPE system (N=256, K=16, M=1000, dt=2 us): fidelity +
        # gradient per pulse by matrix-vector sweeps; one pulse and a batch of 152 (one CTA each)
        w = inputs.config(2, M=args.M if args.M != M_FULL else None)
        t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, levels=not args.digit_table)
        res = {}
        for B in (1, 152):
            rng = np.random.default_rng(2)
            u = torch.tensor(rng.uniform(w.lo[0], w.hi[0], size=(B, w.M, w.K)), device="cuda")
            q = t.quantize(u)
            p0 = np.zeros((B, w.N), dtype=np.complex128)
            p0[:, 0] = 1.0
            pT = rng.normal(size=(B, w.N)) + 1j * rng.normal(size=(B, w.N))
            pT /= np.linalg.norm(pT, axis=1, keepdims=True)
            p0d, pTd = torch.as_tensor(p0, device="cuda"), torch.as_tensor(pT, device="cuda")
            F = torch.empty(B, dtype=torch.float64, device="cuda")
            g = torch.empty((B, w.M, w.K), dtype=torch.float64, device="cuda")
            for prec in ("fp32", "fp64"):
                def it():
                    redo.redo_state_grad(t.handle, q, prec, p0d, pTd, F, g, None)
                it()
                ms = _events_time(it, 2)
                res[f"B{B}_{prec}"] = {"ms_per_iteration": ms, "instance_iters_per_s": B * 1e3 / ms}
        out.update({"metric": "state-transfer GRAPE instance-iterations/s", "unit": "instance-iterations/s",
                    "value": res["B152_fp32"]["instance_iters_per_s"], "results": res,
                    "config": {"N": w.N, "K": w.K, "M": w.M, "dt": w.dt,
                               "table": "digit table" if args.digit_table else "level table"}})
    elif args.workload == "phase":
        # Section III amplitude/phase drive: 6 qubits (N=64), each its own species (x-table of X_i/2,
        # levels on [0, Omega]), phases on [0, 2 pi), B=256 pulses x M=2000 steps, level table,
        # split FP16 with re-unitarisation every 64 steps.  Against the same pulses in x/y form
        # (coefficients A cos phi, A sin phi on 12 per-qubit x/y controls).
        B = args.B if args.B != B_FULL else 256
        M = args.M if args.M != M_FULL else 2000
        w = inputs.phase_config(6, B=B, M=M, seed=1)
        t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=True,
                       levels=args.levels)
        t.set_phase_axes(w.extra["sz"])
        u = torch.tensor(w.u, device="cuda")
        phi = torch.tensor(w.extra["phi"], device="cuda")
        target = torch.as_tensor(w.target, device="cuda")
        q = torch.empty(u.shape, dtype=torch.int32, device="cuda")
        U = torch.empty((B, w.N, w.N), dtype=torch.complex128, device="cuda")
        F = torch.empty(B, dtype=torch.float64, device="cuda")
        tau = torch.empty(B, dtype=torch.complex128, device="cuda")
        ws = torch.empty(redo.redo_propagate_phase_workspace(t.handle, B, M, "fp16x3", REUNIT), dtype=torch.uint8,
                         device="cuda")

        def it():
            redo.redo_quantize(t.handle, u, q)
            redo.redo_propagate_phase(t.handle, q, phi, "fp16x3", U, target, F, tau, ws, reunit_every=REUNIT)
        it()
        ms = _events_time(it, args.steps)
        redo.redo_profile_read()
        redo.redo_profile_enable(True)
        it()
        torch.cuda.synchronize()
        redo.redo_profile_enable(False)
        prof = redo.redo_profile_read()
        tc_ms = prof.get("chain_tc", (0.0, 0))[0]
        # FP64 on 16 pulses: accuracy of the split-FP16 result
        Bs = 16
        U64 = torch.empty((Bs, w.N, w.N), dtype=torch.complex128, device="cuda")
        F64 = torch.empty(Bs, dtype=torch.float64, device="cuda")
        t64 = torch.empty(Bs, dtype=torch.complex128, device="cuda")
        ws64 = torch.empty(redo.redo_propagate_phase_workspace(t.handle, Bs, M, "fp64", 0), dtype=torch.uint8,
                           device="cuda")
        q16, p16 = q[:Bs].contiguous(), phi[:Bs].contiguous()
        ms64 = _events_time(lambda: redo.redo_propagate_phase(t.handle, q16, p16, "fp64", U64, target, F64, t64,
                                                               ws64), 1)
        dF = float((F64 - F[:Bs]).abs().max())
        dU = float((U64 - U[:Bs]).abs().max())
        # GRAPE gradient in amplitudes and phases (FP32 SIMT chains), all pulses
        gA = torch.empty((B, M, w.K), dtype=torch.float64, device="cuda")
        gP = torch.empty_like(gA)
        Fg = torch.empty(B, dtype=torch.float64, device="cuda")
        nbg = ctypes.c_size_t()
        Lr = redo.load_library()
        redo._check(Lr.redo_fidelity_grad_phase_workspace(ctypes.c_void_p(t.handle), B, M, redo._prec("fp32"), 64,
                                                          ctypes.byref(nbg)))
        wsg = torch.empty(nbg.value, dtype=torch.uint8, device="cuda")

        def itg():
            redo.redo_quantize(t.handle, u, q)
            redo._check(Lr.redo_fidelity_grad_phase(ctypes.c_void_p(t.handle), redo._ptr(q), redo._ptr(phi), B, M,
                                                    redo._ptr(target), 0, redo._prec("fp32"), 64, redo._ptr(Fg),
                                                    redo._ptr(gA), redo._ptr(gP), redo._ptr(wsg), wsg.numel(), None,
                                                    None))
        itg()
        msg = _events_time(itg, 1)
        t.close()
        del ws, ws64, wsg
        # the same pulses in x/y form: 12 controls, one more factor per species and step
        Hxy = inputs.controls_local_xy(6)
        txy = redo.Table(w.H0, Hxy, w.dt, np.full(12, -w.extra["Omega"]), np.full(12, w.extra["Omega"]), w.base,
                         w.digits, fp32=True, fp16x3=True, levels=args.levels)
        uxy = torch.stack([u * torch.cos(phi), u * torch.sin(phi)], dim=3).reshape(B, M, 12).contiguous()
        qxy = torch.empty(uxy.shape, dtype=torch.int32, device="cuda")
        wsxy = txy.workspace(B, M, "fp16x3", REUNIT)
        Fxy = torch.empty(B, dtype=torch.float64, device="cuda")

        def itxy():
            redo.redo_quantize(txy.handle, uxy, qxy)
            redo.redo_propagate(txy.handle, qxy, "fp16x3", U, target, Fxy, tau, wsxy, reunit_every=REUNIT)
        itxy()
        msxy = _events_time(itxy, args.steps)
        txy.close()
        K = w.K
        op_bytes = B * M * K * 32768.0
        flop = B * M * K * 8.0 * w.N ** 3 * 3
        pk = _peaks()
        out.update({"metric": "REDO prop steps/s (amplitude/phase controls)", "unit": "pulse-steps/s",
                    "value": B * M / (ms / 1e3), "ms_per_call": ms,
                    "xy_form_same_pulses": {"pulse_steps_per_s": B * M / (msxy / 1e3), "ms_per_call": msxy,
                                            "controls": 12},
                    "speedup_vs_xy_form": msxy / ms,
                    "fp64_same_gpu": {"pulse_steps_per_s": Bs * M / (ms64 / 1e3), "pulses": Bs,
                                      "max_abs_dF_fp16x3_vs_fp64": dF, "max_abs_dU": dU},
                    "grape_gradient_fp32": {"instance_iters_per_s": B * 1e3 / msg, "ms_per_call": msg,
                                            "what": "F, dF/dA and dF/dphi of all pulses, FP32 SIMT chains, "
                                                    "checkpoints every 64 steps"},
                    "roofline": {"kernel": "chain_tc", "kernel_ms": tc_ms,
                                 "hbm_achieved_gbs": op_bytes / (tc_ms / 1e3) / 1e9 if tc_ms else None,
                                 "hbm_frac": (op_bytes / (tc_ms / 1e3) / 1e9 / pk.get("hbm_gbs", 6794.5)
                                              if tc_ms else None),
                                 "tensor_tflops": flop / (tc_ms / 1e3) / 1e12 if tc_ms else None,
                                 "tensor_frac_of_sustained": (flop / (tc_ms / 1e3) / 1e12
                                                              / pk.get("bf16_tflops_sustained", 1709.6)
                                                              if tc_ms else None),
                                 "algorithmic": f"{op_bytes:.4g} B of table operands (B*M*{K} x 32 KB), "
                                                f"{flop:.4g} fp16 flop (B*M*{K} complex products x 3)"},
                    "precision": "fp16x3 (tcgen05 chains; step phases applied in the chain epilogue, FP32)",
                    "config": {"N": w.N, "species": K, "B": B, "M": M, "dt": w.dt, "reunit_every": REUNIT,
                               "table": "level table" if args.levels else "digit table"}})
    elif args.workload == "plain":
        # 3 qubits (N=8), M=1000: latency of one pulse and throughput of 4096 replicas
        res = {}
        for B in (1, 4096):
            w = inputs.config(0, B=B)
            t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
            u = torch.tensor(w.u, device="cuda")
            target = torch.as_tensor(w.target, device="cuda")
            for prec in ("fp64", "fp32"):
                q = t.quantize(u)
                U, F, tau = (torch.empty((B, 8, 8), dtype=torch.complex128, device="cuda"),
                             torch.empty(B, dtype=torch.float64, device="cuda"),
                             torch.empty(B, dtype=torch.complex128, device="cuda"))
                ws = t.workspace(B, w.M, prec)

                def it():
                    redo.redo_quantize(t.handle, u, q)
                    redo.redo_propagate(t.handle, q, prec, U, target, F, tau, ws)
                it()
                ms = _events_time(it, args.steps)
                res[f"B{B}_{prec}"] = {"ms_per_call": ms, "pulse_steps_per_s": B * w.M / (ms / 1e3)}
        out.update({"metric": "REDO prop steps/s (plain REDO, N=8)", "unit": "pulse-steps/s",
                    "value": res["B4096_fp64"]["pulse_steps_per_s"], "results": res})
    elif args.workload == "warmstart_study":
        # 5 qubits, K=10, M=500, dt=2 us; targets from weight-one Pauli strings (reachable)
        from paper_1707_02162_gb300 import warmstart
        # every instance its own offsets and couplings (table without drift, per-pulse diagonal
        # drift); --shared-drift: the one-system study
        w = inputs.config(4, B=1)
        per_instance = not args.shared_drift
        H0 = np.zeros_like(w.H0) if per_instance else w.H0
        t = redo.Table(H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
        t0 = time.time()
        const = np.concatenate([w.extra["nu"][0] / 5e3, w.extra["J"][0][np.triu_indices(w.n_qubits, 1)] / 200.0])
        rep = warmstart.study(t, w.n_qubits, w.M, w.K, w.extra["Omega"], const,
                              n_train=args.B if args.B != B_FULL else 10000, n_test=args.ws_test,
                              per_instance_drift=per_instance, threshold=args.ws_threshold, iters=args.ws_iters,
                              train_threshold=args.ws_train_threshold)
        out.update({"metric": f"GRAPE iterations to F>={args.ws_threshold} (MLP warm start vs random init, "
                              f"L-BFGS ascent)",
                    "unit": "iterations", "value": rep.summary()["median_iters_mlp_init"],
                    "summary": rep.summary(), "wall_s": time.time() - t0,
                    "config": {"N": w.N, "K": w.K, "M": w.M, "dt": w.dt,
                               "systems": ("per instance: nu ~ U[-5,5] kHz, J ~ U[-200,200] Hz" if per_instance
                                           else "one system"),
                               "targets": "exp(-i sum theta_k P_k), 8 weight-one Pauli strings, theta ~ U[0, pi]",
                               "training": f"pulses converged to F >= {args.ws_train_threshold} from one start",
                               "iterations": "fidelity + gradient evaluations (FP32 chains re-unitarised every "
                                             "50 steps), L-BFGS with 8 pairs"}})
    elif args.workload == "warmstart":
        # 5 qubits (N=32), K=10, M=500: batched GRAPE iterations and MLP training throughput
        B = 256
        w = inputs.config(4, B=B)
        t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
        rng = np.random.default_rng(0)
        targets = torch.as_tensor(np.stack([inputs.haar_unitary(rng, w.N) for _ in range(B)]), device="cuda")
        u = torch.tensor(w.u, device="cuda")
        q = torch.empty(u.shape, dtype=torch.int32, device="cuda")
        F = torch.empty(B, dtype=torch.float64, device="cuda")
        g = torch.empty(u.shape, dtype=torch.float64, device="cuda")
        res = {}
        for prec in ("fp32", "fp64"):
            ws = torch.empty(redo.redo_fidelity_grad_workspace(t.handle, B, w.M, prec, 0), dtype=torch.uint8,
                             device="cuda")

            def it():
                redo.redo_quantize(t.handle, u, q)
                redo.redo_fidelity_grad(t.handle, q, targets, prec, 0, F, g, ws)
                redo.redo_grape_step(t.handle, u, g, 1e9)
            it()
            ms = _events_time(it, args.steps if prec == "fp32" else 1)
            res[prec] = {"instance_iters_per_s": B * 1e3 / ms, "ms_per_batched_iter": ms}
        # every instance with its own offsets and couplings: a table without drift and the
        # per-pulse diagonal drift of each instance
        t_nd = redo.Table(np.zeros_like(w.H0), w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
        h = torch.as_tensor(inputs.drift_diagonals(w), device="cuda")
        ws = torch.empty(redo.redo_fidelity_grad_drift_workspace(t_nd.handle, B, w.M, "fp32", 0), dtype=torch.uint8,
                         device="cuda")

        def it_drift():
            redo.redo_quantize(t_nd.handle, u, q)
            redo.redo_fidelity_grad_drift(t_nd.handle, q, h, targets, "fp32", 0, F, g, ws)
            redo.redo_grape_step(t_nd.handle, u, g, 1e9)
        it_drift()
        ms = _events_time(it_drift, args.steps)
        res["fp32_per_instance_drift"] = {"instance_iters_per_s": B * 1e3 / ms, "ms_per_batched_iter": ms}
        from paper_1707_02162_gb300.warmstart import MLP
        sizes = [23, 512, 512, 512, w.M * w.K]
        net = MLP(sizes)
        # forward + backward GEMM flop per sample: 2 in*out for z, 2 for dW, 2 for dh (no dh into x)
        fl = sum(2 * a * b for a, b in zip(sizes[:-1], sizes[1:])) * 3 - 2 * sizes[0] * sizes[1]
        mlp = {}
        for nb in (1024, 8192):
            x = torch.randn(nb, 23)
            y = torch.rand(nb, w.M * w.K) * 2 - 1
            net.train_step(x, y, 1e-3)
            ms = _events_time(lambda: net.train_step(x, y, 1e-3), 5)
            tf = fl * nb / (ms / 1e3) / 1e12
            mlp[f"batch_{nb}"] = {"samples_per_s": nb / (ms / 1e3), "ms_per_step": ms, "gemm_tflops": tf,
                                  "frac_of_bf16_burst": tf / _peaks().get("bf16_tflops", 1908.8),
                                  "hardware_frac_x3": 3 * tf / _peaks().get("bf16_tflops", 1908.8)}
        out.update({"metric": "GRAPE iters/s (batched instances, N=32)", "unit": "instance-iterations/s",
                    "value": res["fp32"]["instance_iters_per_s"], "results": res,
                    "mlp_train_samples_per_s": mlp["batch_1024"]["samples_per_s"], "mlp_training": mlp,
                    "config": {"N": w.N, "K": w.K, "M": w.M, "instances": B, "mlp": "23-512-512-512-5000"}})
    emit(out, args)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="prop",
                    choices=["prop", "grape", "sim", "plain", "warmstart", "warmstart_study", "freeze", "state",
                             "phase"],
                    help="prop (default): the batched propagation line; others: auxiliary measurements")
    ap.add_argument("--B", type=int, default=B_FULL, help="pulses (smaller only for profiling captures)")
    ap.add_argument("--M", type=int, default=M_FULL, help="steps per pulse (smaller only for profiling captures)")
    ap.add_argument("--nq", type=int, default=None, help="qubits of the sim workload (profiling captures only)")
    ap.add_argument("--digit-table", action="store_true",
                    help="multiply digit operators every step instead of using the level table "
                         "(process 3: every level's operator evaluated once, the default)")
    ap.add_argument("--shared-drift", action="store_true",
                    help="warmstart_study: one system for every instance instead of per-instance offsets/couplings")
    ap.add_argument("--ws-threshold", type=float, default=0.999, help="warmstart_study: fidelity threshold")
    ap.add_argument("--ws-train-threshold", type=float, default=0.99,
                    help="warmstart_study: fidelity the training pulses are converged to")
    ap.add_argument("--ws-test", type=int, default=1000, help="warmstart_study: held-out test instances")
    ap.add_argument("--ws-iters", type=int, default=600, help="warmstart_study: GRAPE iteration budget")
    ap.add_argument("--jsonl", default=None, help="also append the JSON line to this file (one record per run)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-grape", action="store_true", help="omit the GRAPE iterations/s sub-measurement")
    ap.add_argument("--skip-extra", action="store_true",
                    help="omit the N=8 plain-REDO and N=1024 ensemble sub-measurements")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    args.levels = not args.digit_table
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "prop":
        run_workload(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
