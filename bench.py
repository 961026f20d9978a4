#!/usr/bin/env python3
"""Benchmark: adaptive-ROM online steps/s on GB300.

Workload: 1D viscous Burgers, N = 16384 cells, nu = 2e-3, dt = 1e-4, seeded
initial condition 1 + 0.5 sin(2 pi x) + 0.1 S(x); r = 32, DEIM-Galerkin with
n_s = 96 sampled cells (QDEIM + feature-guided points), correction snapshot
and iSVD update every z = 5 steps, forgetting factor 0.5; FP64.

One bench step = one adaptation cycle: z reduced backward-Euler steps followed
by the adaptation event (coarse FOM step, iSVD update, sampling refresh, state
transfer), i.e. every part of the online path. ``value`` counts fine online
ROM steps (z per bench step) per second over the whole job; the state is
resident on the device when the timed region starts, and L2 is flushed
(a 256 MiB write) before every timed cycle. ``e2e`` runs the same cycles
through the public API from host buffers: the initial state goes up from
pinned host memory (rom_init, amortised over the run) and q~ comes back to
pinned host memory after every cycle.

The line also carries the other forms of the method (``forms``): the
mixed-precision form of the same workload; the batched form, 256
independent Burgers ROMs of uneven size (N log-uniform in [2048, 65536],
r in 8..48, z in {5, 10, 20}) advanced together for 5 K steps, reported in
aggregate ROM-steps/s with the HBM roofline of its reduced-step kernel; and
the two other single-ROM workloads (Burgers N=512, r=10, z=10, plain
Galerkin; Sod shock tube, 8192 cells, r=40, z=10), both FP64.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--only single|batched] [--batch-count B]
Under torchrun each rank runs an independent replica (the path does not
shard; weak scaling) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

if "--impl" in sys.argv and "reference" in sys.argv or "--oracle-sample" in sys.argv:
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "adaptive-ROM online steps/s"
UNIT = "steps/s"
WORKLOAD = "burgers-deim-N16384-r32-ns96-z5-lambda0.5-fp64"

# FP64 peak derived from the unit counts and clocks: 152 SMs x 2 DFMA/clk x
# 2 flop x 2.07 GHz (the nominal 1.25 TFLOP/s of the part).
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch from
# one ncu capture of each kernel on this workload (summarised under profiles/);
# reported only while the kernel's source file is unchanged (sha1).
TRAFFIC = {
    "isvd_update": {"bytes": 1720576, "src": "paper_2605_28684_gb300/csrc/isvd_impl.cuh",
                    "sha1": "02f79657ce901fced5825170c4e8942e8be9debe"},
    "coarse_fom": {"bytes": 162304, "src": "paper_2605_28684_gb300/csrc/fom.cu",
                   "sha1": "4186dd4b29c5d5f770230efc2cc4ccac8888452c"},
    "reduced_steps": {"bytes": 114944, "src": "paper_2605_28684_gb300/csrc/reduced.cu",
                      "sha1": "514213ca6cefd7d6f48cca53f028daf27b9cd039"},
    "sampling": {"bytes": 1148416, "src": "paper_2605_28684_gb300/csrc/sampling.cu",
                 "sha1": "07104bd9145843788aa23d3b344892c2af930245"},
}


def workload_config():
    return synth.config_burgers_hyper(precision=0)


def config_json(cfg):
    return {"workload": WORKLOAD, "n_cells": cfg.n_cells, "r": cfg.r, "n_s": cfg.n_s, "z": cfg.z,
            "lambda": cfg.lam, "nu": cfg.nu, "dt": cfg.dt, "w_init": cfg.w_init,
            "step": f"one adaptation cycle = {cfg.z} reduced steps + 1 event",
            "l2": "flushed (256 MiB write) before every timed cycle"}


def peaks():
    p = {"hbm_gbs": 6800.0, "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            m = json.load(f)
        p = {"hbm_gbs": float(m["hbm_gbs"]), "source": "measured"}
    return p


# ---------------------------------------------------------------- oracle ---

def oracle_sample(seconds: float):
    """Time the CPU oracle (single thread) on the same workload for about
    ``seconds``; returns online steps/s and the sample description."""
    from oracle import rom as orom
    cfg = workload_config()
    q0 = synth.initial_state(cfg)
    m = orom.AdaptiveROM(cfg, q0)
    steps = 0
    t0 = time.perf_counter()
    while True:
        for _ in range(cfg.z):
            m.step()
        steps += cfg.z
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return steps / dt, steps, dt


def cpu_baseline(seconds=15.0):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(seconds)],
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "failed: " + r.stderr.strip().splitlines()[-1][:200]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{d['steps']} online steps ({d['steps'] // 5} adaptation cycles) of the same "
                      f"workload after the offline stage, {d['seconds']:.1f} s, one thread"}


def max_over_ranks(x, dist, device="cuda"):
    """The largest of every rank's x (a device time); x itself on one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    """The reference arm: the FP64 oracle on the host, same workload and metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import rom as orom
    cfg = workload_config()
    q0 = synth.initial_state(cfg)
    m = orom.AdaptiveROM(cfg, q0)
    for _ in range(args.warmup):
        for _ in range(cfg.z):
            m.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(cfg.z):
            m.step()
    dt = time.perf_counter() - t0
    value = args.steps * cfg.z / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_json(cfg), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} adaptation cycles ({args.steps * cfg.z} online "
                                       f"steps) after {args.warmup} warm-up cycles, one thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- clocks ---

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- roofline ---

def algorithmic_work(phase: str, cfg, rank: int, launches: dict, fom_iters: float, rom_iters: float):
    """Algorithmic bytes and FP64 flops of one launch of a phase (minimum the
    method must move / compute; see the work model of each kernel)."""
    N, k, ns, z = cfg.n_cells, rank, cfg.n_s, cfg.z
    if phase == "isvd_update":
        # CGS2 reads Phi three times, rotation reads and writes it; y, q_ref,
        # D read; yhat and q written and re-read.
        bytes_ = 8 * N * (3 * k + 2 * k) + 8 * N * 3 + 8 * N * 4
        flops = 2 * N * k * 4 + 2 * N * (k + 1) * k
        return bytes_, flops
    if phase == "coarse_fom":
        # per Newton iteration: read q (with halo) and q_prev, write q
        return 24 * N * fom_iters, 30 * N * fom_iters
    if phase == "sampling":
        # QDEIM: the initial norms read Phi (k columns); each of the k - 1
        # updates reads Phi and the s earlier coordinates of every row and
        # writes one coordinate
        return (8 * N * k * k + 8 * N * (k - 1) * k // 2,
                2 * N * k * k + N * (k - 1) * k + 2 * N * (k - 1))
    if phase == "feature_select":
        # read y, write the keys, read them in the selection
        return 24 * N, 2 * N
    # reduced steps: per Newton iteration the stencil mesh (Phi rows, q_ref,
    # d) and (P^T Phi)^+ are read once
    per_it = 8 * (3 * ns * (k + 2) + k * ns)
    return per_it * rom_iters * z, (6 * ns * k + 2 * k * ns + 30 * ns) * rom_iters * z


def src_sha1(rel):
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


# --------------------------------------------------------------- batched ---

def timed_single(g, cfg, n_steps):
    """Online steps/s of one more single-ROM workload (device time of n_steps
    steps on a side stream after 3 adaptation intervals of warm-up)."""
    import torch
    try:
        q0 = synth.initial_state(cfg)
        s = torch.cuda.Stream()
        rom = g.AdaptiveROM(cfg, q0, stream=s.cuda_stream)
        rom.step(3 * cfg.z)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        rom.step(n_steps)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        info = rom.info()
        rom.close()
        return {"value": n_steps / (ms / 1e3), "unit": "steps/s", "steps": n_steps,
                "ms_per_step": ms / n_steps, "rank_k": info["rank"]}
    except Exception as exc:       # an extra form must not cost the main line
        return {"error": f"{type(exc).__name__}: {exc}"}


def timed_full_horizon(g, cfg, n_steps, fom_eps=True, chunk=None):
    """One rom_step over a whole horizon (device time on a side stream and
    wall clock around the call), and the ROM error against the fine FOM
    (the FOM advanced on the GPU by rom_fom_step_dev over the same steps).
    With ``chunk``, rom_step runs in calls of that many steps and the horizon
    ends at the first call that fails (a ROM that leaves the physical range):
    the steps completed before it are timed and reported."""
    import torch
    try:
        q0 = synth.initial_state(cfg)
        s = torch.cuda.Stream()
        rom = g.AdaptiveROM(cfg, q0, stream=s.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record(s)
        err = None
        done = 0
        if chunk is None:
            try:
                rom.step(n_steps)
                done = n_steps
            except g.RomError as exc:
                err = str(exc)
        else:
            while done < n_steps:
                m = min(chunk, n_steps - done)
                try:
                    rom.step(m)
                except g.RomError as exc:
                    err = str(exc)
                    break
                done += m
                e1.record(s)
        if chunk is None or err is None or done == 0:
            e1.record(s)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms = e0.elapsed_time(e1)
        out = {"steps": done, "device_ms": ms, "wall_ms": wall * 1e3,
               "value": done / (ms / 1e3) if done else 0.0, "unit": "steps/s"}
        if err is not None:
            out["stopped"] = f"after {done} of {n_steps} steps (t = {(cfg.w_init + done) * cfg.dt:.4f}): {err}"
            if chunk is None or done == 0:
                out["error"] = err
                rom.close()
                return out
            fom_eps = False
        if not fom_eps:
            rom.close()
            return out
        if fom_eps:
            qt = rom.q_tilde()
            qa = torch.tensor(q0, device="cuda", dtype=torch.float64)
            qb = torch.empty_like(qa)
            for _ in range(cfg.w_init + n_steps):
                g.fom_step_dev(cfg.problem, cfg.n_cells, cfg.nu, cfg.gamma, cfg.dt, cfg.newton_tol,
                               cfg.newton_max, qa.data_ptr(), qb.data_ptr())
                qa, qb = qb, qa
            qf = qa.cpu().numpy()
            out["eps_vs_fom"] = float(np.linalg.norm(qt - qf) / np.linalg.norm(qf))
        rom.close()
        return out
    except Exception as exc:       # an extra form must not cost the main line
        return {"error": f"{type(exc).__name__}: {exc}"}


def timed_adjoint(g):
    """The gradient workload (Burgers N = 65536, r = 64, 1000 steps, z = 10):
    rom_adjoint (offline stage, recorded forward pass and reverse sweep) next
    to the plain FP64 forward of the same steps (rom_init + rom_step), both
    device-timed, and the gradient against the oracle's stored values."""
    import torch
    try:
        cfg = synth.config_adjoint()
        q0 = synth.initial_state(cfg)
        target = synth.burgers_target(cfg.n_cells, cfg.seed + 1)
        g.adjoint(cfg, q0, target, 20, 20)                 # warm-up (allocation, code load)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, dnu, dq0 = g.adjoint(cfg, q0, target, cfg.n_online, 50)
        torch.cuda.synchronize()
        adj_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        rom = g.AdaptiveROM(cfg, q0)
        rom.step(cfg.n_online)
        torch.cuda.synchronize()
        fwd_s = time.perf_counter() - t0
        rom.close()
        dA = float(dq0 @ synth.burgers_ic_amplitude_direction(cfg.n_cells))
        with open(os.path.join(ROOT, "tests", "golden", "adjoint_burgers_n65536_r64.json")) as f:
            gold = json.load(f)
        ref = gold["grad_reverse_sweep"]
        return {"workload": "burgers-N65536-r64-z10-1000steps-terminal-misfit", "steps": cfg.n_online,
                "ckpt_every": 50, "forward_backward_s": adj_s, "plain_forward_s": fwd_s,
                "ratio": adj_s / fwd_s, "J": J, "dJ_dnu": dnu, "dJ_dA": dA,
                "rel_err_vs_oracle": {"nu": abs(dnu - ref["nu"]) / abs(ref["nu"]),
                                      "A": abs(dA - ref["A"]) / abs(ref["A"])},
                "timing": "wall clock around each call (both include the offline stage)"}
    except Exception as exc:
        return {"error": f"{type(exc).__name__}: {exc}"}


def timed_paper_sweep(g):
    """The paper's Burgers setting (Gaussian pulse, N = 1000, dt = 1e-3,
    r = w_init = 4) for z in {5, 10, 25, 50} x lambda in {1e-7 ... 1}: 24 ROMs in
    one batch. Device time of the 496 online steps (one call on a capturable
    stream), then, in a second untimed pass, the mean ROM error against the
    fine FOM over the horizon and, per instance, the error of the correction
    signal (the coarse FOM state of the last event) next to the ROM error at
    that time (the paper's study of the correction signal)."""
    import torch
    try:
        cfgs = synth.config_paper_burgers_sweep()
        q0 = synth.initial_state(cfgs[0])
        n_on, w = cfgs[0].n_online, cfgs[0].w_init
        fom = [q0]
        qa = torch.tensor(q0, device="cuda", dtype=torch.float64)
        qb = torch.empty_like(qa)
        for _ in range(w + n_on):
            g.fom_step_dev(0, 1000, 0.01, 1.4, 1e-3, 1e-12, 20, qa.data_ptr(), qb.data_ptr())
            qa, qb = qb, qa
            fom.append(qa.cpu().numpy())
        s = torch.cuda.Stream()
        b = g.Batch(cfgs, [q0] * len(cfgs), stream=s.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        b.step(n_on)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        b.close()
        b = g.Batch(cfgs, [q0] * len(cfgs))
        mean = np.zeros(len(cfgs))
        stride = 16
        for j in range(n_on // stride):
            b.step(stride)
            qf = fom[w + (j + 1) * stride]
            for i in range(len(cfgs)):
                mean[i] += np.linalg.norm(b.q_tilde(i) - qf) / np.linalg.norm(qf) / (n_on // stride)
        table, signal = {}, {}
        for i, c in enumerate(cfgs):
            st = b.state(i, y_corr=True)
            n_ev = w + (n_on // c.z) * c.z            # time level of the last correction snapshot
            qe = fom[n_ev]
            table.setdefault(str(c.z), {})[f"{c.lam:g}"] = mean[i]
            signal.setdefault(str(c.z), {})[f"{c.lam:g}"] = {
                "signal_error": float(np.linalg.norm(st["y_corr"] - qe) / np.linalg.norm(qe))}
        b.close()
        best = {z: min(row, key=row.get) for z, row in table.items()}
        return {"instances": len(cfgs), "steps": n_on, "device_ms": ms,
                "value": len(cfgs) * n_on / (ms / 1e3), "unit": "ROM-steps/s",
                "mean_rom_error": table, "best_lambda_by_z": best, "correction_signal": signal,
                "note": "mixed form (FP32 basis), plain Galerkin; the paper's ROM is LSPG-QDEIM"}
    except Exception as exc:
        return {"error": f"{type(exc).__name__}: {exc}"}


# DRAM traffic of one launch of the batched reduced-step kernel (5 steps) from
# one ncu capture of the 256-instance workload (summarised under profiles/);
# reported only while csrc/batch.cu is unchanged.
TRAFFIC_BATCH = {"bytes": 862447360, "src": "paper_2605_28684_gb300/csrc/batch.cu",
                 "sha1": "a55f94bf992be31e6f98150451f8427b236596c9"}


def timed_batch(g, args, stream, dist, world):
    """Aggregate ROM-steps/s of the 256-instance batch and the HBM roofline of
    its reduced-step kernel (each Newton iteration streams every active
    instance's FP32 basis and q_ref once)."""
    import torch
    cfgs = synth.config_batch(args.batch_count)
    q0s = [synth.initial_state(c) for c in cfgs]
    bs = torch.cuda.Stream()      # a capturable stream: whole intervals replay a CUDA graph
    b = g.Batch(cfgs, q0s, stream=bs.cuda_stream)
    n_steps = 5 * args.steps
    b.step(5 * args.warmup)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    start.record(bs)
    b.step(n_steps)
    end.record(bs)
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    graph_state = b.layout()["graph"]
    # the same number of steps again with the per-phase timer on (no graph)
    b.profile(True)
    b.step(n_steps)
    torch.cuda.synchronize()
    prof = b.profile_read()
    work = b.work()
    fwork = b.fom_work()
    lay = b.layout()
    b.profile(False)
    b.close()
    ms = max_over_ranks(ms, dist)
    pk = peaks()
    step_s = prof["reduced_steps"]["ms"] / 1e3
    gbs = work["sweep_bytes"] / step_s / 1e9
    launches = max(1, prof["reduced_steps"]["launches"])
    # the coarse FOM kernel: 24 bytes per row and Newton iteration (read the
    # iterate and the previous state, write the update)
    fom_s = prof["coarse_fom"]["ms"] / 1e3
    fom_launches = max(1, prof["coarse_fom"]["launches"])
    fom_gbs = fwork["fom_bytes"] / fom_s / 1e9 if fom_s > 0 else 0.0
    fom_roof = {"bound": "hbm", "kernel": "batch_fom_kernel", "achieved": fom_gbs,
                "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": fom_gbs / pk["hbm_gbs"],
                "peak_source": pk["source"], "algorithmic_bytes": fwork["fom_bytes"] / fom_launches,
                "row_iterations_per_launch": fwork["row_iterations"] / fom_launches,
                "avg_launch_us": fom_s / fom_launches * 1e6, "traffic": None,
                "per": "launch (the coarse step of the instances that adapt at that step)"}
    traffic = None
    if TRAFFIC_BATCH["bytes"] is not None and TRAFFIC_BATCH["sha1"] == src_sha1(TRAFFIC_BATCH["src"]) \
            and len(cfgs) == 256:
        traffic = TRAFFIC_BATCH["bytes"]
    return {"value": world * len(cfgs) * n_steps / (ms / 1e3), "unit": "ROM-steps/s",
            "instances": len(cfgs), "steps": n_steps, "ms_per_step": ms / n_steps,
            "basis_bytes": lay["basis_bytes"], "rows": lay["rows"], "tiles": lay["tiles"],
            "tile_rows_autotuned": lay["tile_rows"],
            "newton_iters_per_instance_step": work["newton_iters"] / (len(cfgs) * n_steps),
            "phases_ms": {p: prof[p]["ms"] for p in prof},
            "graph": {"state": graph_state,
                      "note": "1: each adaptation interval of the timed run replays one captured "
                              "CUDA graph; the phase split comes from a second, profiled run "
                              "of the same length"},
            "launches": {p: prof[p]["launches"] for p in prof},
            "roofline": {"bound": "hbm", "kernel": "batch_steps_kernel", "achieved": gbs,
                         "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
                         "peak_source": pk["source"],
                         "algorithmic_bytes": work["sweep_bytes"] / launches,
                         "avg_launch_us": step_s / launches * 1e6, "traffic": traffic,
                         "per": "launch (5 steps of every instance)"},
            "fom_roofline": fom_roof}


# ------------------------------------------------------------------- main ---

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--oracle-sample", type=float, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", default="all", choices=["all", "single", "batched"],
                    help="single / batched: time only the single-ROM forms or only the "
                         "batched form (for profiling runs)")
    ap.add_argument("--batch-count", type=int, default=256,
                    help="instances of the batched form (256 is the configured workload)")
    args = ap.parse_args()

    if args.oracle_sample is not None:
        v, steps, dt = oracle_sample(args.oracle_sample)
        print(json.dumps({"value": v, "steps": steps, "seconds": dt}))
        return
    if args.impl == "reference":
        run_reference(args)
        return
    args.warmup = max(args.warmup, 3)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2605_28684_gb300 import build as _build
    if rank == 0 or world == 1:
        _build.build()
    if dist is not None:
        dist.barrier()
    import paper_2605_28684_gb300 as g

    stream = torch.cuda.current_stream()
    if args.only == "batched":
        line = timed_batch(g, args, stream, dist, world)
        if rank == 0:
            print(json.dumps({"form": "batched", **line}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    cfg = workload_config()
    q0 = synth.initial_state(cfg)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed_cycles(c, sampler=None):
        """W warm-up cycles, then K timed cycles (CUDA events on the ROM's
        stream around each cycle, L2 flushed before each); returns the summed
        device time, the per-phase profile and the final rank/Newton counts."""
        rom = g.AdaptiveROM(c, q0, stream=stream.cuda_stream)
        for _ in range(args.warmup):
            rom.step(c.z)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        if sampler is not None:
            sampler.start()
        rom.profile(True)
        for i in range(args.steps):
            flush.fill_(float(i))
            starts[i].record(stream)
            rom.step(c.z)
            ends[i].record(stream)
        torch.cuda.synchronize()
        prof = rom.profile_read()
        rom.profile(False)
        if dist is not None:
            dist.barrier()
        clk = sampler.stop() if sampler is not None else None
        total = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
        info = rom.info()
        rom.close()
        return total, prof, info, clk

    sampler = ClockSampler(local)
    total_ms, prof, info, clocks = timed_cycles(cfg, sampler)
    t_max = max_over_ranks(total_ms, dist)
    value = world * args.steps * cfg.z / (t_max / 1e3)

    # the mixed-precision form of the same workload (FP32 basis and projections)
    mcfg = workload_config()
    mcfg.precision = 1
    m_ms, m_prof, m_info, _ = timed_cycles(mcfg)
    m_ms = max_over_ranks(m_ms, dist)
    forms = {
        "fp64": {"value": value, "ms_per_step": t_max / args.steps, "rank_k": info["rank"]},
        "mixed_fp32": {"value": world * args.steps * mcfg.z / (m_ms / 1e3),
                       "ms_per_step": m_ms / args.steps, "rank_k": m_info["rank"],
                       "rank_tol": 1e-5,
                       "phases_avg_us": {p: m_prof[p]["ms"] * 1e3 / max(1, m_prof[p]["launches"])
                                         for p in m_prof}},
    }

    # the batched form: 256 independent Burgers ROMs of uneven size (N
    # log-uniform in [2048, 65536], r in 8..48, z in {5, 10, 20}) advanced in
    # lockstep; ~0.5 GB of FP32 bases, larger than L2, so no flush is needed
    if args.only == "all":
        forms["batched_256"] = timed_batch(g, args, stream, dist, world)
        # the two other single-ROM workloads: Burgers N=512 plain Galerkin, and Sod
        forms["burgers_n512_r10_z10_fp64"] = timed_single(g, synth.config_burgers_small(), 2000)
        forms["sod_n8192_r40_z10_fp64"] = timed_single(g, synth.config_sod(), 500)
        # whole horizons: the headline workload's 20 000 steps; Sod towards
        # t = 0.2 (4938 online steps) in calls of 100 steps, ending at the
        # first call that fails (the Galerkin ROM leaves the physical range
        # near the 4099th online step)
        forms["c1_full_horizon"] = timed_full_horizon(g, workload_config(), 20000)
        sod = synth.config_sod()
        forms["sod_full_horizon"] = timed_full_horizon(g, sod, sod.n_online, chunk=100)
        # the paper's Sod size (256 cells) over its whole horizon to t = 0.2,
        # with the ROM error against the fine FOM
        sod256 = synth.config_sod(256)
        forms["sod_n256_full_horizon"] = timed_full_horizon(g, sod256, sod256.n_online)
        lspg = synth.config_burgers_small()
        lspg.projection = 1
        forms["lspg_burgers_n512_r10_z10_fp64"] = timed_single(g, lspg, 2000)
        # the instantaneous comparison rules of App. A (learning rates of the
        # paper's Burgers tuning at z = 10)
        for name, rule, eta in [("onestep", 3, 0.0), ("oja", 4, 0.01), ("grouse", 5, 0.01)]:
            c = synth.config_burgers_small()
            c.update_rule, c.learning_rate = rule, eta
            forms[f"{name}_burgers_n512_r10_z10_fp64"] = timed_single(g, c, 2000)
        # the explicit form (SSPRK(4,3) fine and reduced steps, coarse BE
        # correction): Sod Galerkin at the configured size, and Burgers
        # DEIM-Galerkin with r QDEIM + r feature-guided points
        sod_x = synth.config_sod()
        sod_x.time_scheme = 1
        forms["sod_explicit_galerkin_n8192_r40_z10_fp64"] = timed_single(g, sod_x, 500)
        bx = synth.config_burgers_small()
        bx.time_scheme, bx.n_s = 1, 20
        forms["burgers_explicit_deim_n512_r10_ns20_fp64"] = timed_single(g, bx, 2000)
        # the Galerkin-FGS form of the paper's RDE ROM on Sod: r QDEIM points
        # and r points of largest squared pressure difference; 30 warm-up and
        # 170 timed steps (the 200-step horizon over which this size is
        # checked against the oracle)
        sfx = synth.config_sod(2048)
        sfx.time_scheme, sfx.r, sfx.n_s = 1, 20, 40
        forms["sod_explicit_deim_fgs_n2048_r20_ns40_fp64"] = timed_single(g, sfx, 170)
        forms["adjoint"] = timed_adjoint(g)
        forms["paper_burgers_sweep"] = timed_paper_sweep(g)

    # roofline of the dominant kernel (largest device time in the timed region)
    dom = max(prof, key=lambda p: prof[p]["ms"])
    launches = prof[dom]["launches"]
    avg_s = prof[dom]["ms"] / 1e3 / max(1, launches)
    bytes_, flops = algorithmic_work(dom, cfg, info["rank"], prof, info["fom_newton_iters"],
                                     info["rom_newton_iters"])
    pk = peaks()
    gbs = bytes_ / avg_s / 1e9
    gfl = flops / avg_s / 1e9
    f_hbm = gbs / pk["hbm_gbs"]
    f_alu = gfl / FP64_PEAK_GFLOPS
    tr = TRAFFIC.get(dom)
    traffic = tr["bytes"] if tr and tr["sha1"] == src_sha1(tr["src"]) else None
    if f_hbm >= f_alu:
        roof = {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": f_hbm, "peak_source": pk["source"]}
    else:
        roof = {"bound": "alu", "achieved": gfl, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s (FP64)",
                "frac": f_alu, "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz"}
    roof.update({"kernel": dom, "traffic": traffic, "algorithmic_bytes": bytes_,
                 "algorithmic_flops": flops, "avg_launch_us": avg_s * 1e6,
                 "hbm_frac": f_hbm, "fp64_frac": f_alu})
    phases = {p: {"ms_total": prof[p]["ms"], "launches": prof[p]["launches"],
                  "avg_us": prof[p]["ms"] * 1e3 / max(1, prof[p]["launches"])} for p in prof}
    # kernels: one per phase launch, two for the feature-guided selection
    gpu_launches = sum(prof[p]["launches"] for p in prof) + prof.get("feature_select", {}).get("launches", 0)

    # end to end through the public API from pinned host buffers
    q0_pin = torch.from_numpy(q0.copy()).pin_memory()
    qt_pin = torch.empty(cfg.n_cells, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rom2 = g.AdaptiveROM(cfg, q0_pin.numpy(), stream=stream.cuda_stream)
    for _ in range(args.steps):
        rom2.step(cfg.z)
        rom2.q_tilde(out=qt_pin.numpy())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    rom2.close()
    e2e_s = max_over_ranks(e2e_s, dist)
    e2e = {"value": world * args.steps * cfg.z / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 8 * cfg.n_cells / args.steps, "d2h_bytes_per_step": 8 * cfg.n_cells,
           "includes": "rom_init from host q0 (offline stage) + every cycle's q~ readback"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config_json(cfg), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": gpu_launches, "clocks": clocks, "phases": phases, "forms": forms,
                "rank_k": info["rank"], "newton_iters": {"rom": info["rom_newton_iters"],
                                                         "fom": info["fom_newton_iters"]}}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
