#!/usr/bin/env python
"""Benchmark: retarded (light-cone) Lyman-Werner field evaluations per second.

Default workload (c5, serving): 8 simulations at 128^3 .. 512^3 (0.78 Mpc
cells, flat LCDM Omega_m = 0.31, h = 0.68, 64-128 equal-conformal-time shells
spanning the LW horizon at z = 15, BF16 spectrum history with a per-slot
FP32 scale, 1e4-1e5 clustered sources each).  Each simulation's history is
filled (untimed), then requests for its next K steps (K = --steps) arrive:
all at once (saturation, the headline value), then as a Poisson stream at
0.8x the saturation rate (latency), then again all at once with the fields
copied to host memory (end to end).  The server admits simulations by an HBM
budget, keeps each one's history resident, runs each on its own CUDA stream
and launches a request as soon as it is the simulation's next step, so the
work of many requests overlaps on the device (continuous batching).  Beside
it: the plain FP32 one-instance path on the same requests, the shell-MAC
roofline of the served steps (each simulation alone, phase events), the FP64
oracle on sampled cells (CPU baseline and the error of the served fields),
and the 256^3 single-instance MAC roofline (c3) as an extra key.

Other workloads (--workload): c1, c2 (128^3 FP32, 64 steps), c3 (256^3 BF16,
128 shells), c3s, c4 (16 uneven instances in one CUDA graph).  A "step" of
those is one push of a step's sources (deposit + forward transform into the
history ring) plus one retarded-field evaluation (shell MAC + inverse
transform), replayed as one CUDA graph; L2 is flushed between timed steps.

Under torchrun each rank runs an independent copy of the workload on its own
GPU (weak scaling, no data-path collective); the reported time is the max over
ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c5] [--impl reference]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "retarded-field evals/s & cell·shell MAC/s vs plain FP32 path; HBM %; p50/p99"
UNIT = "fields/s"
WORKLOADS = {
    "c5": ("serving: 8 simulations N = 128, 192, 256, 256, 384, 384, 512, 512 with 128, 112, 96, 128, 96, 64, "
           "96, 96 shells, BF16 history, 1e4-1e5 clustered sources, K requests each, continuous batching under an "
           "HBM budget; beside it the plain FP32 one-instance path on the same requests"),
    "c2": ("128^3 grid, 150 Mpc box, 64 equal-time steps z=30->10 (<=7 shells), 1e4 clustered sources "
           "(dN/dM~M^-2, 1-4 step lifetimes), FP32 FFT+MAC"),
    "c1": "32^3 grid, 100 Mpc box, 8 equal-time steps z=20->15 (<=2 shells), 200 uniform sources, FP32",
    "c3": ("256^3 grid, 200 Mpc box, 128 equal-conformal-time shells spanning the LW horizon at z=15, "
           "1e5 clustered sources, BF16 history with per-slot FP32 scale"),
    "c3s": ("256^3 grid, 200 Mpc box, 32 equal-conformal-time shells, 40 steps, 1e5 clustered sources, "
            "BF16 history (profiling size of the c3 path)"),
    "c5s": ("512^3 grid, 400 Mpc box, 16 equal-conformal-time shells, 24 steps, 4e4 clustered sources, BF16 history "
            "(profiling size of the served 512^3 path)"),
    "c5m": ("384^3 grid, 300 Mpc box, 16 equal-conformal-time shells, 24 steps, 3e4 clustered sources, BF16 history "
            "(profiling size of the served 384^3 path)"),
    "c4": ("16 uneven instances (grids 64..256 cycled, 32..128 shells, 1e3..1e5 clustered sources, 0.78 Mpc "
           "cells), FP32, all instances' step in one CUDA graph replay (parallel branches)"),
}
# accuracy the FP32 / BF16-history fields must meet against the FP64 oracle
TOL = {"fp32": {"rel_l2": 1e-5, "max_beyond_2ulp_over_mean": 1e-4}, "bf16": {"rel_l2": 5e-3}}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (c5: requests per simulation and pass, default 20; 2048 for c1/c2, 64 for c3, "
                         "32 for c3s/c4, 16 for --impl reference)")
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--flush-mb", type=int, default=512)
    ap.add_argument("--kernel", default="lw", choices=["lw", "exp"],
                    help="radial kernel: Lyman-Werner (Eqs. 14-17) or exp(-r/30 Mpc) cut off at 80 Mpc")
    ap.add_argument("--near", default="ngp", choices=["ngp", "subcell"],
                    help="innermost slice's near field: cell-centred (NGP) or from the sources' own positions")
    ap.add_argument("--e2e-pipelined", action="store_true",
                    help="also time the host-I/O loop with Plan.field_async (each step's output copy overlaps the "
                         "next step; no L2 flush between steps, which would serialise that overlap)")
    ap.add_argument("--fdiff", action="store_true",
                    help="each step also builds the instantaneous field (Eq. 18) and the f_diff map")
    ap.add_argument("--no-c3", action="store_true", help="c5: skip the 256^3 single-instance extra key")
    ap.add_argument("--equal-priorities", action="store_true",
                    help="c5: every simulation's stream at the default CUDA stream priority (default: small grids "
                         "higher, the Server's default)")
    return ap.parse_args(argv)


EXP_KERNEL = (1, 30.0, 80.0)  # exp(-r / 30 Mpc), cut off at r_max = 80 Mpc


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- FP64 oracle
def oracle_sample(w, steps, cells_per_step, seed=0, dense=True):
    """The FP64 oracle on a bounded sample: for each step, its Green's
    functions plus sampled cells (uniform draws, plus the x-line through the
    brightest source when `dense`); the full-field time is extrapolated from
    the per-cell rate.  Returns (fields/s, seconds spent, description,
    {step: (cells, values)})."""
    import oracle

    oracle.build()
    P = oracle.Problem.from_workload(w)
    spent = 0.0
    per_field = []
    samples = {}
    for s in steps:
        slices = oracle.source_lists(P, w.cat, s)
        one = np.array([0], dtype=np.int64)
        t0 = time.perf_counter()
        P.field_sparse(s, slices, cells=one)  # Green's functions + one cell: the fixed cost
        t1 = time.perf_counter()
        pos, lum = w.cat.active(s)
        line = None
        if dense and lum.shape[0]:
            line = np.floor(pos[np.argmax(lum)] / (w.box / w.n) + 0.5).astype(int) % w.n
        import synth

        cells = synth.sample_cells(seed + s, w.n, cells_per_step, dense_line_through=line)
        uniform = np.isin(cells, synth.sample_cells(seed + s, w.n, cells_per_step))
        ref = P.field_sparse(s, slices, cells=cells)
        t2 = time.perf_counter()
        fixed = t1 - t0
        per_cell = max(0.0, (t2 - t1) - fixed) / len(cells)
        per_field.append(fixed + per_cell * w.n ** 3)
        spent += t2 - t0
        samples[s] = (cells, ref, uniform)
    desc = (f"oracle FP64 on steps {list(steps)}: Green's functions + {cells_per_step} sampled cells per step"
            f"{' (+ the x-line through the brightest source)' if dense else ''}, full-field time extrapolated from "
            f"the per-cell rate")
    return 1.0 / float(np.mean(per_field)), spent, desc, samples


def field_errors(got, ref):
    """(relative L2, max error beyond 2 FP32 ulps / mean, raw max error / mean)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.abs(got - ref)
    mean = np.abs(ref).mean()
    ulp = np.exp2(np.floor(np.log2(np.maximum(np.abs(ref), np.finfo(np.float32).tiny))) - 23)
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref)) if np.linalg.norm(ref) > 0 else 0.0
    return rel, float(np.maximum(d - 2 * ulp, 0).max() / mean) if mean > 0 else 0.0, \
        float(d.max() / mean) if mean > 0 else 0.0


def sample_errors(label, J, sample):
    """One error_summary row: the GPU field J (flat) at an oracle sample
    (cells, values, uniform-cell mask), over all sampled cells and over the
    uniform draws alone (without the line through the brightest source)."""
    cells, ref, uniform = sample
    r, m, x = field_errors(J[cells], ref)
    ru = field_errors(J[cells[uniform]], ref[uniform])[0] if uniform.any() else None
    return (label, r, m, x, ru)


def error_summary(results, history):
    """error_vs_fp64 of a line from per-result (label, rel, max2ulp, raw, rel over uniform cells) rows."""
    kind = "bf16" if history else "fp32"
    tol = TOL[kind]
    rows = [{"result": lab, "rel_l2": r, "max_beyond_2ulp_over_mean": m, "raw_max_over_mean": x,
             "rel_l2_uniform_cells": ru} for lab, r, m, x, ru in results]
    ok = all(r["rel_l2"] <= tol["rel_l2"] and (kind == "bf16" or r["max_beyond_2ulp_over_mean"]
                                                 <= tol["max_beyond_2ulp_over_mean"]) for r in rows)
    return {"history": kind, "tolerance": tol, "within_tolerance": ok,
            "rel_l2_max": max((r["rel_l2"] for r in rows), default=None),
            "max_beyond_2ulp_over_mean_max": max((r["max_beyond_2ulp_over_mean"] for r in rows), default=None),
            "raw_max_over_mean_max": max((r["raw_max_over_mean"] for r in rows), default=None),
            "per_result": rows,
            "rel_l2_uniform_cells_max": max((r["rel_l2_uniform_cells"] for r in rows
                                             if r["rel_l2_uniform_cells"] is not None), default=None),
            "method": "GPU field at the sampled cells of the CPU-baseline leg (uniform draws plus the x-line through "
                      "the brightest source) against the FP64 oracle (Eq. 11); max criterion on the error beyond two "
                      "FP32 ulps of the oracle value; rel_l2_uniform_cells: the uniform draws alone, where the field "
                      "is weakest and a BF16 history's nearly uniform rounding noise is largest relative to it"}


# ---------------------------------------------------------------- helpers
def active_shell_work(plan, w, s):
    """Shells the MAC reads at step s: active slices whose step had sources."""
    lo, hi, rh = plan.shells(s)
    return sum(1 for j in range(len(lo)) if w.cat.active(s - j)[1].shape[0] > 0), len(lo)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def hbm_peak():
    p = measured_peaks()
    if "hbm_gbs" in p:
        return float(p["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured)"
    return 6800.0, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


def max_over_ranks(x, device):
    """The largest of every rank's x (the job's time is its slowest rank's);
    x itself when no process group is running."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def fft_choices(ns):
    """The FFT pass form in use for each grid size in ns (autotuned when the
    first plan of that size was created): {N: name}."""
    import paper_1502_02294_gb300 as lc

    names = {lc.FFT_STAGES: "stages", lc.FFT_LANES: "lanes", lc.FFT_LANES3: "lanes3", lc.FFT_TMA: "tma", lc.FFT_TMA4: "tma4",
             lc.FFT_PLANE4: "plane4"}
    return {int(n): names.get(lc.fft_variant(int(n)), "-") for n in sorted(set(ns))}


def config_of(workload, w=None, extra=None):
    """The `config` object, the same for both arms of one workload."""
    c = {"workload": f"{workload}: {WORKLOADS[workload]}"}
    if w is not None:
        c.update({"grid": w.n, "box_mpc": w.box, "steps_in_run": w.steps.n_steps,
                  "history": "bf16" if w.history else "fp32"})
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------- c4: uneven instances
def run_batched(args):
    """16 uneven instances, one batch-graph replay per step."""
    import torch

    import paper_1502_02294_gb300 as lc
    import synth

    lc.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    ws = synth.batched_instances()
    window = 8
    plans, srcs, outs = [], [], []
    for w in ws:
        p = lc.Plan.from_workload(w, stream=stream)
        p.prepare(w.steps.n_shell, w.steps.n_shell + window)
        plans.append(p)
        srcs.append([(torch.from_numpy(w.cat.active(s)[0]).to(dev), torch.from_numpy(w.cat.active(s)[1]).to(dev))
                     for s in range(w.steps.n_steps)])
        outs.append(torch.empty((w.n,) * 3, dtype=torch.float32, device=dev))

    def refill():
        for p, w, sr in zip(plans, ws, srcs):
            p.reset()
            for s in range(w.steps.n_shell):
                p.push(s, *sr[s])

    graphs = [lc.BatchGraph(plans, [w.steps.n_shell + k for w in ws],
                            [sr[w.steps.n_shell + k] for w, sr in zip(ws, srcs)], outs) for k in range(window)]
    flush = torch.empty(args.flush_mb << 20, dtype=torch.uint8, device=dev)
    refill()
    for k in range(min(max(3, args.warmup), window)):
        graphs[k].launch(stream)
    torch.cuda.synchronize()
    refill()
    sampler = ClockSampler(0)
    sampler.start()
    launches0 = lc.kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        k = i % window
        if i and k == 0:
            refill()
        flush.zero_()
        evs[i][0].record(stream)
        graphs[k].launch(stream)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    launches = lc.kernel_launches() - launches0
    clocks = sampler.stop()
    per = np.array([a.elapsed_time(b) for a, b in evs])
    T = per.sum() / 1e3
    # the alternative form: the same steps as one step graph per instance,
    # launched one instance after another on one stream (no overlap)
    sgs = [[p.graph(w.steps.n_shell + k, *sr[w.steps.n_shell + k], o) for k in range(window)]
           for p, w, sr, o in zip(plans, ws, srcs, outs)]
    refill()
    seq_ms = []
    for i in range(args.steps):
        k = i % window
        if i and k == 0:
            refill()
        flush.zero_()
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        for sg in sgs:
            sg[k].launch()
        b_.record(stream)
        seq_ms.append((a_, b_))
    torch.cuda.synchronize()
    T_seq = sum(a_.elapsed_time(b_) for a_, b_ in seq_ms) / 1e3
    for sg in sgs:
        for g in sg:
            g.close()
    # MAC roofline: the same steps with per-instance timed graphs, one instance at a time
    mac_ms, mac_bytes = 0.0, 0.0
    refill()
    for p in plans:
        p.set_timing(True)
        p.timing(reset=True)
    tgs = [[p.graph(w.steps.n_shell + k, *sr[w.steps.n_shell + k], o) for k in range(window)]
           for p, w, sr, o in zip(plans, ws, srcs, outs)]
    for p in plans:
        p.set_timing(False)
    for k in range(window):
        for tg in tgs:
            tg[k].launch()
    torch.cuda.synchronize()
    for p, w in zip(plans, ws):
        ph = p.timing(reset=True)
        mac_ms += ph["mac_x"][0]
        nk = w.n * w.n * (w.n // 2 + 1)
        for k in range(window):
            s = w.steps.n_shell + k
            nsh, A = active_shell_work(p, w, s)
            mac_bytes += nk * (8 * nsh + 8) + p.wedge_size * 4 * A
    for tg in tgs:
        for g in tg:
            g.close()
    peak, peak_src = hbm_peak()
    mac_gbs = mac_bytes / (mac_ms / 1e3) / 1e9 if mac_ms > 0 else None
    # e2e: host buffers through the plain batched call
    host_in = [[(np.ascontiguousarray(w.cat.active(s)[0]), np.ascontiguousarray(w.cat.active(s)[1]))
                for s in range(w.steps.n_steps)] for w in ws]
    refill()
    e2e_t, h2d = 0.0, 0
    for i in range(args.steps):
        k = i % window
        if i and k == 0:
            refill()
        torch.cuda.synchronize()
        tic = time.perf_counter()
        for p, w, hi in zip(plans, ws, host_in):
            s = w.steps.n_shell + k
            p.push(s, *hi[s])
        for p, w in zip(plans, ws):
            o = np.empty((w.n,) * 3, dtype=np.float32)
            p.field(w.steps.n_shell + k, o)
        e2e_t += time.perf_counter() - tic
        h2d += sum(hi[w.steps.n_shell + k][0].nbytes + hi[w.steps.n_shell + k][1].nbytes for w, hi in zip(ws, host_in))
    # error_vs_fp64 and cpu_baseline: the batch graph's first window step of
    # the three smallest instances against the FP64 oracle on sampled cells
    err, cpu = None, None
    if not args.no_cpu_baseline:
        import oracle

        refill()
        graphs[0].launch(stream)
        torch.cuda.synchronize()
        picks = sorted(range(len(ws)), key=lambda i: (ws[i].n, i))[:3]
        rows, times, spent_all = [], [], 0.0
        for i in picks:
            w = ws[i]
            s = w.steps.n_shell
            rate, spent, desc, samples = oracle_sample(w, [s], cells_per_step=2048, seed=400 + i)
            J = outs[i].cpu().numpy().reshape(-1)
            rows.append(sample_errors(f"instance {i} ({w.n}^3, {w.steps.n_shell} shells) step {s}", J, samples[s]))
            times.append(1.0 / rate)
            spent_all += spent
        err = error_summary(rows, 0)
        cpu = {"value": len(times) / float(np.sum(times)), "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
               "sample": f"instances {picks} (the three smallest grids), their first timed step each: " + desc,
               "seconds": round(spent_all, 2)}
    for g in graphs:
        g.close()
    for p in plans:
        p.close()
    n_inst = len(ws)
    line = {
        "metric": METRIC, "value": n_inst * args.steps / T, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of("c4", extra={"instances": n_inst, "grids": [w.n for w in ws],
                                         "shells": [w.steps.n_shell for w in ws]}),
        "details": {"timed_window_steps": window, "fft_passes": fft_choices([w.n for w in ws]),
                    "l2": f"flushed between timed steps ({args.flush_mb} MB write outside the events)",
                    "inputs": "device-resident"},
        "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99))},
        "roofline": {"bound": "hbm", "kernel": "shell MAC fused with the inverse x pass (all instances)",
                     "achieved": mac_gbs, "peak": peak, "unit": "GB/s",
                     "frac": (mac_gbs / peak) if mac_gbs else None, "traffic": None, "peak_source": peak_src},
        "clocks": clocks,
        "e2e": {"value": n_inst * args.steps / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d // args.steps),
                "d2h_bytes_per_step": int(sum(4 * w.n ** 3 for w in ws))},
        "gpu_launches": int(launches), "cpu_baseline": cpu, "error_vs_fp64": err,
        "launch": "one batch CUDA graph per step: 16 parallel branches (one per instance)",
        "instances_one_after_another": {"fields_per_s": n_inst * args.steps / T_seq,
                                         "form": "one step graph per instance, launched in turn on one stream"},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- c5: serving
def run_serving(args):
    """Continuous batching of field requests from the 8 served simulations
    (128^3..512^3, BF16 history), beside the plain FP32 one-instance path on
    the same requests."""
    import torch

    import paper_1502_02294_gb300 as lc
    import synth
    from paper_1502_02294_gb300.serve import Request, Server

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    lc.build()
    K = args.steps
    ws = synth.served_simulations(served_steps=max(32, K))
    grids = [w.n for w in ws]
    shells = [w.steps.n_shell for w in ws]

    def fill(p, w):
        for s in range(w.steps.n_shell):
            p.push(s, *w.cat.active(s))

    def requests():
        return [Request(w.name, s, *w.cat.active(s)) for w in ws
                for s in range(w.steps.n_shell, w.steps.n_shell + K)]

    def poisson(reqs, rate, seed=7):
        # Poisson arrivals of the whole stream; each simulation's requests keep step order
        rng = np.random.default_rng(seed)
        t = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
        arr = [0.0] * len(reqs)
        for slot, i in enumerate(rng.permutation(len(reqs))):
            arr[i] = float(t[slot])
        for w in ws:
            idx = [i for i, r in enumerate(reqs) if r.sim == w.name]
            for i, tt in zip(idx, sorted(arr[i] for i in idx)):
                arr[i] = tt
        return arr

    budget = int(0.6 * torch.cuda.get_device_properties(dev).total_memory)
    srv = Server(hbm_budget_bytes=budget, slots=4, retain=True, priorities=not args.equal_priorities)
    for w in ws:
        srv.add_simulation(w.name, w, w.steps.n_shell, w.steps.n_shell + K - 1, fill=lambda p, w=w: fill(p, w))
    admitted = [n for n, s in srv.sims.items() if s.plan is not None]
    if len(admitted) < len(ws):
        raise RuntimeError(f"HBM budget {budget} admits {len(admitted)} of {len(ws)} simulations at once")
    torch.cuda.synchronize()
    # warm-up pass (autotuned kernels, every table touched), then the timed ones
    srv.run_stream(reqs := requests(), [0.0] * len(reqs), limit_s=600.0)
    srv.rewind()
    sampler = ClockSampler(dev.index)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    launches0 = lc.kernel_launches()
    sat = srv.run_stream(reqs := requests(), [0.0] * len(reqs), limit_s=600.0)
    launches = lc.kernel_launches() - launches0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    t_sat = max_over_ranks(sat["device_seconds"], dev)
    value = world * sat["requests"] / t_sat
    srv.rewind()
    pois = srv.run_stream(reqs := requests(), poisson(reqs, 0.8 * sat["fields_per_s"]), limit_s=600.0)
    # end to end: host sources (page-locked staging) in, every field copied to page-locked host memory
    srv.host_outputs = True
    for sim in srv.sims.values():
        for sl in sim.slots:
            sl.out = torch.empty((sim.workload.n,) * 3, dtype=torch.float32).pin_memory()
    for _ in range(2):  # the first pass sets up the library's output stages (untimed)
        srv.rewind()
        e2e = srv.run_stream(reqs := requests(), [0.0] * len(reqs), limit_s=600.0)
    e2e_t = max_over_ranks(e2e["device_seconds"], dev)
    h2d = sum(r.pos.nbytes + r.lum.nbytes for r in reqs)
    srv.host_outputs = False
    for sim in srv.sims.values():
        for sl in sim.slots:
            sl.out = None
    # shell-MAC roofline of the served steps: each simulation alone, phase events on its stream
    mac_ms, mac_bytes, mac_launches = 0.0, 0.0, 0
    for w in ws:
        sim = srv.sims[w.name]
        p = sim.plan
        srv.rewind()
        p.set_timing(True)
        p.timing(reset=True)
        out = torch.empty((w.n,) * 3, dtype=torch.float32, device=dev)
        with torch.cuda.stream(sim.stream):
            for s in range(w.steps.n_shell, w.steps.n_shell + K):
                p.push(s, *w.cat.active(s))
                p.field(s, out)
        ph = p.timing(reset=True)
        p.set_timing(False)
        mac_ms += ph["mac_x"][0]
        mac_launches += ph["mac_x"][1]
        nk = w.n * w.n * (w.n // 2 + 1)
        for s in range(w.steps.n_shell, w.steps.n_shell + K):
            nsh, A = active_shell_work(p, w, s)
            mac_bytes += nk * (4 * nsh + 8) + p.wedge_size * 4 * A
        del out
    peak, peak_src = hbm_peak()
    mac_gbs = mac_bytes / (mac_ms / 1e3) / 1e9 if mac_ms > 0 else None
    # served fields against the FP64 oracle (and the CPU baseline): the
    # simulations up to 256^3, first served step, sampled cells
    checked = [w for w in ws if w.n <= 256]
    errs, cpu_times, cpu_spent, cpu_desc = [], [], 0.0, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        for w in checked:
            sim = srv.sims[w.name]
            srv.rewind()
            s = w.steps.n_shell
            out = torch.empty((w.n,) * 3, dtype=torch.float32, device=dev)
            with torch.cuda.stream(sim.stream):
                sim.plan.push(s, *w.cat.active(s))
                sim.plan.field(s, out)
            sim.stream.synchronize()
            J = out.reshape(-1).cpu().numpy()
            rate, spent, desc, samp = oracle_sample(w, [s], 2048, seed=31)
            errs.append(sample_errors(f"{w.name} ({w.n}^3, {w.steps.n_shell} shells) step {s}", J, samp[s]))
            cpu_times.append(1.0 / rate)
            cpu_spent += spent
            cpu_desc = desc
        oracle_threads = oracle.threads()
    srv.close()
    del srv
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    def plain_fp32():
        """The same requests, one simulation at a time in FP32 history: eager
        push + field per request on the default stream, no graph, no overlap;
        tables and history filled before the clock starts."""
        total, n = 0.0, 0
        for w in ws:
            wf = dataclasses.replace(w, history=synth.HISTORY_FP32)
            sh = w.steps.n_shell
            plan = lc.Plan.from_workload(wf)
            plan.prepare(sh, sh + K)
            fill(plan, wf)
            reqs = [wf.cat.active(s) for s in range(sh, sh + K)]
            out = torch.empty((w.n,) * 3, dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for k, (pos, lum) in enumerate(reqs):
                plan.push(sh + k, torch.from_numpy(pos).to("cuda"), torch.from_numpy(lum).to("cuda"))
                plan.field(sh + k, out)
            b.record()
            b.synchronize()
            total += a.elapsed_time(b) / 1e3
            n += len(reqs)
            plan.close()
            del out
            torch.cuda.empty_cache()
        return n / total, total

    plain_rate, plain_s = plain_fp32()
    c3 = None
    if not args.no_c3:
        a3 = parse(["--workload", "c3", "--steps", "16", "--warmup", "3", "--no-cpu-baseline"])
        c3 = run_single(a3, synth.config("c3"), {}, quick=True)
    if rank != 0:
        return 0
    cpu = None
    if cpu_times:
        cpu = {"value": len(cpu_times) / sum(cpu_times), "unit": UNIT, "cores": oracle_threads, "kind": "oracle",
               "sample": f"simulations {[w.name for w in checked]} (N = {[w.n for w in checked]}), first served step "
                         f"each; per simulation: {cpu_desc}; value = simulations / sum of their extrapolated "
                         f"full-field times (the 384^3 and 512^3 simulations are not sampled: their Green's "
                         f"functions alone take the oracle 10-20 s each)",
               "seconds": round(cpu_spent, 2)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": sat["requests"],
        "warmup": sat["requests"], "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic",
        "config": config_of("c5", extra={"grids": grids, "shells": shells, "requests_per_sim": K}),
        "details": {"hbm_budget_bytes": budget, "admitted_at_once": len(admitted), "slots_per_sim": 4,
                    "stream_priorities": "equal" if args.equal_priorities else "by grid size (small first)",
                    "fft_passes": fft_choices(grids),
                    "mac_kernel": {k: v for k, v in lc.autotune_report().items() if k.startswith("mac")},
                    "l2": "no flush: every request streams its simulation's history ring (0.55-26 GB, far above "
                          "the 129 MB L2) from HBM",
                    "inputs": "host sources staged through page-locked slots, fields on the device",
                    "timing": "device: CUDA events around the whole stream (every simulation's stream waits on "
                              "the start event; the end event waits on every stream); max over ranks",
                    "poisson_rate_fields_per_s": 0.8 * sat["fields_per_s"]},
        "latency_ms": {"saturation_p50": sat["p50_ms"], "saturation_p99": sat["p99_ms"],
                       "poisson_p50": pois["p50_ms"], "poisson_p99": pois["p99_ms"],
                       "poisson_p50_without_admission_wait": pois["p50_ms_without_admission_wait"],
                       "poisson_p99_without_admission_wait": pois["p99_ms_without_admission_wait"],
                       "poisson_service_p50": pois["service_p50_ms"], "poisson_service_p99": pois["service_p99_ms"],
                       "poisson_by_grid": pois["by_grid"],
                       # the mix spans about 20x in service time (128^3 to 512^3), so the
                       # overall p99/p50 compares different request sizes; per grid size:
                       "poisson_p99_over_p50_by_grid": {n: (g["p99_ms"] / g["p50_ms"]) if g["p50_ms"] else None
                                                        for n, g in pois["by_grid"].items()},
                       "poisson_p99_over_p50_by_grid_max": max((g["p99_ms"] / g["p50_ms"])
                                                               for g in pois["by_grid"].values() if g["p50_ms"])},
        "poisson_fields_per_s": pois["fields_per_s"],
        "plain_fp32_one_instance": {"fields_per_s": plain_rate, "seconds": plain_s,
                                    "served_over_plain": value / world / plain_rate,
                                    "path": "FP32 history, one plan at a time, eager push + field per request, "
                                            "no graph, no overlap (tables and history prepared untimed); CUDA events"},
        "cell_shell_mac_per_s": None,
        "roofline": {"bound": "hbm", "kernel": "shell-MAC phase of every served step (each simulation alone): "
                     "k_mac_ws paired (ws2) or the autotuned variant, fused with the inverse x pass",
                     "achieved": mac_gbs, "peak": peak, "unit": "GB/s",
                     "frac": (mac_gbs / peak) if mac_gbs else None,
                     "traffic": MAC512_TRAFFIC["bytes"] if MAC512_TRAFFIC["sources"] == mac_sources_hash() else None,
                     "traffic_algorithmic": MAC512_TRAFFIC["algorithmic"],
                     "traffic_note": "per launch of the dominant kernel, k_mac_ws<512, bf16, pair> at 96 slices: "
                                     "DRAM bytes scaled from a 16-slice capture (" + MAC512_TRAFFIC["from"] + "), "
                                     "reads x 96/16, writes as captured",
                     "peak_source": peak_src, "bytes": mac_bytes, "ms": mac_ms, "launches": mac_launches,
                     "bytes_per_unit": "N_k (4 A + 8) + 4 W A per field (N_k = N^2 (N/2+1) modes, A active "
                                       "slices with sources, W wedge rows)"},
        "clocks": clocks,
        "e2e": {"value": world * e2e["requests"] / e2e_t, "unit": UNIT,
                "h2d_bytes_per_step": int(h2d / max(1, len(reqs))),
                "d2h_bytes_per_step": int(sum(4 * w.n ** 3 for w in ws) / len(ws)),
                "api": "Server with host sources (page-locked staging) and host outputs (lc_retarded_field_async "
                       "into page-locked memory, polled with lc_plan_poll)"},
        "gpu_launches": int(launches),
        "cpu_baseline": cpu,
        "error_vs_fp64": error_summary(errs, 1) if errs else None,
        "launch": "per-simulation streams, requests launched as they arrive (continuous batching)",
    }
    mac_cells = sum(w.n * w.n * (w.n // 2 + 1) * w.steps.n_shell * K for w in ws)
    line["cell_shell_mac_per_s"] = world * mac_cells / t_sat
    if c3 is not None:
        line["c3_single_instance"] = {k: c3[k] for k in ("value", "unit", "ms_per_step", "latency_ms", "roofline",
                                                         "phase_ms_per_step", "config") if k in c3}
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum) of the
# shell-MAC launch, from the captures summarised in profiles/, valid only for
# the kernel sources they were taken with: the warp-specialised kernels
# (all of lc_mac.cuh; the kernel the c3 and served 512^3 lines run).  c3 is the
# c3s capture (32 slices) with its reads scaled to 128 slices.  The 128^3
# line has none: its steps mix three MAC kernels, and a capture over a whole
# window of launches is beyond what this pool's profiling rules allow.
WS_SOURCES = "260d34c3405dd767"
MAC_TRAFFIC = {
    "c3": {"sources": WS_SOURCES, "bytes": 4 * 1.192879e9 + 73.619e6,
           "from": "profiles/k_mac_ws_256_bf16_pair.md (c3s, reads x 128/32)"},
}


# the served 512^3 MAC launch (96 slices, BF16, paired kernel): DRAM traffic
# scaled from the c5s capture (16 slices: reads x 96/16, writes as captured)
# and the launch's algorithmic bytes N_k (4 A + 8) + 4 W A
MAC512_TRAFFIC = {"sources": WS_SOURCES, "bytes": 4.877360555e9 * 96 / 16 + 0.598957994e9,
                  "algorithmic": 67371008 * (4 * 96 + 8) + 4 * 2862209 * 96,
                  "from": "profiles/k_mac_ws_512_bf16_pair.md"}


def mac_sources_hash():
    """Hash of the warp-specialised MAC kernels' sources (lc_mac.cuh)."""
    import hashlib

    with open(os.path.join(ROOT, "paper_1502_02294_gb300", "csrc", "lc_mac.cuh"), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def mac_traffic(workload):
    t = MAC_TRAFFIC.get(workload)
    if t is None or t["sources"] != mac_sources_hash():
        return None, None
    return t["bytes"], t["from"]


DEFAULT_STEPS = {"c1": 2048, "c2": 2048, "c3": 64, "c3s": 32, "c5s": 16, "c5m": 16, "c4": 32, "c5": 20}


# ---------------------------------------------------------------- single instance (c1, c2, c3, c3s)
def run_single(args, w, variant, quick=False):
    """One simulation replayed as one CUDA graph per step; returns the JSON
    line (rank 0) or None.  quick: the headline and roofline only (no e2e,
    CPU baseline or error check), for the extra key of the serving line."""
    import torch

    import paper_1502_02294_gb300 as lc
    import synth

    world = 1 if quick else int(os.environ.get("WORLD_SIZE", "1"))
    rank = 0 if quick else int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif not quick:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    lc.build()
    stream = torch.cuda.current_stream()
    plan = lc.Plan.from_workload(w, stream=stream)
    T = w.steps.n_steps
    t_first = 0 if w.steps.kind != synth.STEPS_EQUAL_TAU else w.steps.n_shell
    plan.prepare(t_first, T)  # the observed steps' Green's function tables (plan time)
    # device-resident inputs of every step
    src_dev = []
    for s in range(T):
        pos, lum = w.cat.active(s)
        src_dev.append((torch.from_numpy(pos).to(dev), torch.from_numpy(lum).to(dev)))
    out = torch.empty((w.n,) * 3, dtype=torch.float32, device=dev)
    out_inst = torch.empty_like(out) if args.fdiff else None
    out_fdiff = torch.empty_like(out) if args.fdiff else None
    flush = torch.empty(args.flush_mb << 20, dtype=torch.uint8, device=dev)

    def fdiff_after(s):
        # the instantaneous field of step s and f_diff = (J_inst - J) / J per cell
        plan.instant_field(s, out_inst)
        lc.fdiff_map(out, out_inst, out_fdiff, stream=stream)
    # timed window: every step for the equal-time runs; for the equal-conformal-time
    # run the last n_shell/4 steps, after n_shell untimed fill steps (history only)
    t0 = 0 if w.steps.kind != synth.STEPS_EQUAL_TAU else w.steps.n_shell
    work = {s: active_shell_work(plan, w, s) for s in range(t0, T)}
    nk = w.n * w.n * (w.n // 2 + 1)

    def refill():
        plan.reset()
        for s in range(t0):
            plan.push(s, *src_dev[s])

    # one CUDA graph per observed step (push + field on device buffers).  The
    # headline pass replays graphs without instrumentation; a second pass
    # replays graphs captured with the per-phase events inside, which time the
    # shell-MAC kernel on its own for the roofline.
    window = T - t0
    graphs = {s: plan.graph(s, *src_dev[s], out) for s in range(t0, T)}
    plan.set_timing(True)
    graphs_timed = {s: plan.graph(s, *src_dev[s], out) for s in range(t0, T)}
    plan.set_timing(False)
    # which shell-MAC kernel the autotuner picked for each active-slice count
    tag = f"/N{w.n}/{'bf16' if w.history else 'fp32'}/"
    mac_choice = {k.rsplit("/", 1)[1]: v for k, v in lc.autotune_report().items() if tag in k}

    def run_pass(gs, evs=None, nvtx=False):
        refill()
        steps_done = []
        for i in range(args.steps):
            s = t0 + i % window
            if i and s == t0:
                refill()  # history restarts (untimed: outside the events)
            flush.zero_()  # L2 flush between timed steps, outside the events
            if evs:
                evs[i][0].record(stream)
            if nvtx:
                torch.cuda.nvtx.range_push("step")  # lets a profiler select the timed replays
            gs[s].launch()
            if args.fdiff:
                fdiff_after(s)
            if nvtx:
                torch.cuda.nvtx.range_pop()
            if evs:
                evs[i][1].record(stream)
            steps_done.append(s)
        return steps_done

    refill()
    for i in range(max(3, args.warmup)):
        s = t0 + i % window
        if i and s == t0:
            refill()
        graphs[s].launch()
        if args.fdiff:
            fdiff_after(s)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = lc.kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    done_steps = run_pass(graphs, evs, nvtx=True)
    torch.cuda.synchronize()
    launches = lc.kernel_launches() - launches0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    # profiling pass (same steps, graphs with in-graph phase events)
    plan.timing(reset=True)
    mac_steps = run_pass(graphs_timed)
    torch.cuda.synchronize()
    phases = plan.timing(reset=True)
    for g in list(graphs.values()) + list(graphs_timed.values()):
        g.close()
    fdiff_stats = None
    if args.fdiff:
        # the profiling pass ended on the same step as the timed one: its maps are in place
        f = out_fdiff.double()
        lit = out > 0
        fa = f[lit].abs()
        fdiff_stats = {"step": done_steps[-1], "cells_with_flux": int(lit.sum()),
                       "mean_abs": float(fa.mean()) if fa.numel() else None,
                       "p50_abs": float(fa.kthvalue(max(1, fa.numel() // 2))[0]) if fa.numel() else None,
                       "p99_abs": float(fa.kthvalue(max(1, int(0.99 * fa.numel())))[0]) if fa.numel() else None,
                       "frac_over_10pct": float((fa > 0.1).double().mean()) if fa.numel() else None}
    per_step_ms = np.array([a.elapsed_time(b) for a, b in evs])
    t_total = float(per_step_ms.sum()) / 1e3
    t_max = max_over_ranks(t_total, dev)
    value = world * args.steps / t_max
    mac_cells = sum(nk * work[s][0] for s in done_steps)

    # roofline of the dominant kernel (shell MAC fused with the inverse x pass):
    # algorithmic bytes = ring reads (b_h B per k per non-empty shell) + the
    # complex write (8 B per k) + one read of the step's Ghat wedge table
    mac_ms, mac_launches = phases["mac_x"]
    W = plan.wedge_size
    hb = 4 if w.history else 8
    mac_bytes = sum(nk * (hb * work[s][0] + 8) + W * 4 * work[s][1] for s in mac_steps)
    peak, peak_src = hbm_peak()
    mac_gbs = mac_bytes / (mac_ms / 1e3) / 1e9 if mac_ms > 0 else None
    # the captured DRAM traffic is for the Lyman-Werner kernel's shell count
    traffic, traffic_src = mac_traffic(args.workload) if args.kernel == "lw" else (None, None)
    phase_share = {k: round(v[0] / max(1e-12, sum(x[0] for x in phases.values())), 4) for k, v in phases.items()}

    e2e, e2e_pipe, cpu, err = None, None, None, None
    if not quick:
        # end to end through the public API: pinned host inputs, host output
        pinned = []
        for s in range(T):
            pos, lum = w.cat.active(s)
            pinned.append((torch.from_numpy(pos).pin_memory(), torch.from_numpy(lum).pin_memory()))
        host_out = torch.empty((w.n,) * 3, dtype=torch.float32).pin_memory()
        host_fdiff = torch.empty((w.n,) * 3, dtype=torch.float32).pin_memory() if args.fdiff else None

        def e2e_field(s):
            if not args.fdiff:
                plan.field(s, host_out)  # synchronises and copies to the host
                return
            plan.field(s, out)
            fdiff_after(s)
            host_out.copy_(out, non_blocking=True)
            host_fdiff.copy_(out_fdiff, non_blocking=True)
            stream.synchronize()

        refill()
        e_cursor = t0
        for _ in range(max(3, args.warmup)):
            plan.push(e_cursor, *pinned[e_cursor])
            e2e_field(e_cursor)
            e_cursor += 1
            if e_cursor == T:
                refill()
                e_cursor = t0
        e2e_t = 0.0
        h2d = 0
        for i in range(args.steps):
            s = e_cursor
            if s == t0:
                refill()
            flush.zero_()
            torch.cuda.synchronize()
            tic = time.perf_counter()
            plan.push(s, *pinned[s])
            e2e_field(s)
            e2e_t += time.perf_counter() - tic
            h2d += pinned[s][0].numel() * 8 + pinned[s][1].numel() * 8
            e_cursor = t0 + (s + 1 - t0) % (T - t0)
        e2e_t = max_over_ranks(e2e_t, dev)
        e2e = {"value": world * args.steps / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d // args.steps),
               "d2h_bytes_per_step": int(w.n ** 3 * 4 * (2 if args.fdiff else 1))}
        if args.e2e_pipelined and not args.fdiff:
            # the same steps and copies through field_async: step i's output copy
            # drains while step i+1 computes; refills (history restarts) untimed
            outs = [torch.empty((w.n,) * 3, dtype=torch.float32).pin_memory() for _ in range(2)]
            refill()
            torch.cuda.synchronize()
            p_t, prev, cur = 0.0, 0, t0
            tic = time.perf_counter()
            for i in range(args.steps):
                if i and cur == t0:
                    if prev:
                        plan.wait(prev)
                    p_t += time.perf_counter() - tic
                    refill()
                    torch.cuda.synchronize()
                    prev = 0
                    tic = time.perf_counter()
                plan.push(cur, *pinned[cur])
                tk = plan.field_async(cur, outs[i % 2])
                if prev:
                    plan.wait(prev)
                prev = tk
                cur = t0 + (cur + 1 - t0) % (T - t0)
            plan.wait(prev)
            p_t += time.perf_counter() - tic
            p_t = max_over_ranks(p_t, dev)
            e2e_pipe = {"value": world * args.steps / p_t, "unit": UNIT,
                        "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                        "d2h_bytes_per_step": e2e["d2h_bytes_per_step"], "api": "Plan.push + Plan.field_async/wait",
                        "l2": "not flushed between steps"}

        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            import oracle

            if args.workload == "c2":
                csteps, ncell = [10, 20, 30, 41, 50, 63], 131072
            elif args.workload == "c1":
                csteps, ncell = [3, 7], w.n ** 3 // 2
            else:
                csteps, ncell = [T - 1], 2048
            rate, spent, desc, samp = oracle_sample(w, csteps, ncell)
            if args.near != "ngp" or args.fdiff:
                desc += "; the sample times the retarded field alone (cell-centred near field, no f_diff map)"
            cpu = {"value": rate, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle", "sample": desc,
                   "seconds": round(spent, 2)}
            if args.near == "ngp":
                # the GPU's fields of the same steps (eager pushes from step 0)
                plan.reset()
                rows = []
                for s in range(max(csteps) + 1):
                    plan.push(s, *src_dev[s])
                    if s in samp:
                        J = plan.field(s, out).reshape(-1).cpu().numpy()
                        rows.append(sample_errors(f"step {s}", J, samp[s]))
                err = error_summary(rows, w.history)

    out_line = None
    if rank == 0:
        out_line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32" if w.history else "f32", "data": "synthetic",
            "config": config_of(args.workload, w, variant),
            "details": {"timed_window": [t0, T], "ring_slots": plan.n_ring,
                        "mac_kernel": dict(sorted(mac_choice.items(), key=lambda kv: int(kv[0][1:]))),
                        "fft_passes": fft_choices([w.n]),
                        "l2": f"flushed between timed steps ({args.flush_mb} MB write outside the events)",
                        "inputs": "device-resident"},
            "cell_shell_mac_per_s": world * mac_cells / t_max,
            "latency_ms": {"p50": float(np.percentile(per_step_ms, 50)),
                           "p99": float(np.percentile(per_step_ms, 99))},
            "roofline": {"bound": "hbm", "kernel": "shell-MAC phase: the autotuned kernel (details.mac_kernel: gather "
                         "= k_cols<N,+1,MAC>, bulk = k_mac_tma + Nyquist k_cols, ws/ws2 = k_mac_ws single/paired), "
                         "fused with the inverse x pass",
                         "achieved": mac_gbs, "peak": peak, "unit": "GB/s",
                         "frac": (mac_gbs / peak) if mac_gbs else None,
                         "traffic": traffic, "traffic_source": traffic_src, "peak_source": peak_src,
                         "bytes_per_launch": mac_bytes / max(1, len(mac_steps)),
                         "ms_per_launch": mac_ms / max(1, len(mac_steps))},
            "phase_ms_per_step": {k: v[0] / max(1, len(mac_steps)) for k, v in phases.items()},
            "launch": "one CUDA graph replay per step (push + field captured once per observed step); "
                      "phase times from a second pass of graphs with in-graph events",
            "phase_share": phase_share,
            "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "cpu_baseline": cpu,
            "error_vs_fp64": err,
        }
        if fdiff_stats is not None:
            out_line["fdiff"] = fdiff_stats
        if e2e_pipe is not None:
            out_line["e2e_pipelined"] = e2e_pipe
    plan.close()
    del graphs, graphs_timed, src_dev, flush
    torch.cuda.empty_cache()
    return out_line


# ---------------------------------------------------------------- reference arm (the oracle)
def run_reference(args, w, variant):
    """The FP64 oracle as it stands, on the host cores, on the same workload:
    each step is one observing step's Green's functions plus a cell sample,
    its full-field time extrapolated from the per-cell rate."""
    import oracle
    import synth

    threads = oracle.threads()
    if args.workload == "c5":
        ws = synth.served_simulations(served_steps=max(32, args.steps))
        seq = [(ws[i % len(ws)], ws[i % len(ws)].steps.n_shell + i // len(ws)) for i in range(args.steps)]
        warm = [(ws[0], ws[0].steps.n_shell)] * args.warmup
    else:
        pool = list(range(max(1, w.steps.n_steps // 2), w.steps.n_steps))
        seq = [(w, pool[i % len(pool)]) for i in range(args.steps)]
        warm = [(w, pool[i % len(pool)]) for i in range(args.warmup)]
    for ww, s in warm:
        oracle_sample(ww, [s], 256, dense=False)
    cells = 1024
    times, spent = [], 0.0
    for i, (ww, s) in enumerate(seq):
        r, sp, desc, _ = oracle_sample(ww, [s], cells_per_step=cells, seed=i, dense=False)
        times.append(1.0 / r)
        spent += sp
        if i == 0 and args.workload != "c5":
            cells = int(min(65536, ww.n ** 3, max(64, cells * (120.0 / args.steps) / max(sp, 1e-3))))
    value = len(times) / float(np.sum(times))
    sample = (f"each step: one observing step's Green's functions + {cells} sampled cells (1024 on the first), "
              "full-field time extrapolated from the per-cell rate")
    if args.workload == "c5":
        sample = ("each step: one request of the served mix (simulations round-robin: N = "
                  f"{sorted(set(x.n for x, _ in seq))}), its Green's functions + 1024 sampled cells, full-field time "
                  "extrapolated from the per-cell rate; value = requests / sum of their extrapolated times")
    if args.near != "ngp" or args.fdiff:
        sample += "; the retarded field alone (cell-centred near field, no f_diff map)"
    extra = dict(variant)
    if args.workload == "c5":
        extra.update({"grids": [x.n for x in ws], "shells": [x.steps.n_shell for x in ws],
                      "requests_per_sim": args.steps})
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "value_basis": "extrapolated: full-field times projected from sampled cells (the oracle cannot finish "
                           "whole fields of these grids in minutes)",
            "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            # a step here is the bounded sample that was actually timed; the
            # full field it stands for is `ms_per_field_extrapolated`
            "ms_per_step": 1e3 * spent / max(1, len(seq)), "ms_per_field_extrapolated": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args.workload, None if args.workload == "c5" else w, extra),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu_seconds": spent}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.steps is None:
        args.steps = 16 if (args.impl == "reference" and args.workload != "c5") else DEFAULT_STEPS.get(args.workload, 64)
    rank = int(os.environ.get("RANK", "0"))
    import synth

    w = synth.config(args.workload) if args.workload in ("c1", "c2", "c3", "c3s", "c5s", "c5m") else None
    variant = {}
    if w is not None:
        if args.kernel == "exp":
            w = dataclasses.replace(w, kernel=EXP_KERNEL)
            variant["radial_kernel"] = "exp(-r/30 Mpc), cut off at 80 Mpc"
        if args.near == "subcell":
            w = dataclasses.replace(w, near_mode=1)
            variant["near_field"] = "sub-cell (s^3 sub-samples around each source's own position)"
        if args.fdiff:
            variant["step_adds"] = "instantaneous field (Eq. 18) + f_diff map, inside the timed step"
    if args.impl == "reference":
        if rank != 0:
            return 0
        return run_reference(args, w, variant)
    if args.workload == "c4":
        return run_batched(args)
    if args.workload == "c5":
        return run_serving(args)
    line = run_single(args, w, variant)
    if line is not None:
        print(json.dumps(line))
    import torch

    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and torch.distributed.is_initialized():
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
