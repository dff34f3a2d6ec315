"""Benchmark: cell-updates/s of the FitzHugh-Nagumo RD-CNN stepper on GB300.

Headline workload ("slow growth", Sec. III.A / Table I scale): a 4096 x 4096
FP32 torus, default gene (Sec. II.A), u = v = 0 except a seeded 16 x 16
U[-1, 1] patch at the centre, T = 100000 steps.  One benchmark step = one
pass of the hot path over that input: u = v = ka*x (init kernel) followed by
T applications of Eq. 1 (AUTO variant = temporally blocked kernel).

  value   device-resident input, CUDA events around K steps, cell-updates/s
  e2e     the same through the C ABI with HOST buffers: x copied in (pinned
          host -> device) and (u_T, v_T) read back every step
  roofline  dominant kernel, algorithmic work per launch / measured duration
  cpu_baseline  the FP64 CPU oracle on this host's cores, bounded sample
  batched / adjoint  the two follow-on patterns, each against plain forward
                     runs on the same GPU

``--impl reference`` times the FP64 CPU oracle instead (the reference arm).
Multi-GPU: the workload does not shard (one grid per GPU): N ranks run N
independent replicas (weak scaling) and value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import rdcnn_inputs as inp  # noqa: E402

N_GRID = 4096
T_STEPS = 100_000
PATCH = 16
L2_BYTES = 126 * 2 ** 20
FLOPS_PER_CELL_STEP = 27      # Eq. 1-3 as evaluated: 2 x (3 add + 1 fma) Laplacians + 7 reaction + 4 update
BYTES_PER_CELL_STEP = 16      # FP32: read u, v; write u+, v+
PAPER_MCELLS_4096 = 14545.0   # Table I, PyCUDA on Tesla P100-PCIE, N = 4096 (context only)
METRIC = "Gcell-updates/s @4096^2 FP32 (frac of HBM roofline); batched & adjoint vs plain fwd"
WORKLOAD = (f"slow-growth {N_GRID}x{N_GRID} FP32, {PATCH}x{PATCH} centre patch U[-1,1] seed 0, "
            f"default gene, T={T_STEPS}")


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return {"hbm_gbs": float(pk["hbm_gbs"]), "sm_max_mhz": float(pk.get("sm_max_mhz", 2070.0)),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm_, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm_)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def profiled_traffic(kernel_md: str, k: int, rows: int):
    """DRAM bytes per launch from a committed ncu summary, if the kernel and its launch shape
    are unchanged.

    The summary records a hash of the headers that define the kernel's device code and the
    (k, rows) it was captured with; a different hash or shape yields None.
    """
    import hashlib
    import re

    path = os.path.join(ROOT, "profiles", kernel_md)
    try:
        text = open(path).read()
    except OSError:
        return None, "no profile"
    m = re.search(r"source-sha256-16:\s*([0-9a-f]{16})", text)
    t = re.search(r"dram traffic per launch:\s*([0-9.]+)\s*MB", text)
    shape = re.search(r"launch shape:\s*k=(\d+)\s+rows=(\d+)", text)
    if not m or not t or not shape:
        return None, "profile lacks hash, shape or traffic"
    if (int(shape.group(1)), int(shape.group(2))) != (int(k), int(rows)):
        return None, f"profile taken at k={shape.group(1)} rows={shape.group(2)}"
    csrc = os.path.join(ROOT, "paper_2102_10340_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("common.cuh", "temporal.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != m.group(1):
        return None, "kernel changed since the profile was taken"
    return float(t.group(1)) * 1e6, f"profiles/{kernel_md}"


def profiled_instructions(kernel_md: str):
    """Warp instructions per launch from the same committed summary (None if absent)."""
    import re

    try:
        text = open(os.path.join(ROOT, "profiles", kernel_md)).read()
    except OSError:
        return None
    m = re.search(r"warp instructions per launch:\s*([0-9.]+)\s*M", text)
    return float(m.group(1)) * 1e6 if m else None


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over all ranks (the slowest replica sets the job time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(cells: int, T: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job cell-updates/s (in G) of `world` replicas, each doing steps x T steps on `cells` cells."""
    return cells * T * steps * world / seconds / 1e9


# ----------------------------------------------------------------------------- CPU oracle legs

def oracle_sample(target_s: float = 12.0, n=N_GRID):
    """Time the FP64 oracle on a bounded sample of the headline workload (host cores)."""
    import oracle

    threads = max(1, os.cpu_count() or 1)
    params = inp.default_params()
    x = np.asarray(inp.mid_patch(0, n, n), dtype=np.float32).astype(np.float64)
    u, v = oracle.init_state(x, 1.0)
    u, v = oracle.run(u, v, params, 1, nthreads=threads)  # first touch of the pages
    t0 = time.perf_counter()
    u, v = oracle.run(u, v, params, 2, nthreads=threads)
    one = (time.perf_counter() - t0) / 2
    steps = int(max(1, min(2000, target_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(u, v, params, steps, nthreads=threads)
    dt = time.perf_counter() - t0
    rate = n * n * steps / dt / 1e9
    # the same oracle at 1024^2, one thread and all threads (short samples, ~1.5 s each)
    detail = {}
    xs = np.asarray(inp.smooth_noise(0, 1024, 1024), dtype=np.float32).astype(np.float64)
    for name, nt in (("single_thread_1024", 1), ("all_threads_1024", threads)):
        su, sv = oracle.run(xs, xs, params, 1, nthreads=nt)
        t0 = time.perf_counter()
        oracle.run(su, sv, params, 2, nthreads=nt)
        per = (time.perf_counter() - t0) / 2
        k = int(max(1, min(500, 1.5 / max(per, 1e-6))))
        t0 = time.perf_counter()
        oracle.run(su, sv, params, k, nthreads=nt)
        detail[name] = {"value": 1024 * 1024 * k / (time.perf_counter() - t0) / 1e9, "steps": k, "threads": nt}
    return {"value": rate, "unit": "Gcell-updates/s", "cores": threads, "kind": "oracle",
            "sample": f"{steps} FP64 steps of the {n}x{n} headline grid (OpenMP rows, {threads} threads), "
                      f"{dt:.1f} s", "detail": detail}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, timed as it stands, on the same workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    N = args.grid
    threads = max(1, os.cpu_count() or 1)
    params = inp.default_params()
    x = np.asarray(inp.mid_patch(0, N, N), dtype=np.float32).astype(np.float64)
    # size each step to ~10 s of oracle work so K + W steps finish within minutes
    u, v = oracle.init_state(x, 1.0)
    oracle.run(u, v, params, 1, nthreads=threads)  # first touch of the pages
    t0 = time.perf_counter()
    oracle.run(u, v, params, 2, nthreads=threads)
    one = (time.perf_counter() - t0) / 2
    per_step = int(max(1, min(100, args.T, 10.0 / max(one, 1e-6))))
    for _ in range(args.warmup):
        u, v = oracle.init_state(x, 1.0)
        oracle.run(u, v, params, per_step, nthreads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u, v = oracle.init_state(x, 1.0)
        oracle.run(u, v, params, per_step, nthreads=threads)
    dt = time.perf_counter() - t0
    val = N * N * per_step * args.steps / dt / 1e9
    sample = (f"each step: init + {per_step} FP64 oracle steps of the {N}x{N} grid "
              f"({threads} threads), instead of the workload's T={args.T}")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Gcell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if (N, args.T) == (N_GRID, T_STEPS) else f"{N}x{N} FP32 patch, T={args.T}",
                       "grid": [N, N], "T": args.T, "sample_steps_per_step": per_step},
            "cpu_baseline": {"value": val, "unit": "Gcell-updates/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU legs

def measure_launch_ms(rd, grid, variant, k, launches_per_call, reps, torch):
    """Average duration of one kernel launch, CUDA events on the launching stream."""
    stream = torch.cuda.current_stream()
    T = k * launches_per_call
    grid.run(T, variant=variant, k=k)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for s, e in ev:
        s.record(stream)
        grid.run(T, variant=variant, k=k)
        e.record(stream)
    torch.cuda.synchronize()
    return float(np.mean([s.elapsed_time(e) for s, e in ev])) / launches_per_call


CENN_GENE = {"dt": 0.1, "a": 0.0, "b": 0.0, "eps": 0.0, "c": 1.2, "Du": 0.1, "Dv": 0.0}


def measure_models(rd, torch, N=N_GRID, quick=False):
    """Throughput of the model variants (zero-flux boundary, Chua-Yang CeNN cell) on an N x N
    FP32 grid: the temporal kernel (k = 8, 128 rows) and the single-step kernel, per launch,
    CUDA events on the launching stream."""
    if quick:
        N = 1024
    x = torch.from_numpy(np.asarray(inp.uniform_field(7, N, N), dtype=np.float32)).cuda()
    out = {}
    for name, reaction, boundary, gene in (("fhn_periodic", "fhn", "periodic", inp.default_params()),
                                           ("fhn_zeroflux", "fhn", "zeroflux", inp.default_params()),
                                           ("cenn_periodic", "cenn", "periodic", CENN_GENE),
                                           ("cenn_zeroflux", "cenn", "zeroflux", CENN_GENE)):
        g = rd.Grid(N, N, gene, dtype=torch.float32, reaction=reaction, boundary=boundary)
        g.set_state((1.5 * x).contiguous(), (0.3 * x).contiguous())
        res = {}
        for variant, k, rows in (("temporal", 8, 128), ("step1", 1, 0)):
            g.set_tune(k=k, rows=rows)
            ms = measure_launch_ms(rd, g, variant, k, 4, 10, torch)
            res[variant] = {"k": k, "rows": rows, "launch_ms": ms, "gcell_s": N * N * k / (ms * 1e-3) / 1e9}
        out[name] = res
        g.close()
    return {"grid": [N, N], "dtype": "f32", "models": out,
            "note": "per-launch CUDA-event time; fhn_periodic is the paper's model for comparison"}


def measure_storage(rd, torch, N=N_GRID, quick=False):
    """Throughput of 16-bit state storage (FP32 arithmetic) against FP32 storage on the headline
    grid: the single-step kernel (HBM-bound: 8 instead of 16 algorithmic bytes per cell-step)
    and the temporal kernel (k = 8, 128 rows), per launch, CUDA events on the launching stream."""
    if quick:
        N = 1024
    x = torch.from_numpy(np.asarray(inp.mid_patch(0, N, N), dtype=np.float32)).cuda()
    peaks = load_peaks()
    out = {}
    for name, dt, esz in (("f32", torch.float32, 4), ("bf16", torch.bfloat16, 2), ("f16", torch.float16, 2)):
        g = rd.Grid(N, N, inp.default_params(), dtype=dt)
        g.set_state(x.to(dt), x.to(dt))
        res = {}
        for variant, k, rows in (("temporal", 8, 128), ("step1", 1, 0)):
            g.set_tune(k=k, rows=rows)
            # the single step in windows of 20 back-to-back launches, as for the FP32 single step
            ms = measure_launch_ms(rd, g, variant, k, 20 if variant == "step1" else 4, 10, torch)
            res[variant] = {"k": k, "launch_ms": ms, "gcell_s": N * N * k / (ms * 1e-3) / 1e9}
        gbs = 4 * esz * N * N / (res["step1"]["launch_ms"] * 1e-3) / 1e9
        res["step1"].update({"algorithmic_bytes_per_cell_step": 4 * esz, "achieved_gbs": gbs,
                             "frac_hbm": gbs / peaks["hbm_gbs"]})
        out[name] = res
        g.close()
    return {"grid": [N, N], "storage": out, "error": measure_storage_error(rd, torch, quick=quick),
            "note": "16-bit planes hold the state; every launch computes in FP32 and rounds once on store"}


def measure_storage_error(rd, torch, N=512, quick=False):
    """Accuracy cost of 16-bit storage: normwise distance of u_T (and of the gradient-area
    statistic) from the FP64 kernels' u_T (pinned to the oracle at 1e-12) on an N x N grid,
    default gene, x ~ U[-1, 1] seed 0, u = v = x, for storage formats and steps per launch."""
    x = np.asarray(inp.uniform_field(0, N, N), dtype=np.float32)
    xt = torch.from_numpy(x).cuda()
    Ts = (100, 1000) if quick else (100, 1000, 5000)

    def run(dt, variant, k, T):
        g = rd.Grid(N, N, inp.default_params(), dtype=dt)
        g.set_state(xt.to(dt), xt.to(dt))
        g.run(T, variant=variant, k=k)
        u, v = g.state()
        g.close()
        return u.double(), v.double()

    out = {}
    for T in Ts:
        ru, rv = run(torch.float64, "temporal", 4, T)
        ref_edge = float(rd.grid_summary(ru, rv)[rd.SUMMARY_FIELDS.index("edge_frac")])
        row = {}
        for name, dt, variant, k in (("f32_k8", torch.float32, "temporal", 8), ("bf16_k1", torch.bfloat16, "step1", 1),
                                     ("bf16_k8", torch.bfloat16, "temporal", 8), ("f16_k1", torch.float16, "step1", 1),
                                     ("f16_k8", torch.float16, "temporal", 8)):
            u, v = run(dt, variant, k, T)
            edge = float(rd.grid_summary(u, v)[rd.SUMMARY_FIELDS.index("edge_frac")])
            row[name] = {"normwise_u": float(torch.linalg.norm(u - ru) / torch.linalg.norm(ru)),
                         "edge_frac": edge, "edge_frac_ref": ref_edge}
        out[f"T={T}"] = row
    return {"grid": [N, N], "init": "x ~ U[-1,1] seed 0, u = v = x", "reference": "FP64 kernels", "runs": out}


def measure_image(rd, torch, N=1024, T=10000, quick=False):
    """Image-processing mode: N x N FP32 smooth-noise image (periodic Gaussian blur, sigma = 8,
    of U[0, 1] seed 0, rescaled to [-1, 1]), u = v = x, default gene, T steps.  The four planes
    (16 MiB at 1024^2) stay in L2, so this is an L2-resident number, not an HBM one."""
    from paper_2102_10340_gb300 import autotune

    if quick:
        T = 1000
    x = torch.from_numpy(np.asarray(inp.smooth_noise(0, N, N), dtype=np.float32)).cuda()
    g = rd.Grid(N, N, inp.default_params(), dtype=torch.float32)
    tune = autotune.tune_grid(g, x)
    g.init(x, 1.0).run(64, variant=tune["variant"], k=tune["k"])
    g.init(x, 1.0)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    g.run(T, variant=tune["variant"], k=tune["k"])
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e)
    g.close()
    return {"grid": [N, N], "T": T, "value": N * N * T / (ms * 1e-3) / 1e9, "unit": "Gcell-updates/s",
            "ms": ms, "tune": {k: tune[k] for k in ("variant", "k", "rows")},
            "note": "state + ping-pong = 16 MiB, L2-resident (126 MiB L2)"}


def measure_batched(rd, torch, T=5000, quick=False, tune=None, full_sweep=False):
    """Batched sweep: the 256-instance workload (or its first 32 instances with quick) advanced T
    steps by rdcnn_batch_run, against one instance at a time through the single-grid path."""
    specs = inp.sweep_instances(0)
    if quick and not full_sweep:
        specs = specs[:32]
        T = 500
    b = rd.Batch(specs, dtype=torch.float32)
    xs = []
    for i, s in enumerate(specs):
        x = torch.from_numpy(inp.uniform_field(s["x_seed"], s["nn"], s["nm"])).float()
        xs.append(x)
        b.set_state(i, x, x)
    from paper_2102_10340_gb300 import autotune

    if tune is None:
        tune = autotune.tune_batch(b, trial_steps=40 if not quick else 8)
    b.set_tune(**tune)
    for i, x in enumerate(xs):
        b.set_state(i, x, x)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(); b.run(T); e.record(); torch.cuda.synchronize()
    ms_b = s.elapsed_time(e)
    cells = b.cells()
    # plain forward, one Grid per instance, same stream
    grids = [rd.Grid(sp["nn"], sp["nm"], sp["params"], dtype=torch.float32) for sp in specs]
    for g, x in zip(grids, xs):
        g.set_state(x.cuda(), x.cuda())
    for g in grids:
        g.run(8)
    torch.cuda.synchronize()
    s.record()
    for g in grids:
        g.run(T)
    e.record(); torch.cuda.synchronize()
    ms_p = s.elapsed_time(e)
    for g in grids:
        g.close()
    # on-device search statistics of all instances (reads u and v once: 8 B per cell)
    b.summary(0.05)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        b.summary(0.05)
    t_sum = (time.perf_counter() - t0) / 5
    return {"value": cells * T / (ms_b * 1e-3) / 1e9, "unit": "Gcell-updates/s",
            "instances": len(specs), "T": T, "cells": cells, "ms": ms_b, "tune": tune,
            "plain_fwd_value": cells * T / (ms_p * 1e-3) / 1e9, "plain_fwd_ms": ms_p,
            "vs_plain_fwd": ms_p / ms_b,
            "summary": {"ms": t_sum * 1e3, "gbs": 8 * cells / t_sum / 1e9,
                        "note": "rdcnn_batch_summary, all instances, host wall time incl. result copy"}}


def measure_search(torch, N=256, T=2000, quick=False):
    """(Du, Dv) sweep of Sec. III.A: an 8 x 8 grid of genes around the defaults, 16 x 16
    centre patch, statistics at 4 checkpoints; whole-harness cell-updates/s and labels."""
    from paper_2102_10340_gb300 import search

    if quick:
        T = 200
    genes = search.du_dv_grid(np.linspace(0.05, 0.75, 8), np.linspace(0.3, 1.0, 8))
    search.sweep(genes[:2], N=N, T=8, checkpoints=1)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = search.sweep(genes, N=N, T=T, checkpoints=4)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    labels = {k: res["labels"].count(k) for k in sorted(set(res["labels"]))}
    return {"genes": len(genes), "grid": [N, N], "T": T, "ms": dt * 1e3,
            "value": len(genes) * N * N * T / dt / 1e9, "unit": "Gcell-updates/s (incl. statistics)",
            "labels": labels}


def measure_snapshots(rd, grid, x_dev, torch, T=2000, every=200):
    """Snapshot capture (the paper's A_show / B_show, every `every` steps to pinned host
    memory) against the same run without snapshots, on the headline grid, with the paper's
    loop structure (one single-step launch per step)."""
    grid.set_tune(k=1, rows=0)
    grid.init(x_dev, 1.0).run(T)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grid.init(x_dev, 1.0).run(T)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    grid.init(x_dev, 1.0)
    us, vs = grid.run_snapshots(T, every, out="host", n_stage=2)  # warm; allocates the pinned outputs
    grid.init(x_dev, 1.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grid.run_snapshots(T, every, out="host", n_stage=2, buffers=(us, vs))
    t_snap = time.perf_counter() - t0
    n = T // every + 1
    nbytes = int(2 * n * us[0].numel() * us.element_size())
    return {"T": T, "every": every, "snapshots": n, "bytes_to_host": nbytes, "kernel": "single step (k = 1)",
            "ms": t_snap * 1e3, "plain_ms": t_plain * 1e3, "overhead": t_snap / t_plain - 1.0,
            "host_gbs": nbytes / t_snap / 1e9}


def measure_adjoint(rd, torch, N=512, T=2000, quick=False):
    if quick:
        T = 200
    p = inp.default_params()
    x = torch.from_numpy(inp.uniform_field(0, N, N)).float().cuda()
    target = torch.from_numpy(inp.checkerboard(0, N, N)).float().cuda()
    g = rd.Grid(N, N, p, dtype=torch.float32)
    g.set_state(x, x).run(T)
    uT = g.u.clone()
    gu = (2.0 * (uT - target) / uT.numel()).contiguous()
    gv = torch.zeros_like(gu)
    ws = torch.empty(g.adjoint_workspace_bytes(T), dtype=torch.uint8, device="cuda")
    g.adjoint(T, x, x, gu, gv, workspace=ws)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.adjoint(T, x, x, gu, gv, workspace=ws)
    t_adj = time.perf_counter() - t0
    # one checkpoint: the reverse sweep reads all T states, rebuilt once (no separate
    # checkpoint sweep), at T states of memory (4 GiB here) instead of ~2 sqrt(T)
    del ws
    ws1 = torch.empty(g.adjoint_workspace_bytes(T, 1), dtype=torch.uint8, device="cuda")
    g.adjoint(T, x, x, gu, gv, 1, workspace=ws1)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.adjoint(T, x, x, gu, gv, 1, workspace=ws1)
    t_all = time.perf_counter() - t0
    all_bytes = ws1.numel()
    del ws1
    # every state a checkpoint: the adjoint's own forward sweep stores all T states (4 GiB here)
    # and the reverse sweep reads them, rebuilding nothing
    wsT = torch.empty(g.adjoint_workspace_bytes(T, T), dtype=torch.uint8, device="cuda")
    g.adjoint(T, x, x, gu, gv, T, workspace=wsT)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.adjoint(T, x, x, gu, gv, T, workspace=wsT)
    t_every = time.perf_counter() - t0
    every_bytes = wsT.numel()
    del wsT
    g.set_state(x, x).run(T)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.set_state(x, x).run(T)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0

    # training-loop form: the forward that produces the loss records a tape (rdcnn_run_record),
    # the backward reads it (rdcnn_adjoint_tape) instead of sweeping forward again
    def tape_pass(nck):
        g.set_state(x, x)
        tape = g.run_record(T, nck)
        _, wb = g.tape_bytes(T, nck)
        wst = torch.empty(wb, dtype=torch.uint8, device="cuda")
        g.adjoint_tape(T, tape, gu, gv, nck, workspace=wst)  # warm
        g.set_state(x, x)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.run_record(T, nck, tape=tape)
        torch.cuda.synchronize()
        t_rec = time.perf_counter() - t0
        t0 = time.perf_counter()
        g.adjoint_tape(T, tape, gu, gv, nck, workspace=wst)
        t_bwd = time.perf_counter() - t0
        nb = tape.numel()
        del tape, wst
        return {"n_checkpoints": nck if nck else int(np.ceil(np.sqrt(T))), "tape_bytes": int(nb),
                "record_ms": t_rec * 1e3, "backward_ms": t_bwd * 1e3, "record_over_fwd": t_rec / t_fwd,
                "backward_over_fwd": t_bwd / t_fwd, "fwd_plus_bwd_over_fwd": (t_rec + t_bwd) / t_fwd}

    tape_sqrt = tape_pass(0)
    tape_all = tape_pass(T)
    g.close()
    return {"grid": [N, N], "T": T, "checkpoints": int(np.ceil(np.sqrt(T))), "adjoint_ms": t_adj * 1e3,
            "plain_fwd_ms": t_fwd * 1e3, "adjoint_over_fwd": t_adj / t_fwd,
            "value": N * N * T / t_adj / 1e9, "unit": "Gcell-updates/s (forward steps differentiated)",
            "all_states": {"checkpoints": 1, "adjoint_ms": t_all * 1e3, "adjoint_over_fwd": t_all / t_fwd,
                           "workspace_bytes": int(all_bytes)},
            "every_state": {"checkpoints": T, "adjoint_ms": t_every * 1e3, "adjoint_over_fwd": t_every / t_fwd,
                            "workspace_bytes": int(every_bytes)},
            "tape": {"sqrt": tape_sqrt, "all": tape_all,
                     "note": "backward_ms: rdcnn_adjoint_tape after a recording forward (rdcnn_run_record) "
                             "of the same T; adjoint_ms above includes its own forward sweep"},
            "gradient_check": adjoint_gradient_check(rd, torch, N=N, T=T, quick=quick)}


def adjoint_gradient_check(rd, torch, N=512, T=2000, quick=False):
    """Accuracy of the adjoint's gradients on the adjoint workload (N x N, loss
    L = mean((u_T - target)^2), target the seeded +-1 checkerboard of period 32) for the FP32 and
    the FP64 kernels, against FP64 central differences of the FP64 forward kernels (which the
    parity tests hold to the oracle at 1e-12 normwise).  Both adjoints start from the same
    FP32-rounded x.

    Two horizons.  At T = 100 the forward map is smooth at the difference step, so dL/du0 and
    dL/dv0 are checked as directional derivatives along seeded U[-1, 1] directions (steps h and
    h / 10 show the quotient has converged) and the six gene entries one by one.  At the
    workload's T the gene entries are checked the same way; the state directions are not: by
    then a perturbation of 1e-5 per cell flips cells near the middle branch of the cubic and the
    difference quotient no longer approximates the derivative (it changes by orders of magnitude
    with the step), so the FP32 state gradient is reported as its normwise distance from the FP64
    adjoint's instead."""
    p = inp.default_params()
    x = torch.from_numpy(np.asarray(inp.uniform_field(0, N, N), dtype=np.float32).astype(np.float64)).cuda()
    tgt = torch.from_numpy(inp.checkerboard(0, N, N)).cuda()
    du = torch.from_numpy(inp.uniform_field(101, N, N)).cuda()
    dv = torch.from_numpy(inp.uniform_field(102, N, N)).cuda()
    g64 = rd.Grid(N, N, p, dtype=torch.float64)

    def loss(u0, v0, steps, params=None):
        if params is not None:
            g64.set_params(params)
        g64.set_state(u0.contiguous(), v0.contiguous()).run(steps)
        val = float(torch.mean((g64.u - tgt) ** 2))
        if params is not None:
            g64.set_params(p)
        return val

    def central(fn, h):
        return (fn(h) - fn(-h)) / (2.0 * h)

    def gene_fd(steps, h_rel=1e-5):
        out = []
        for name in rd.GRAD_NAMES:
            step = h_rel * max(abs(p[name]), 1e-3)

            def f(h, name=name):
                q = dict(p)
                q[name] = p[name] + h
                return loss(x, x, steps, q)
            out.append(central(f, step))
        return np.array(out)

    adjoint_ms = {}

    def adjoints(steps):
        res = {}
        for tag, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
            g = rd.Grid(N, N, p, dtype=dt)
            xs = x.to(dt)
            g.set_state(xs, xs).run(steps)
            gu = (2.0 * (g.u.double() - tgt) / g.u.numel()).to(dt).contiguous()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            du0, dv0, gp = g.adjoint(steps, xs, xs, gu, torch.zeros_like(gu))
            adjoint_ms[f"{tag}_T{steps}"] = (time.perf_counter() - t0) * 1e3  # first call: includes set-up
            res[tag] = (du0.double(), dv0.double(), np.array([gp[k] for k in rd.GRAD_NAMES]))
            g.close()
        return res

    def rel(a, b):
        return float(abs(a - b) / abs(b))

    out = {"grid": [N, N], "loss": "mean((u_T - target)^2), target +-1 checkerboard, period 32",
           "reference": "FP64 central differences of the FP64 forward kernels"}
    # short horizon: every gradient against differences
    Ts = 100
    h = 1e-6
    fd = {}
    for name, d in (("u0", du), ("v0", dv)):
        f = (lambda s, d=d: loss(x + s * d, x, Ts)) if name == "u0" else (lambda s, d=d: loss(x, x + s * d, Ts))
        fd[name] = (central(f, h), central(f, 10 * h))
    fdg = gene_fd(Ts)
    adj = adjoints(Ts)
    short = {"T": Ts, "h_state": h, "fd_converged": {k: rel(a, b) for k, (b, a) in fd.items()}}
    for tag, (a_u, a_v, a_g) in adj.items():
        short[tag] = {"dLdu0_dir_rel_err": rel(float(torch.sum(a_u * du)), fd["u0"][0]),
                      "dLdv0_dir_rel_err": rel(float(torch.sum(a_v * dv)), fd["v0"][0]),
                      "gene_rel_err": float(np.linalg.norm(a_g - fdg) / np.linalg.norm(fdg))}
    out["short_horizon"] = short
    if quick:
        out["adjoint_ms_first_call"] = adjoint_ms
        return out
    # the workload's horizon: gene entries against differences, state against the FP64 adjoint
    fdg = gene_fd(T)
    adj = adjoints(T)
    su, sv = adj["fp64"][0], adj["fp64"][1]
    full = {"T": T}
    for tag, (a_u, a_v, a_g) in adj.items():
        full[tag] = {"gene_rel_err": float(np.linalg.norm(a_g - fdg) / np.linalg.norm(fdg)),
                     "gene_entry_rel_err": {k: rel(a, b) for k, a, b in zip(rd.GRAD_NAMES, a_g, fdg)}}
    full["fp32"]["dLdu0_vs_fp64_adjoint"] = float(torch.linalg.norm(adj["fp32"][0] - su) / torch.linalg.norm(su))
    full["fp32"]["dLdv0_vs_fp64_adjoint"] = float(torch.linalg.norm(adj["fp32"][1] - sv) / torch.linalg.norm(sv))
    fu = lambda s: loss(x + s * du, x, T)  # noqa: E731
    full["state_fd_unresolved"] = {"h_1e-5": central(fu, 1e-5), "h_1e-4": central(fu, 1e-4),
                                   "adjoint_fp64": float(torch.sum(su * du))}
    out["workload_horizon"] = full
    out["adjoint_ms_first_call"] = adjoint_ms
    g64.close()
    return out


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2102_10340_gb300 import rdcnn as rd

    rd.launch_count()  # loads librdcnn.so or raises
    N, T = args.grid, args.T
    x_host = torch.from_numpy(np.asarray(inp.mid_patch(0, N, N), dtype=np.float32)).pin_memory()
    x_dev = x_host.to(dev)
    grid = rd.Grid(N, N, inp.default_params(), dtype=torch.float32, device=dev)
    from paper_2102_10340_gb300 import autotune

    if args.no_tune:
        tune = {"variant": args.variant, "k": args.k, "rows": args.rows}
    else:
        tune = autotune.tune_grid(grid, x_dev, trial_steps=max(8, T // 2000))
    grid.set_tune(k=tune["k"], rows=tune["rows"])
    variant = tune["variant"]
    plan = grid.plan(variant, tune["k"])  # rows = 0 resolves to the launcher's own choice

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def step():
        grid.init(x_dev, 1.0)
        grid.run(T, variant=variant, k=tune["k"])

    for _ in range(args.warmup):
        step()
    barrier()
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    sampler.start()
    l0 = rd.launch_count()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(args.steps):
        step()
    e.record()
    barrier()
    launches = rd.launch_count() - l0
    clocks = sampler.stop()
    ms = max_over_ranks(s.elapsed_time(e), world, dev)
    value = replica_throughput(N * N, T, args.steps, world, ms * 1e-3)

    # end to end through the C ABI with host buffers (pinned): H2D x, run, D2H (u, v)
    hu = torch.empty((N, N), dtype=torch.float32).pin_memory()
    hv = torch.empty((N, N), dtype=torch.float32).pin_memory()
    grid.init(x_host, 1.0).run(T, variant=variant, k=tune["k"])
    grid.get_state(hu, hv)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        grid.init(x_host, 1.0)
        grid.run(T, variant=variant, k=tune["k"])
        grid.get_state(hu, hv)
    t_e2e = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_value = replica_throughput(N * N, T, args.steps, world, t_e2e)
    finite = bool(torch.isfinite(torch.from_numpy(hu.numpy())).all())

    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank != 0:
        return 0

    peaks = load_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    # roofline of the dominant kernel (one launch advances k steps over the whole grid)
    fused = variant in ("temporal", "temporal2", "temporal_wide")
    k = tune["k"] if fused else 1
    # the dominant kernel is every launch of the timed region (99.8 % of the launch list), so
    # its average launch duration is the region's time over its launches; a short isolated
    # sample (2 launches per call, so each window also holds one launch's start-up) is kept
    # beside it
    launch_ms = ms / (args.steps * -(-T // k))
    launch_ms_isolated = measure_launch_ms(rd, grid, variant, k, 2, 20, torch)
    cells = N * N
    if fused and k > 1:
        flops = FLOPS_PER_CELL_STEP * cells * k
        # FP32 FMA peak: SMs x 128 lanes x 2 flop x max SM clock
        peak_tf = n_sm * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
        ach = flops / (launch_ms * 1e-3) / 1e12
        kname = {"temporal": "k_temporal", "temporal2": "k_temporal_split",
                 "temporal_wide": "k_temporal_wide"}[variant]
        traffic, tsrc = (profiled_traffic(f"{kname}_f32_k{k}_4096.md", k, plan["rows"]) if N == 4096
                         else (None, "other grid"))
        issue = None
        inst = profiled_instructions(f"{kname}_f32_k{k}_4096.md") if traffic is not None else None
        if inst:
            # warp-instruction issue: 4 schedulers per SM, one instruction per clock each
            peak_issue = n_sm * 4 * peaks["sm_max_mhz"] * 1e6
            issue = {"achieved": inst / (launch_ms * 1e-3), "peak": peak_issue, "unit": "warp-inst/s",
                     "frac": inst / (launch_ms * 1e-3) / peak_issue, "instructions_per_launch": inst,
                     "source": tsrc}
        roofline = {"bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s", "frac": ach / peak_tf,
                    "issue": issue,
                    "traffic": traffic, "traffic_source": tsrc,
                    "algorithmic_bytes": BYTES_PER_CELL_STEP * cells, "kernel": f"{kname}<float,K={k}>",
                    "peak_source": f"{n_sm} SM (device) x 128 FP32 lanes x 2 flop x sm_max_mhz "
                                   f"({peaks['sm_max_mhz']:.0f} MHz, {peaks['source']})",
                    "launch_ms": launch_ms, "launch_ms_source": "timed region / launches in it",
                    "launch_ms_isolated": launch_ms_isolated,
                    "hbm_equiv": {"achieved": BYTES_PER_CELL_STEP * cells / (launch_ms * 1e-3) / 1e9,
                                  "peak": peaks["hbm_gbs"], "unit": "GB/s"}}
    else:
        byts = BYTES_PER_CELL_STEP * cells
        ach = byts / (launch_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": None, "kernel": "k_step1<float>",
                    "peak_source": peaks["source"], "launch_ms": launch_ms,
                    "launch_ms_source": "timed region / launches in it", "launch_ms_isolated": launch_ms_isolated}
    # the unfused single-step kernel against the HBM roofline (16 B per cell-step)
    grid.set_tune(k=1, rows=0)  # the single-step kernel's own default strip length
    s1_ms = measure_launch_ms(rd, grid, "step1", 1, 20, 10, torch)  # 20 back-to-back launches per window
    s1_gbs = BYTES_PER_CELL_STEP * cells / (s1_ms * 1e-3) / 1e9
    step1 = {"kernel": "k_step1<float>", "launch_ms": s1_ms, "gcell_s": cells / (s1_ms * 1e-3) / 1e9,
             "achieved_gbs": s1_gbs, "peak_gbs": peaks["hbm_gbs"], "frac": s1_gbs / peaks["hbm_gbs"]}

    extra = {}
    if not args.no_extras:
        extra["image"] = measure_image(rd, torch, quick=args.quick)
        extra["snapshots"] = measure_snapshots(rd, grid, x_dev, torch, T=200 if args.quick else 2000,
                                               every=20 if args.quick else 200)
        extra["batched"] = measure_batched(rd, torch, quick=args.quick)
        extra["search"] = measure_search(torch, quick=args.quick)
        extra["adjoint"] = measure_adjoint(rd, torch, quick=args.quick)
        extra["models"] = measure_models(rd, torch, quick=args.quick)
        extra["storage"] = measure_storage(rd, torch, quick=args.quick)
    cpu = None if args.no_cpu else oracle_sample(6.0 if args.quick else 12.0, n=N)

    line = {"metric": METRIC, "value": value, "unit": "Gcell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": value / (PAPER_MCELLS_4096 / 1000.0), "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if (N, T) == (N_GRID, T_STEPS) else f"{N}x{N} FP32 patch, T={T}",
                       "grid": [N, N], "T": T, "variant": variant, "k": k, "rows": plan["rows"],
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "launch": "programmatic dependent launch" if os.environ.get("RDCNN_PDL", "1")[:1] != "0"
                                 else "plain launches (RDCNN_PDL=0)",
                       "l2": "inputs larger than L2: 4 x 64 MiB planes (state + ping-pong) vs 126 MiB L2",
                       "vs_baseline_ref": "Table I PyCUDA 14545 Mcell/s at N=4096, Tesla P100 (context)"},
            "e2e": {"value": e2e_value, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 4 * N * N,
                    "d2h_bytes_per_step": 2 * 4 * N * N, "finite": finite},
            "gpu_launches": int(launches), "clocks": clocks, "roofline": roofline,
            "single_step_kernel": step1, "cpu_baseline": cpu}
    line.update(extra)
    line["followon"] = followon_summary(line)  # last key: the compact ratios end the line
    print(json.dumps(line), flush=True)
    return 0


def followon_summary(line):
    """The headline's companion figures in a few hundred bytes: the single-step kernel against
    the HBM roofline, the batched sweep and the adjoint against plain forward runs, and the
    adjoint's gradient errors."""
    out = {"headline_gcell_s": line["value"], "roofline_frac": line["roofline"]["frac"],
           "single_step": {"gcell_s": line["single_step_kernel"]["gcell_s"],
                           "frac_hbm": line["single_step_kernel"]["frac"]}}
    b = line.get("batched")
    if b:
        out["batched"] = {"gcell_s": b["value"], "plain_fwd_gcell_s": b["plain_fwd_value"],
                          "vs_plain_fwd": b["vs_plain_fwd"]}
    a = line.get("adjoint")
    if a:
        out["adjoint"] = {"ms": a["adjoint_ms"], "plain_fwd_ms": a["plain_fwd_ms"],
                          "adjoint_over_fwd": a["adjoint_over_fwd"],
                          "all_states_over_fwd": a["all_states"]["adjoint_over_fwd"],
                          "every_state_over_fwd": a["every_state"]["adjoint_over_fwd"]}
        if "tape" in a:
            for key in ("sqrt", "all"):
                t = a["tape"][key]
                out["adjoint"][f"tape_{key}"] = {"record_over_fwd": t["record_over_fwd"],
                                                 "backward_over_fwd": t["backward_over_fwd"]}
        gc = a.get("gradient_check")
        if gc:
            sh, wl = gc["short_horizon"], gc.get("workload_horizon")
            for tag in ("fp32", "fp64"):
                e = {f"T{sh['T']}_{k}": sh[tag][k] for k in ("dLdu0_dir_rel_err", "dLdv0_dir_rel_err", "gene_rel_err")}
                if wl:
                    e[f"T{wl['T']}_gene_rel_err"] = wl[tag]["gene_rel_err"]
                    if tag == "fp32":
                        e[f"T{wl['T']}_dLdu0_vs_fp64"] = wl[tag]["dLdu0_vs_fp64_adjoint"]
                out["adjoint"][f"grad_err_{tag}"] = e
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--grid", type=int, default=N_GRID)
    ap.add_argument("--T", type=int, default=T_STEPS)
    ap.add_argument("--quick", action="store_true", help="small batched/adjoint/cpu legs")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and adjoint legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--no-tune", action="store_true",
                    help="use --variant/--k/--rows instead of autotuning (with --leg batched: --k/--rows)")
    ap.add_argument("--leg", choices=("batched", "batched_full", "adjoint", "search", "models", "storage", "image"),
                    default=None,
                    help="run only this follow-on measurement (small, for profiling) and print it; "
                         "batched_full: all 256 sweep instances for --T steps")
    ap.add_argument("--variant", default="temporal",
                    choices=("temporal", "temporal2", "temporal_wide", "step1", "generic"))
    ap.add_argument("--k", type=int, default=8)
    ap.add_argument("--rows", type=int, default=128)
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.leg:
        import torch

        from paper_2102_10340_gb300 import rdcnn as rd

        btune = {"k": args.k, "rows": args.rows} if args.no_tune else None
        fn = {"batched": lambda: measure_batched(rd, torch, quick=True, tune=btune),
              "batched_full": lambda: measure_batched(rd, torch, T=args.T, quick=True, tune=btune, full_sweep=True),
              "adjoint": lambda: measure_adjoint(rd, torch, quick=True),
              "search": lambda: measure_search(torch, quick=True),
              "models": lambda: measure_models(rd, torch),
              "storage": lambda: measure_storage(rd, torch),
              "image": lambda: measure_image(rd, torch)}[args.leg]
        print(json.dumps({"leg": args.leg, **fn()}), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
