"""Launch-shape autotuner: picks the temporal depth k and rows per warp strip.

Neither choice changes results (every variant computes identical bits); they
only trade halo recomputation and registers against DRAM traffic and
occupancy.  Candidates are timed with CUDA events on the current stream on
the caller's own buffers, and the winner is cached per problem signature.
"""
from __future__ import annotations

import torch

_cache: dict = {}

GRID_CANDIDATES_F32 = [("temporal", k, r) for k in (2, 3, 4, 5, 6, 8) for r in (0, 8, 16, 32, 64, 128, 256)] + \
                      [("temporal2", k, r) for k in (4, 6, 8) for r in (0, 64, 176, 256)] + \
                      [("temporal_wide", k, r) for k in (2, 3, 4) for r in (0, 32, 64, 128)] + \
                      [("step1", 1, r) for r in (4, 8, 16, 32)]
GRID_CANDIDATES_F64 = [("temporal", k, r) for k in (2, 3, 4) for r in (0, 32, 64, 128)] + \
                      [("temporal2", k, r) for k in (2, 4) for r in (0, 64)] + \
                      [("step1", 1, r) for r in (4, 8, 16)]
# 256-row strips won at the 256-instance sweep with four-warp blocks (k = 4: 1156 against 1130
# Gcell/s at 128 rows), 128-row strips with one-warp blocks (1298); 96 and 192 lie between
BATCH_CANDIDATES = [(k, r) for k in (2, 3, 4, 6, 8) for r in (16, 32, 64, 96, 128, 192, 256, 512)]


def _time(fn, reps: int = 2) -> float:
    fn()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e))
    return best


def tune_grid(grid, x=None, trial_steps: int = 48, force: bool = False) -> dict:
    """Best {variant, k, rows} for this grid's size and dtype (cached)."""
    key = ("grid", grid.nn, grid.nm, grid.dtype, grid.reaction, getattr(grid, "boundary", "periodic"))
    if key in _cache and not force:
        return dict(_cache[key])
    vec = 4 if grid.dtype == torch.float32 else 2
    if grid.nm % vec != 0:
        best = {"variant": "generic", "k": 1, "rows": 0, "ms_per_step": None}
        _cache[key] = best
        return dict(best)
    cands = GRID_CANDIDATES_F64 if grid.dtype == torch.float64 else GRID_CANDIDATES_F32
    if grid.dtype in (torch.bfloat16, torch.float16):
        cands = [c for c in cands if c[0] != "temporal2"]  # FP32 / FP64 planes only
    if grid.nm % 8 != 0:
        cands = [c for c in cands if c[0] != "temporal_wide"]  # 8 values per lane
    T = 240 * max(1, trial_steps // 48)  # divisible by every candidate depth
    best = None
    for variant, k, rows in cands:
        if x is not None:
            grid.init(x, 1.0)
        grid.set_tune(k=k, rows=rows)
        ms = _time(lambda: grid.run(T, variant=variant, k=k))
        if best is None or ms < best["ms_per_step"] * T:
            best = {"variant": variant, "k": k, "rows": rows, "ms_per_step": ms / T}
    grid.set_tune(k=best["k"], rows=best["rows"])
    _cache[key] = best
    return dict(best)


def tune_batch(batch, trial_steps: int = 48, force: bool = False) -> dict:
    """Best {k, rows} for a Batch (cached per instance-size signature)."""
    sig = tuple(sorted((it["nn"], it["nm"]) for it in batch.items))
    key = ("batch", sig, batch.dtype, batch.reaction, getattr(batch, "boundary", "periodic"))
    if key in _cache and not force:
        return dict(_cache[key])
    T = 24 * max(1, trial_steps // 24)
    maxk = 8 if batch.dtype == torch.float32 else 4
    best = None
    for k, rows in BATCH_CANDIDATES:
        if k > maxk:
            continue
        batch.set_tune(k=k, rows=rows)
        ms = _time(lambda: batch.run(T))
        if best is None or ms < best[2]:
            best = (k, rows, ms)
    out = {"k": best[0], "rows": best[1]}
    batch.set_tune(**out)
    _cache[key] = out
    return dict(out)
