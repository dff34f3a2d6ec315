"""16-bit state storage (bf16 / IEEE half planes, FP32 arithmetic) against the
oracle's storage reference, through the C ABI.

The storage variant is a different discrete map from the FP32 one: the state
is rounded to the 16-bit format at the end of every launch (every k steps of
the temporal kernel, every step of the single-step and generic kernels), so
results depend on k, and the oracle reference (oracle.run_storage) applies the
same rounding schedule to FP32 steps in the paper's literal order.  The two
round the same FP32 values except where the kernels' fused evaluation differs
from the literal one by an FP32 rounding near a 16-bit rounding boundary, so
a few cells in ten thousand differ by one 16-bit unit.  Bars (measured on
GB300 far below them): on grids under 1024 cells every cell within 8 units
of the 16-bit format of the reference (one unit dominates a norm there);
otherwise normwise distance to the storage reference <= 5e-4,
and <= 0.1 x the storage error itself (the reference's distance to the FP64
model), so the kernels demonstrably implement the rounded map; at most 1e-3
of the cells differ.  Variants with the same rounding schedule (k = 1:
generic, single-step at either lane width, temporal k = 1) agree bit for bit.
"""
import numpy as np
import pytest
import torch

import rdcnn_inputs as inp
from _util import gpu_run, normwise

pytestmark = pytest.mark.gpu

STORAGE = [("bf16", torch.bfloat16), ("f16", torch.float16)]


def storage_ulp(x, storage):
    """Spacing of the 16-bit format at |x| (normal range; the smallest normal's below it)."""
    bits = 7 if storage == "bf16" else 10
    emin = -126 if storage == "bf16" else -14
    e = np.floor(np.log2(np.maximum(np.abs(x), 2.0 ** emin)))
    return 2.0 ** (e - bits)


def _close(gu, gv, su, sv, storage, what):
    """Tiny grids (< 1024 cells): one one-unit rounding difference dominates a norm, so every
    cell must be within 8 units of the format; larger grids: normwise <= 5e-4 (there a rare
    difference may grow locally through the dynamics while the norm stays small)."""
    if gu.size < 1024:
        assert np.all(np.abs(gu - su) <= 8 * storage_ulp(su, storage)), what
        assert np.all(np.abs(gv - sv) <= 8 * storage_ulp(sv, storage)), what
    else:
        assert normwise(gu, su) <= 5e-4 and normwise(gv, sv) <= 5e-4, what


def _check(gu, gv, su, sv, fu, fv):
    eu, ev = normwise(gu, su), normwise(gv, sv)
    assert eu <= 5e-4 and ev <= 5e-4, (eu, ev)
    ref_err = max(normwise(su, fu), normwise(sv, fv))
    assert max(eu, ev) <= 0.1 * ref_err, (eu, ev, ref_err)
    assert np.count_nonzero(gu != su) <= 1e-3 * gu.size


@pytest.mark.parametrize("storage,dt", STORAGE, ids=[s for s, _ in STORAGE])
@pytest.mark.parametrize("k", [1, 4, 8])
def test_storage_matches_rounded_reference(rd, oracle_mod, storage, dt, k):
    """64 x 64, default gene, x ~ U[-1, 1] seed 0 (rounded to the format), u = v = x, T = 200."""
    x = oracle_mod.round_to_storage(inp.uniform_field(0, 64, 64), storage).astype(np.float64)
    T = 200
    gu, gv = gpu_run(rd, x, x, inp.default_params(), T, dt, "step1" if k == 1 else "temporal", k)
    su, sv = oracle_mod.run_storage(x, x, inp.default_params(), T, k, storage)
    fu, fv = oracle_mod.run(x, x, inp.default_params(), T)
    _check(gu, gv, su, sv, fu, fv)


SHAPES = [(1, 4), (3, 8), (5, 12), (7, 20), (37, 56), (65, 244), (129, 264)]


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a}x{b}" for a, b in SHAPES])
@pytest.mark.parametrize("storage,dt", STORAGE, ids=[s for s, _ in STORAGE])
def test_storage_variants_and_ragged_grids(rd, oracle_mod, shape, storage, dt):
    nn, nm = shape
    x = oracle_mod.round_to_storage(inp.uniform_field(90, nn, nm), storage).astype(np.float64)
    y = oracle_mod.round_to_storage(0.5 * inp.uniform_field(91, nn, nm), storage).astype(np.float64)
    T = 40
    su, sv = oracle_mod.run_storage(x, y, inp.default_params(), T, 1, storage)
    first = None
    for variant, k in (("generic", 0), ("step1", 0), ("temporal", 1)):
        gu, gv = gpu_run(rd, x, y, inp.default_params(), T, dt, variant, k)
        _close(gu, gv, su, sv, storage, variant)
        if first is None:
            first = (gu, gv)
        else:  # same rounding schedule (every step): identical bits
            assert np.array_equal(gu, first[0]) and np.array_equal(gv, first[1]), variant
    # a deeper launch rounds less often: its own reference
    s3u, s3v = oracle_mod.run_storage(x, y, inp.default_params(), T, 3, storage)
    gu, gv = gpu_run(rd, x, y, inp.default_params(), T, dt, "temporal", 3)
    _close(gu, gv, s3u, s3v, storage, "temporal k=3")


@pytest.mark.parametrize("storage,dt", STORAGE, ids=[s for s, _ in STORAGE])
def test_storage_models_zero_flux_and_cenn(rd, oracle_mod, storage, dt):
    x = oracle_mod.round_to_storage(1.5 * inp.uniform_field(92, 40, 72), storage).astype(np.float64)
    w = oracle_mod.round_to_storage(0.3 * inp.uniform_field(93, 40, 72), storage).astype(np.float64)
    gene = {"dt": 0.1, "a": 0.0, "b": 0.0, "eps": 0.0, "c": 1.2, "Du": 0.1, "Dv": 0.0}
    su, sv = oracle_mod.run_storage(x, w, gene, 30, 5, storage, reaction=oracle_mod.CENN,
                                    boundary=oracle_mod.ZEROFLUX)
    gu, gv = gpu_run(rd, x, w, gene, 30, dt, "temporal", 5, reaction="cenn", boundary="zeroflux")
    assert normwise(gu, su) <= 5e-4 and np.array_equal(gv, w)


@pytest.mark.parametrize("storage,dt", STORAGE, ids=[s for s, _ in STORAGE])
def test_storage_full_size_windows(rd, oracle_mod, storage, dt):
    """4096 x 4096 in 16-bit storage, the single-step variant (the depth-1 ring pipeline with
    16-row strips, as in the storage leg of the benchmark), T = 16.  Rounding is per cell, so the light-cone argument holds for the rounded
    map: a 64 x 64 window run alone (wrapping) fixes its cells farther than T from its sides."""
    N, W, T = 4096, 64, 16
    x = oracle_mod.round_to_storage(inp.uniform_field(94, N, N), storage).astype(np.float64)
    gu, gv = gpu_run(rd, x, x, inp.default_params(), T, dt, "step1", 0)
    for r0, c0 in ((0, 0), (N // 2 - 7, 1000), (N - W, N - W)):
        win = (slice(r0, r0 + W), slice(c0, c0 + W))
        su, sv = oracle_mod.run_storage(x[win], x[win], inp.default_params(), T, 1, storage)
        core = (slice(T, W - T), slice(T, W - T))
        assert normwise(gu[win][core], su[core]) <= 5e-4 and normwise(gv[win][core], sv[core]) <= 5e-4


@pytest.mark.parametrize("storage,dt", STORAGE, ids=[s for s, _ in STORAGE])
def test_storage_wide_lanes_same_bits(rd, oracle_mod, storage, dt):
    """8 values per lane (RDCNN_VARIANT_TEMPORAL_WIDE) against 4 at the same depth: same bits."""
    x = oracle_mod.round_to_storage(inp.uniform_field(95, 70, 264), storage).astype(np.float64)
    for k in (1, 3, 4):
        a = gpu_run(rd, x, x, inp.default_params(), 2 * k + 1, dt, "temporal", k)
        b = gpu_run(rd, x, x, inp.default_params(), 2 * k + 1, dt, "temporal_wide", k)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), k
    su, sv = oracle_mod.run_storage(x, x, inp.default_params(), 9, 4, storage)
    _close(b[0], b[1], su, sv, storage, "wide k=4")
