"""GPU forward path of the model variants (zero-flux boundary, Chua-Yang CeNN
cell) against the FP64 oracle, through the C ABI.

The zero-flux temporal kernel loads mirrored halos instead of testing for the
edge at every stage; the single-step and generic kernels clamp neighbour
indices.  The two designs must give the same bits, and both must match the
oracle (which pins zero flux to the mirrored torus and the CeNN cell to
closed forms).  Tolerances as in test_gpu_forward: normwise relative 1e-12
(FP64) and 1e-5 (FP32).
"""
import numpy as np
import pytest
import torch

import rdcnn_inputs as inp
from _util import f32, gpu_run, normwise

pytestmark = pytest.mark.gpu

F32, F64 = torch.float32, torch.float64
TOL = {F32: 1e-5, F64: 1e-12}

# Chua-Yang gene: feedback centre c, arms Du (moderate linear growth, so that FP32
# rounding is not amplified past the tolerance within the test horizons).
CENN_GENE = {"dt": 0.1, "a": 0.0, "b": 0.0, "eps": 0.0, "c": 1.2, "Du": 0.1, "Dv": 0.0}

MODELS = [("fhn", "zeroflux"), ("none", "zeroflux"), ("cenn", "periodic"), ("cenn", "zeroflux")]


def _gene(reaction):
    return CENN_GENE if reaction == "cenn" else inp.default_params()


def _inputs(reaction, nn, nm, seed):
    x = inp.uniform_field(seed, nn, nm)
    y = inp.uniform_field(seed + 1, nn, nm)
    if reaction == "cenn":
        return 1.5 * x, 0.3 * y  # state spans both saturated arms; small offset plane
    return x, y


def _variants(nm, dtype):
    vec = 4 if dtype == F32 else 2
    out = [("generic", 0)]
    if nm % vec == 0:
        out += [("step1", 0)] + [("temporal", k) for k in ((1, 2, 3, 5, 8) if dtype == F32 else (1, 2, 3, 4))]
        out += [("temporal2", k) for k in ((2, 5, 8) if dtype == F32 else (2, 4))]
    if dtype == F32 and nm % 8 == 0:
        out += [("temporal_wide", 2), ("temporal_wide", 4)]
    return out


def _oracle(oracle_mod, reaction, boundary, x, y, T):
    rx = {"fhn": oracle_mod.FHN, "none": oracle_mod.NONE, "cenn": oracle_mod.CENN}[reaction]
    bc = oracle_mod.ZEROFLUX if boundary == "zeroflux" else oracle_mod.PERIODIC
    return oracle_mod.run(x, y, _gene(reaction), T, reaction=rx, boundary=bc)


SHAPES = [(1, 1), (1, 4), (2, 2), (3, 8), (4, 5), (7, 20), (37, 53), (33, 64), (65, 244), (129, 260), (300, 8)]


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a}x{b}" for a, b in SHAPES])
@pytest.mark.parametrize("model", MODELS, ids=[f"{r}-{b}" for r, b in MODELS])
@pytest.mark.parametrize("dtype", [F64, F32], ids=["f64", "f32"])
def test_models_ragged_grids(rd, oracle_mod, shape, model, dtype):
    reaction, boundary = model
    nn, nm = shape
    x, y = _inputs(reaction, nn, nm, 40)
    if dtype == F32:
        x, y = f32(x), f32(y)
    T = 29
    ref_u, ref_v = _oracle(oracle_mod, reaction, boundary, x, y, T)
    first = None
    for variant, k in _variants(nm, dtype):
        u, v = gpu_run(rd, x, y, _gene(reaction), T, dtype, variant, k, reaction=reaction, boundary=boundary)
        assert normwise(u, ref_u) <= TOL[dtype] and normwise(v, ref_v) <= TOL[dtype], (variant, k)
        if first is None:
            first = (u, v)
        else:  # clamped indices and mirrored halos give identical bits
            assert np.array_equal(u, first[0]) and np.array_equal(v, first[1]), (variant, k)
    if reaction == "cenn":
        assert np.array_equal(first[1], y)  # the offset plane never changes


@pytest.mark.parametrize("model", MODELS, ids=[f"{r}-{b}" for r, b in MODELS])
def test_models_several_tiles_and_launches(rd, oracle_mod, model):
    """A grid spanning many warp bands and strips, T not a multiple of k (ragged last launch)."""
    reaction, boundary = model
    x, y = _inputs(reaction, 203, 516, 50)
    x, y = f32(x), f32(y)
    T = 61
    ref_u, ref_v = _oracle(oracle_mod, reaction, boundary, x, y, T)
    for variant, k in (("temporal", 8), ("temporal", 6), ("step1", 0), ("temporal2", 8), ("temporal2", 3)):
        u, v = gpu_run(rd, x, y, _gene(reaction), T, F32, variant, k, reaction=reaction, boundary=boundary,
                       rows=16)
        assert normwise(u, ref_u) <= TOL[F32] and normwise(v, ref_v) <= TOL[F32], (variant, k)


@pytest.mark.parametrize("reaction", ["fhn", "cenn"])
def test_zero_flux_corners_at_full_size(rd, oracle_mod, reaction):
    """4096 x 4096 zero-flux grid in the benchmark's launch shape (k = 8, 128 rows).  After T
    steps a cell depends only on cells within T of it, so each W x W corner window, run by the
    oracle with its own zero-flux edges, fixes every cell farther than T from the window's
    inner sides: the grid's true edges are the window's edges there."""
    N, W, T = 4096, 72, 24
    x, y = _inputs(reaction, N, N, 60)
    x, y = f32(x), f32(y)
    u, v = gpu_run(rd, x, y, _gene(reaction), T, F32, "temporal", 8, reaction=reaction, boundary="zeroflux",
                   rows=128)
    keep = W - T
    for ri in (slice(0, W), slice(N - W, N)):
        for ci in (slice(0, W), slice(N - W, N)):
            ref_u, ref_v = _oracle(oracle_mod, reaction, "zeroflux", x[ri, ci], y[ri, ci], T)
            r = slice(0, keep) if ri.start == 0 else slice(W - keep, W)
            c = slice(0, keep) if ci.start == 0 else slice(W - keep, W)
            gu = u[ri, ci][r, c]
            gv = v[ri, ci][r, c]
            assert normwise(gu, ref_u[r, c]) <= TOL[F32] and normwise(gv, ref_v[r, c]) <= TOL[F32]


def test_temporal2_rejects_16bit_planes(rd):
    x = torch.zeros((16, 16), device="cuda", dtype=torch.bfloat16)
    g = rd.Grid(16, 16, None, dtype=torch.bfloat16, boundary="zeroflux")
    g.set_state(x, x)
    with pytest.raises(rd.RDCNNError):
        g.run(8, variant="temporal2", k=4)
    g.close()


def test_plan_reports_the_launch_shape_that_runs(rd):
    """rdcnn_plan resolves AUTO, the default depth and the launcher's own rows choice; pinning
    the reported rows explicitly must run the same launches (same bits)."""
    g = rd.Grid(1024, 1024, None, dtype=F32)
    plan = g.plan("auto")
    assert plan["variant"] == "temporal" and 1 <= plan["k"] <= 8 and plan["rows"] >= 1
    assert g.plan("step1") == {"variant": "step1", "k": 1, "rows": 2}  # FP32: 2-row strips
    x = torch.from_numpy(f32(inp.uniform_field(70, 1024, 1024))).cuda().float()
    g.set_state(x, -x)
    g.run(3 * plan["k"] + 1)
    a = [t.clone() for t in g.state()]
    g.set_tune(k=plan["k"], rows=plan["rows"])
    assert g.plan("auto") == plan
    g.set_state(x, -x)
    g.run(3 * plan["k"] + 1)
    b = g.state()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    g.close()
