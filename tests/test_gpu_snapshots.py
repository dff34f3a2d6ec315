"""rdcnn_run_snapshots: the paper's A_show / B_show capture (every test_mod steps,
slot 0 = initial state) against separate runs (bit-identical: same kernels) and
against the FP64 oracle."""
import numpy as np
import pytest
import torch

import rdcnn_inputs as inp
from _util import f32, gpu_run, normwise

pytestmark = pytest.mark.gpu

F32, F64 = torch.float32, torch.float64


def _grid(rd, x, dtype, params=None):
    g = rd.Grid(x.shape[0], x.shape[1], params or inp.default_params(), dtype=dtype)
    g.set_state(torch.from_numpy(x).to("cuda", dtype), torch.from_numpy(x).to("cuda", dtype))
    return g


@pytest.mark.parametrize("out,n_stage,pin", [("device", 0, True), ("host", 1, True), ("host", 3, True),
                                             ("host", 2, False)])
@pytest.mark.parametrize("T,every", [(50, 7), (21, 1), (30, 30), (40, 100), (0, 5)])
def test_snapshots_equal_separate_runs(rd, out, n_stage, pin, T, every):
    x = f32(inp.uniform_field(4, 96, 128))
    g = _grid(rd, x, F32)
    us, vs = g.run_snapshots(T, every, out=out, n_stage=max(n_stage, 1), pin=pin)
    torch.cuda.synchronize()
    n = T // every + 1
    assert us.shape == (n, 96, 128) and vs.shape == (n, 96, 128)
    for s in range(n):
        ru, rv = gpu_run(rd, x, x, inp.default_params(), s * every, F32, "auto")
        assert np.array_equal(us[s].double().cpu().numpy(), ru), (s, out)
        assert np.array_equal(vs[s].double().cpu().numpy(), rv), (s, out)
    fu, fv = gpu_run(rd, x, x, inp.default_params(), T, F32, "auto")
    assert np.array_equal(g.u.double().cpu().numpy(), fu) and np.array_equal(g.v.double().cpu().numpy(), fv)


def test_snapshots_f64_vs_oracle(rd, oracle_mod):
    x = inp.uniform_field(6, 40, 64)
    g = _grid(rd, x, F64)
    us, vs = g.run_snapshots(60, 15, out="host")
    for s in range(5):
        ou, ov = oracle_mod.run(x, x, inp.default_params(), 15 * s)
        assert normwise(us[s].numpy(), ou) <= 1e-12 and normwise(vs[s].numpy(), ov) <= 1e-12


def test_snapshots_full_size_host(rd):
    """4096^2 slow-growth grid, 5 snapshots to pinned host memory through 2 staging slots."""
    N = 4096
    x = f32(inp.mid_patch(0, N, N))
    g = _grid(rd, x, F32)
    us, vs = g.run_snapshots(400, 100, out="host", n_stage=2)
    assert us.shape == (5, N, N)
    assert np.array_equal(us[0].numpy(), x.astype(np.float32))
    assert torch.equal(us[-1], g.u.cpu()) and torch.equal(vs[-1], g.v.cpu())
    mid_u, _ = gpu_run(rd, x, x, inp.default_params(), 200, F32, "auto")
    assert np.array_equal(us[2].double().numpy(), mid_u)


def test_snapshots_into_caller_buffers(rd):
    x = f32(inp.uniform_field(8, 32, 64))
    g = _grid(rd, x, F32)
    bu = torch.empty((4, 32, 64), dtype=F32).pin_memory()
    bv = torch.empty((4, 32, 64), dtype=F32).pin_memory()
    us, vs = g.run_snapshots(30, 10, out="host", buffers=(bu, bv))
    assert us.data_ptr() == bu.data_ptr() and vs.data_ptr() == bv.data_ptr()
    ru, rv = gpu_run(rd, x, x, inp.default_params(), 20, F32, "auto")
    assert np.array_equal(bu[2].double().numpy(), ru) and np.array_equal(bv[2].double().numpy(), rv)
    with pytest.raises(ValueError):
        g.run_snapshots(30, 10, out="host", buffers=(bu[:3], bv[:3]))


def test_snapshot_argument_errors(rd):
    x = f32(inp.uniform_field(1, 8, 8))
    g = _grid(rd, x, F32)
    with pytest.raises(rd.RDCNNError):
        g.run_snapshots(10, 0)
    from paper_2102_10340_gb300 import _lib as L

    hu = torch.empty((3, 8, 8), dtype=F32)
    rc = g.lib.rdcnn_run_snapshots(g.h, 10, 5, hu.data_ptr(), hu.data_ptr(), 0, None, 0)
    assert rc == L.ESPACE


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32], ids=["bf16", "f32"])
def test_snapshots_of_model_variants(rd, dtype):
    """A zero-flux CeNN grid (16-bit or FP32 planes): the captures equal separate runs.  Launches
    end at multiples of `every`, so with `every` a multiple of the depth the 16-bit rounding
    schedule is the plain run's too."""
    gene = {"dt": 0.1, "a": 0.0, "b": 0.0, "eps": 0.0, "c": 1.2, "Du": 0.1, "Dv": 0.0}
    x = (1.5 * inp.uniform_field(8, 96, 128)).astype(np.float32)
    w = (0.3 * inp.uniform_field(9, 96, 128)).astype(np.float32)
    g = rd.Grid(96, 128, gene, dtype=dtype, reaction="cenn", boundary="zeroflux")
    g.set_state(torch.from_numpy(x).to("cuda", dtype), torch.from_numpy(w).to("cuda", dtype))
    us, vs = g.run_snapshots(48, 8, out="host", n_stage=2)
    for s in range(7):
        ru, rv = gpu_run(rd, torch.from_numpy(x).to(dtype).double().numpy(),
                         torch.from_numpy(w).to(dtype).double().numpy(), gene, 8 * s, dtype, "auto",
                         reaction="cenn", boundary="zeroflux")
        assert np.array_equal(us[s].double().numpy(), ru) and np.array_equal(vs[s].double().numpy(), rv), s
