"""On-device search statistics (rdcnn_batch_summary) against the oracle's plain
definitions, on evolved states of a mixed-size batch."""
import numpy as np
import pytest
import torch

import rdcnn_inputs as inp
from _util import f32

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_batch_summary_matches_definitions(rd, oracle_mod, dtype):
    specs = [{"nn": 64, "nm": 64, "params": inp.default_params(Du=0.3, Dv=1.0)},
             {"nn": 37, "nm": 132, "params": inp.default_params(Du=0.5, Dv=0.8)},
             {"nn": 256, "nm": 256, "params": inp.default_params(Du=0.7, Dv=0.8)},
             {"nn": 1, "nm": 8, "params": inp.default_params()}]
    b = rd.Batch(specs, dtype=dtype)
    for i, s in enumerate(specs):
        x = inp.mid_patch(i, s["nn"], s["nm"], patch=min(16, s["nn"])) if s["nn"] > 1 else inp.uniform_field(i, 1, 8)
        if dtype == torch.float32:
            x = f32(x)
        b.set_state(i, torch.from_numpy(x), torch.from_numpy(0.5 * x))
    b.run(60)
    thr = 0.02
    got = b.summary(thr).numpy()
    prec = np.float32 if dtype == torch.float32 else np.float64
    for i in range(len(specs)):
        u, v = (t.cpu().numpy() for t in b.state(i))
        ref = oracle_mod.summary(u, v, thr, precision=prec)
        tol = 1e-5 if dtype == torch.float32 else 1e-12
        np.testing.assert_allclose(got[i][[0, 4, 6]], ref[[0, 4, 6]], rtol=tol, atol=tol)
        np.testing.assert_allclose(got[i][[1, 5]], ref[[1, 5]], rtol=1e-4 if dtype == torch.float32 else 1e-10,
                                   atol=1e-7 if dtype == torch.float32 else 1e-14)
        assert got[i][2] == ref[2] and got[i][3] == ref[3]
        assert got[i][7] == ref[7]  # the threshold test is taken in the state's precision on both sides


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16], ids=["bf16", "f16"])
def test_batch_summary_16bit_planes(rd, oracle_mod, dtype):
    """16-bit planes are read into FP32: the statistics equal the FP32 definitions on the
    planes' values."""
    specs = [{"nn": 64, "nm": 64, "params": inp.default_params(Du=0.3, Dv=1.0)},
             {"nn": 37, "nm": 132, "params": inp.default_params(Du=0.5, Dv=0.8)}]
    b = rd.Batch(specs, dtype=dtype)
    for i, s in enumerate(specs):
        x = inp.mid_patch(i, s["nn"], s["nm"], patch=16)
        b.set_state(i, torch.from_numpy(x), torch.from_numpy(0.5 * x))
    b.set_tune(k=4)
    b.run(40)
    thr = 0.02
    got = b.summary(thr).numpy()
    for i in range(len(specs)):
        u, v = (t.float().cpu().numpy() for t in b.state(i))
        ref = oracle_mod.summary(u, v, thr, precision=np.float32)
        np.testing.assert_allclose(got[i][[0, 4, 6]], ref[[0, 4, 6]], rtol=1e-5, atol=1e-5)
        np.testing.assert_allclose(got[i][[1, 5]], ref[[1, 5]], rtol=1e-4, atol=1e-7)
        assert got[i][2] == ref[2] and got[i][3] == ref[3]
        assert got[i][7] == ref[7]


def test_grid_summary_full_size(rd, oracle_mod):
    N = 4096
    x = f32(inp.smooth_noise(0, N, N))
    u = torch.from_numpy(x).float().cuda()
    v = (0.25 * u).contiguous()
    got = rd.grid_summary(u, v, 0.01).numpy()
    ref = oracle_mod.summary(x, 0.25 * x.astype(np.float32), 0.01, precision=np.float32)
    np.testing.assert_allclose(got[[0, 4, 6]], ref[[0, 4, 6]], rtol=1e-5, atol=1e-6)
    assert got[7] == ref[7] and got[2] == ref[2] and got[3] == ref[3]


def test_search_sweep_statistics_match_single_runs(rd, oracle_mod):
    """The sweep's checkpoint statistics equal the summary of the same gene run alone,
    and the run covers the three (Du, Dv) points Sec. III.A names."""
    from paper_2102_10340_gb300 import search

    genes = search.du_dv_grid([0.3, 0.5, 0.7], [0.8, 1.0])
    res = search.sweep(genes, N=128, T=300, checkpoints=3)
    assert res["stats"].shape == (6, 4, 8) and len(res["labels"]) == 6
    x = f32(inp.mid_patch(0, 128, 128))
    for i in (0, 3):
        g = rd.Grid(128, 128, genes[i], dtype=torch.float32)
        g.set_state(torch.from_numpy(x).cuda(), torch.from_numpy(x).cuda()).run(300)
        single = rd.grid_summary(g.u, g.v, 0.05).numpy()
        np.testing.assert_array_equal(res["stats"][i, -1], single)
        ref = oracle_mod.summary(g.u.cpu().numpy(), g.v.cpu().numpy(), 0.05, precision=np.float32)
        assert single[7] == ref[7]
