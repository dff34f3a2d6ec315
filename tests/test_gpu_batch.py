"""Batched sweep (one launch per k steps for all instances) vs the oracle and
vs single-grid runs of the same instances (bit-identical: same cell arithmetic)."""
import numpy as np
import pytest
import torch

import rdcnn_inputs as inp
from _util import cpu_threads, f32, gpu_run, normwise

pytestmark = pytest.mark.gpu

F32, F64 = torch.float32, torch.float64


def _two_per_size(seed=0):
    picked, seen = [], {}
    for spec in inp.sweep_instances(seed):
        if seen.get(spec["nn"], 0) < 2:
            seen[spec["nn"]] = seen.get(spec["nn"], 0) + 1
            picked.append(spec)
    return sorted(picked, key=lambda s: s["nn"])


def _load(batch, specs, dtype):
    xs = []
    for i, s in enumerate(specs):
        x = inp.uniform_field(s["x_seed"], s["nn"], s["nm"])
        if dtype == F32:
            x = f32(x)
        batch.set_state(i, torch.from_numpy(x), torch.from_numpy(x))
        xs.append(x)
    return xs


def test_sweep_eight_instances_vs_oracle(rd, oracle_mod):
    """Two instances of each size {128, 256, 512, 1024} from the seeded sweep, T = 500."""
    specs = _two_per_size()
    assert sorted(s["nn"] for s in specs) == [128, 128, 256, 256, 512, 512, 1024, 1024]
    b = rd.Batch(specs, dtype=F32)
    xs = _load(b, specs, F32)
    b.run(500)
    torch.cuda.synchronize()
    for i, s in enumerate(specs):
        ref_u, ref_v = oracle_mod.run(xs[i], xs[i], s["params"], 500, nthreads=cpu_threads())
        u, v = (t.double().cpu().numpy() for t in b.state(i))
        assert normwise(u, ref_u) <= 1e-5 and normwise(v, ref_v) <= 1e-5, (i, s["nn"])


@pytest.mark.parametrize("T,k", [(37, 4), (1, 4), (9, 1), (16, 8), (5, 6), (100, 3)])
def test_batch_bitwise_equals_single_grid_runs(rd, T, k):
    specs = [{"nn": 37, "nm": 64, "params": inp.default_params(Du=0.2, Dv=0.1)},
             {"nn": 5, "nm": 8, "params": inp.default_params(a=0.1)},
             {"nn": 128, "nm": 132, "params": inp.default_params(c=0.8, eps=-0.12)},
             {"nn": 200, "nm": 256, "params": inp.default_params()}]
    for i, s in enumerate(specs):
        s["x_seed"] = 50 + i
    b = rd.Batch(specs, dtype=F32)
    b.set_tune(k=k)
    xs = _load(b, specs, F32)
    b.run(T)
    torch.cuda.synchronize()
    for i, s in enumerate(specs):
        ref = gpu_run(rd, xs[i], xs[i], s["params"], T, F32, "generic")
        u, v = (t.double().cpu().numpy() for t in b.state(i))
        assert np.array_equal(u, ref[0]) and np.array_equal(v, ref[1]), (i, T, k)


def test_batch_f64_vs_oracle(rd, oracle_mod):
    specs = [{"nn": n, "nm": m, "params": inp.default_params(Du=du), "x_seed": 70 + n}
             for n, m, du in ((16, 16, 0.05), (40, 24, 0.2), (9, 130, 0.11))]
    b = rd.Batch(specs, dtype=F64)
    b.set_tune(k=3, rows=8)
    xs = _load(b, specs, F64)
    b.run(41)
    torch.cuda.synchronize()
    for i, s in enumerate(specs):
        ref_u, ref_v = oracle_mod.run(xs[i], xs[i], s["params"], 41)
        u, v = (t.cpu().numpy() for t in b.state(i))
        assert normwise(u, ref_u) <= 1e-12 and normwise(v, ref_v) <= 1e-12


def test_batch_rejects_bad_instance(rd):
    with pytest.raises(rd.RDCNNError):
        b = rd.Batch([{"nn": 8, "nm": 6}], dtype=F32)
        b.run(3)


# Chua-Yang gene with moderate linear growth (as in test_gpu_models).
CENN_GENE = {"dt": 0.1, "a": 0.0, "b": 0.0, "eps": 0.0, "c": 1.2, "Du": 0.1, "Dv": 0.0}
MODELS = [("fhn", "zeroflux"), ("none", "zeroflux"), ("cenn", "periodic"), ("cenn", "zeroflux")]


@pytest.mark.parametrize("k", [1, 3, 4, 8])
@pytest.mark.parametrize("model", MODELS, ids=[f"{r}-{b}" for r, b in MODELS])
def test_batch_models_vs_oracle_and_single_grid(rd, oracle_mod, model, k):
    """Zero-flux boundary and the CeNN cell in the batched sweep: the oracle within 1e-5
    and the same bits as a single-grid run of each instance (T = 23, ragged last launch)."""
    reaction, boundary = model
    shapes = [(37, 64), (5, 8), (128, 132), (1, 4), (66, 260)]
    specs = []
    for i, (nn, nm) in enumerate(shapes):
        gene = dict(CENN_GENE, Du=0.05 + 0.02 * i) if reaction == "cenn" else inp.default_params(Du=0.1 + 0.05 * i)
        specs.append({"nn": nn, "nm": nm, "params": gene})
    b = rd.Batch(specs, dtype=F32, reaction=reaction, boundary=boundary)
    b.set_tune(k=k)
    starts = []
    for i, s in enumerate(specs):
        x = inp.uniform_field(90 + i, s["nn"], s["nm"])
        y = inp.uniform_field(190 + i, s["nn"], s["nm"])
        u0, v0 = (f32(1.5 * x), f32(0.3 * y)) if reaction == "cenn" else (f32(x), f32(y))
        b.set_state(i, torch.from_numpy(u0), torch.from_numpy(v0))
        starts.append((u0, v0))
    T = 23
    b.run(T)
    torch.cuda.synchronize()
    rx = {"fhn": oracle_mod.FHN, "none": oracle_mod.NONE, "cenn": oracle_mod.CENN}[reaction]
    bc = oracle_mod.ZEROFLUX if boundary == "zeroflux" else oracle_mod.PERIODIC
    for i, s in enumerate(specs):
        u0, v0 = starts[i]
        u, v = (t.double().cpu().numpy() for t in b.state(i))
        ref_u, ref_v = oracle_mod.run(u0, v0, s["params"], T, reaction=rx, boundary=bc)
        assert normwise(u, ref_u) <= 1e-5 and normwise(v, ref_v) <= 1e-5, (i, s["nn"], s["nm"])
        one = gpu_run(rd, u0, v0, s["params"], T, F32, "generic", reaction=reaction, boundary=boundary)
        assert np.array_equal(u, one[0]) and np.array_equal(v, one[1]), (i, s["nn"], s["nm"])
        if reaction == "cenn":
            assert np.array_equal(v, v0)


@pytest.mark.parametrize("model", MODELS, ids=[f"{r}-{b}" for r, b in MODELS])
def test_batch_f64_models_vs_oracle(rd, oracle_mod, model):
    """The FP64 batched sweep with every model: the oracle within 1e-12 and the bits of
    single-grid FP64 runs."""
    reaction, boundary = model
    shapes = [(24, 40), (9, 6), (1, 2), (33, 130)]
    specs = [{"nn": a, "nm": b, "params": dict(CENN_GENE, Du=0.05 + 0.01 * i) if reaction == "cenn"
              else inp.default_params(Du=0.1 + 0.03 * i)} for i, (a, b) in enumerate(shapes)]
    b = rd.Batch(specs, dtype=F64, reaction=reaction, boundary=boundary)
    b.set_tune(k=3)
    starts = []
    for i, s in enumerate(specs):
        x = inp.uniform_field(110 + i, s["nn"], s["nm"])
        y = inp.uniform_field(210 + i, s["nn"], s["nm"])
        starts.append((1.5 * x, 0.3 * y) if reaction == "cenn" else (x, y))
        b.set_state(i, torch.from_numpy(starts[-1][0]), torch.from_numpy(starts[-1][1]))
    T = 19
    b.run(T)
    torch.cuda.synchronize()
    rx = {"fhn": oracle_mod.FHN, "none": oracle_mod.NONE, "cenn": oracle_mod.CENN}[reaction]
    bc = oracle_mod.ZEROFLUX if boundary == "zeroflux" else oracle_mod.PERIODIC
    for i, s in enumerate(specs):
        u0, v0 = starts[i]
        u, v = (t.cpu().numpy() for t in b.state(i))
        ref_u, ref_v = oracle_mod.run(u0, v0, s["params"], T, reaction=rx, boundary=bc)
        assert normwise(u, ref_u) <= 1e-12 and normwise(v, ref_v) <= 1e-12, i
        one = gpu_run(rd, u0, v0, s["params"], T, F64, "generic", reaction=reaction, boundary=boundary)
        assert np.array_equal(u, one[0]) and np.array_equal(v, one[1]), i


STORAGE = [("bf16", torch.bfloat16), ("f16", torch.float16)]
MODELS16 = [("fhn", "periodic"), ("fhn", "zeroflux"), ("cenn", "zeroflux")]


@pytest.mark.parametrize("k", [4, 8])
@pytest.mark.parametrize("model", MODELS16, ids=[f"{r}-{b}" for r, b in MODELS16])
@pytest.mark.parametrize("storage,dt", STORAGE, ids=[s for s, _ in STORAGE])
def test_batch_16bit_vs_single_grid_and_storage_oracle(rd, oracle_mod, storage, dt, model, k):
    """16-bit planes in the batched sweep: T = 4k runs as four launches of k steps, the same
    rounding schedule as a single-grid temporal run at depth k (same bits) and as the
    oracle's storage reference with blocks of k steps (bars of test_gpu_storage)."""
    from test_gpu_storage import _close

    reaction, boundary = model
    shapes = [(37, 64), (5, 8), (128, 132)]
    specs = [{"nn": a, "nm": b, "params": dict(CENN_GENE, Du=0.05 + 0.02 * i) if reaction == "cenn"
              else inp.default_params(Du=0.1 + 0.05 * i)} for i, (a, b) in enumerate(shapes)]
    b = rd.Batch(specs, dtype=dt, reaction=reaction, boundary=boundary)
    b.set_tune(k=k)
    starts = []
    for i, s in enumerate(specs):
        x = inp.uniform_field(120 + i, s["nn"], s["nm"])
        y = inp.uniform_field(220 + i, s["nn"], s["nm"])
        u0, v0 = (1.5 * x, 0.3 * y) if reaction == "cenn" else (x, y)
        # start from the 16-bit values both sides use
        u0 = torch.from_numpy(u0).to(dt).double().numpy()
        v0 = torch.from_numpy(v0).to(dt).double().numpy()
        starts.append((u0, v0))
        b.set_state(i, torch.from_numpy(u0), torch.from_numpy(v0))
    T = 4 * k
    b.run(T)
    torch.cuda.synchronize()
    rx = {"fhn": oracle_mod.FHN, "none": oracle_mod.NONE, "cenn": oracle_mod.CENN}[reaction]
    bc = oracle_mod.ZEROFLUX if boundary == "zeroflux" else oracle_mod.PERIODIC
    for i, s in enumerate(specs):
        u0, v0 = starts[i]
        u, v = (t.double().cpu().numpy() for t in b.state(i))
        one = gpu_run(rd, u0, v0, s["params"], T, dt, "temporal", k, reaction=reaction, boundary=boundary)
        assert np.array_equal(u, one[0]) and np.array_equal(v, one[1]), i
        su, sv = oracle_mod.run_storage(u0, v0, s["params"], T, k, storage, reaction=rx, boundary=bc)
        _close(u, v, su.astype(np.float64), sv.astype(np.float64), storage, (i, s["nn"], s["nm"]))


def test_sweep_zero_flux_cenn(rd):
    """search.sweep forwards the model variant to the batch."""
    from paper_2102_10340_gb300 import search
    genes = [dict(CENN_GENE, Du=d) for d in (0.05, 0.1)]
    out = search.sweep(genes, N=64, T=40, reaction="cenn", boundary="zeroflux", checkpoints=2)
    assert out["stats"].shape == (2, 3, 8) and np.isfinite(out["stats"]).all()


def test_full_sweep_in_the_benchmark_launch_shape(rd, oracle_mod):
    """All 256 instances of the seeded sweep (sides 128 .. 1024), k = 4 and 128-row strips as
    the benchmark times them: after T = 500 two instances of each size match the oracle run
    one by one (1e-5), and after T = 5000 sampled instances carry the bits of single-grid
    runs of the same gene and start (FP32 results do not depend on the launch shape)."""
    specs = inp.sweep_instances(0)
    b = rd.Batch(specs, dtype=F32)
    b.set_tune(k=4, rows=128)
    xs = _load(b, specs, F32)
    b.run(500)
    torch.cuda.synchronize()
    picked, seen = [], {}
    for i, s in enumerate(specs):
        if seen.get(s["nn"], 0) < 2:
            seen[s["nn"]] = seen.get(s["nn"], 0) + 1
            picked.append(i)
    assert len(picked) == 8
    for i in picked:
        s = specs[i]
        ref_u, ref_v = oracle_mod.run(xs[i], xs[i], s["params"], 500, nthreads=cpu_threads())
        u, v = (t.double().cpu().numpy() for t in b.state(i))
        assert normwise(u, ref_u) <= 1e-5 and normwise(v, ref_v) <= 1e-5, (i, s["nn"])
    b.run(4500)
    torch.cuda.synchronize()
    for i in (picked[0], picked[3], picked[5], picked[7], len(specs) - 1):
        s = specs[i]
        one = gpu_run(rd, xs[i], xs[i], s["params"], 5000, F32, "temporal", 8)
        u, v = (t.double().cpu().numpy() for t in b.state(i))
        assert np.array_equal(u, one[0]) and np.array_equal(v, one[1]), (i, s["nn"])
