"""Randomised launch shapes (seeded): every vectorised variant, at random
depths and strip lengths, on random grid shapes, models and plane types,
must give exactly the bits of the one-thread-per-cell generic kernel (for
16-bit planes: at the same rounding interval, i.e. the generic kernel run
with the same number of steps per rounding is the single-step schedule, so
the comparison there is at k = 1).  Bit identity across the variants is what
lets the oracle comparisons of the other tests cover every launch shape."""
import numpy as np
import pytest
import torch

import rdcnn_inputs as inp
from _util import gpu_run

pytestmark = pytest.mark.gpu

CENN_GENE = {"dt": 0.1, "a": 0.0, "b": 0.0, "eps": 0.0, "c": 1.2, "Du": 0.1, "Dv": 0.0}


def _cases(n=64, seed=2021):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        dtype = [torch.float32, torch.float64, torch.bfloat16][rng.integers(0, 3)]
        vec = 2 if dtype == torch.float64 else 4
        nn = int(rng.integers(1, 180))
        nm = int(vec * rng.integers(1, 70))
        reaction = ["fhn", "none", "cenn"][rng.integers(0, 3)]
        boundary = ["periodic", "zeroflux"][rng.integers(0, 2)]
        maxk = 4 if dtype == torch.float64 else 8
        if dtype == torch.bfloat16:
            k = 1  # one rounding per step: the schedule the generic kernel follows
        else:
            k = int(rng.integers(1, maxk + 1))
        eligible = ["temporal"]
        if k <= 4 and dtype != torch.float64 and nm % 8 == 0:
            eligible.append("temporal_wide")
        if dtype != torch.bfloat16 and k >= 2:
            eligible.append("temporal2")
        variant = str(rng.choice(eligible))
        rows = int(rng.choice([0, 1, 2, 3, 5, 8, 16, 33, 128]))
        T = int(rng.integers(1, 3 * k + 4))
        out.append((i, dtype, nn, nm, reaction, boundary, variant, k, rows, T))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[f"c{c[0]}" for c in CASES])
def test_variant_bits_equal_generic(rd, case):
    _, dtype, nn, nm, reaction, boundary, variant, k, rows, T = case
    gene = CENN_GENE if reaction == "cenn" else inp.default_params()
    x = 1.5 * inp.uniform_field(7, nn, nm)
    y = 0.4 * inp.uniform_field(8, nn, nm)
    if dtype == torch.bfloat16:
        x = torch.from_numpy(x).to(dtype).double().numpy()
        y = torch.from_numpy(y).to(dtype).double().numpy()
    ref = gpu_run(rd, x, y, gene, T, dtype, "generic", 0, reaction=reaction, boundary=boundary)
    got = gpu_run(rd, x, y, gene, T, dtype, variant, k, reaction=reaction, boundary=boundary, rows=rows)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), case
    step = gpu_run(rd, x, y, gene, T, dtype, "step1", 0, reaction=reaction, boundary=boundary)
    if dtype != torch.bfloat16 or k == 1:
        assert np.array_equal(step[0], ref[0]) and np.array_equal(step[1], ref[1]), case


def _batch_cases(n=16, seed=77):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        dtype = [torch.float32, torch.float64, torch.bfloat16][rng.integers(0, 3)]
        vec = 2 if dtype == torch.float64 else 4
        reaction = ["fhn", "none", "cenn"][rng.integers(0, 3)]
        boundary = ["periodic", "zeroflux"][rng.integers(0, 2)]
        maxk = 4 if dtype == torch.float64 else 8
        k = 1 if dtype == torch.bfloat16 else int(rng.integers(1, maxk + 1))
        rows = int(rng.choice([0, 3, 16, 64, 256]))
        shapes = [(int(rng.integers(1, 150)), int(vec * rng.integers(1, 40))) for _ in range(int(rng.integers(1, 6)))]
        T = int(rng.integers(1, 3 * k + 4))
        out.append((i, dtype, reaction, boundary, k, rows, shapes, T))
    return out


BATCH_CASES = _batch_cases()


@pytest.mark.parametrize("case", BATCH_CASES, ids=[f"b{c[0]}" for c in BATCH_CASES])
def test_batch_bits_equal_generic(rd, case):
    """Random instance lists (sizes, genes), models, plane types and launch shapes: every
    instance of a batched sweep carries the bits of its own generic single-grid run (16-bit
    planes at one step per launch, the generic kernel's rounding schedule)."""
    _, dtype, reaction, boundary, k, rows, shapes, T = case
    specs = []
    for j, (nn, nm) in enumerate(shapes):
        gene = dict(CENN_GENE, Du=0.05 + 0.03 * j) if reaction == "cenn" else inp.default_params(Du=0.1 + 0.04 * j)
        specs.append({"nn": nn, "nm": nm, "params": gene})
    b = rd.Batch(specs, dtype=dtype, reaction=reaction, boundary=boundary)
    b.set_tune(k=k, rows=rows)
    starts = []
    for j, s in enumerate(specs):
        x = 1.5 * inp.uniform_field(30 + j, s["nn"], s["nm"])
        y = 0.4 * inp.uniform_field(60 + j, s["nn"], s["nm"])
        x = torch.from_numpy(x).to(dtype).double().numpy()
        y = torch.from_numpy(y).to(dtype).double().numpy()
        starts.append((x, y))
        b.set_state(j, torch.from_numpy(x), torch.from_numpy(y))
    b.run(T)
    torch.cuda.synchronize()
    for j, s in enumerate(specs):
        ref = gpu_run(rd, starts[j][0], starts[j][1], s["params"], T, dtype, "generic", 0, reaction=reaction,
                      boundary=boundary)
        u, v = (t.double().cpu().numpy() for t in b.state(j))
        assert np.array_equal(u, ref[0]) and np.array_equal(v, ref[1]), (case, j)
