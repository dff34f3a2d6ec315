"""GPU forward path vs the FP64 oracle, through the C ABI.

Tolerances (normwise relative error ||gpu - oracle|| / ||oracle||):
  FP64 kernels: 1e-12 -- the two sides differ only in rounding order (FMA,
                the form of u^3/3), amplified mildly by the dynamics;
  FP32 kernels: 1e-5  -- the stated target after 1000 steps on the 64 x 64
                workload; the FP32 rounding unit is 6e-8.
Variants that share the cell arithmetic (generic, single-step, temporal of
any depth, batched) must agree bit for bit with each other.
"""
import numpy as np
import pytest
import torch

import rdcnn_inputs as inp
from _util import cpu_threads, f32, gpu_run, normwise

pytestmark = pytest.mark.gpu

F32, F64 = torch.float32, torch.float64
TOL = {F32: 1e-5, F64: 1e-12}


def _variants(nm, dtype):
    vec = 4 if dtype == F32 else 2
    out = [("generic", 0)]
    if nm % vec == 0:
        out += [("step1", 0), ("temporal", 1), ("temporal", 2)]
        out += [("temporal", k) for k in ((3, 4, 5, 8) if dtype == F32 else (3, 4))]
        out += [("temporal2", k) for k in ((2, 5, 8) if dtype == F32 else (2, 4))]
    if dtype == F32 and nm % 8 == 0:
        out += [("temporal_wide", k) for k in (1, 2, 4)]
    return out


@pytest.mark.parametrize("dtype", [F64, F32], ids=["f64", "f32"])
def test_config_64x64_T1000(rd, oracle_mod, dtype):
    """64 x 64, default gene, x ~ U[-1,1] seed 0, u = v = x, T = 1000."""
    x = inp.uniform_field(0, 64, 64)
    if dtype == F32:
        x = f32(x)
    ref_u, ref_v = oracle_mod.run(x, x, inp.default_params(), 1000)
    for variant, k in _variants(64, dtype):
        u, v = gpu_run(rd, x, x, inp.default_params(), 1000, dtype, variant, k)
        eu, ev = normwise(u, ref_u), normwise(v, ref_v)
        assert eu <= TOL[dtype] and ev <= TOL[dtype], (variant, k, eu, ev)
        assert np.max(np.abs(u - ref_u)) <= (1e-10 if dtype == F64 else 1e-4)


SHAPES = [(1, 1), (1, 4), (2, 2), (3, 3), (4, 5), (4, 4), (3, 8), (5, 12), (7, 20), (37, 53),
          (33, 64), (17, 132), (129, 260), (64, 120), (65, 244), (300, 8)]


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a}x{b}" for a, b in SHAPES])
@pytest.mark.parametrize("dtype", [F64, F32], ids=["f64", "f32"])
def test_ragged_and_tiny_grids(rd, oracle_mod, shape, dtype):
    nn, nm = shape
    x = inp.uniform_field(3, nn, nm)
    y = inp.uniform_field(4, nn, nm)
    if dtype == F32:
        x, y = f32(x), f32(y)
    T = 37
    ref_u, ref_v = oracle_mod.run(x, y, inp.default_params(), T)
    first = None
    for variant, k in _variants(nm, dtype):
        u, v = gpu_run(rd, x, y, inp.default_params(), T, dtype, variant, k)
        assert normwise(u, ref_u) <= TOL[dtype] and normwise(v, ref_v) <= TOL[dtype], (variant, k)
        if first is None:
            first = (u, v)
        else:  # identical cell arithmetic in every variant
            assert np.array_equal(u, first[0]) and np.array_equal(v, first[1]), (variant, k)


@pytest.mark.parametrize("rows", [1, 3, 8, 64])
def test_launch_shape_does_not_change_bits(rd, rows):
    x = f32(inp.uniform_field(9, 70, 136))
    base = gpu_run(rd, x, -x, inp.default_params(), 23, F32, "generic")
    for variant, k in (("step1", 0), ("temporal", 3), ("temporal", 8), ("temporal2", 3), ("temporal2", 8),
                       ("temporal_wide", 3), ("temporal_wide", 4)):
        got = gpu_run(rd, x, -x, inp.default_params(), 23, F32, variant, k, rows=rows)
        assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1]), (variant, k, rows)


@pytest.mark.parametrize("dtype", [F64, F32], ids=["f64", "f32"])
def test_uniform_stays_uniform_and_matches_1x1(rd, dtype):
    u0 = np.full((40, 64), 0.37)
    v0 = np.full((40, 64), -0.21)
    u, v = gpu_run(rd, u0, v0, inp.default_params(), 301, dtype, "temporal", 0)
    assert np.all(u == u[0, 0]) and np.all(v == v[0, 0])
    su, sv = gpu_run(rd, u0[:1, :1], v0[:1, :1], inp.default_params(), 301, dtype, "generic")
    assert u[0, 0] == su[0, 0] and v[0, 0] == sv[0, 0]


@pytest.mark.parametrize("variant,k", [("step1", 0), ("temporal", 4), ("generic", 0)])
def test_fourier_mode_decay_f64(rd, variant, k):
    nn, nm, p, q = 48, 80, 3, 5
    par = {"dt": 0.05, "a": 0.2, "b": 0.7, "eps": 0.3, "c": 0.5, "Du": 0.11, "Dv": 0.37}
    u0 = inp.fourier_mode(nn, nm, p, q)
    v0 = inp.fourier_mode(nn, nm, q, p)
    T = 40
    u, v = gpu_run(rd, u0, v0, par, T, F64, variant, k, reaction="none")

    def gain(D, pp, qq):
        return 1 - par["dt"] * D * (4 - 2 * np.cos(2 * np.pi * pp / nn) - 2 * np.cos(2 * np.pi * qq / nm))

    assert np.max(np.abs(u - gain(par["Du"], p, q) ** T * u0)) < 1e-12
    assert np.max(np.abs(v - gain(par["Dv"], q, p) ** T * v0)) < 1e-12


def test_mass_conserved_without_reaction_f64(rd):
    x = inp.uniform_field(5, 96, 128)
    y = inp.uniform_field(6, 96, 128)
    u, v = gpu_run(rd, x, y, inp.default_params(), 57, F64, "temporal", 3, reaction="none")
    assert abs(u.sum() - x.sum()) < 1e-9 and abs(v.sum() - y.sum()) < 1e-9


def test_shift_and_transpose_equivariance_bitwise(rd):
    x = f32(inp.uniform_field(7, 128, 128))
    base = gpu_run(rd, x, -x, inp.default_params(), 29, F32, "temporal", 4)
    sh = gpu_run(rd, np.roll(x, (5, -12), (0, 1)), np.roll(-x, (5, -12), (0, 1)), inp.default_params(),
                 29, F32, "temporal", 4)
    assert np.array_equal(sh[0], np.roll(base[0], (5, -12), (0, 1)))
    tr = gpu_run(rd, x.T.copy(), -x.T.copy(), inp.default_params(), 29, F32, "temporal", 4)
    assert np.array_equal(tr[0], base[0].T) and np.array_equal(tr[1], base[1].T)


def test_zero_steps_and_state_roundtrip(rd):
    x = f32(inp.uniform_field(8, 16, 32))
    g = rd.Grid(16, 32, inp.default_params(), dtype=F32)
    g.set_state(torch.from_numpy(x).float(), torch.from_numpy(-x).float())  # host -> device
    g.run(0)
    hu = torch.empty((16, 32), dtype=F32).pin_memory()
    hv = torch.empty((16, 32), dtype=F32)
    g.get_state(hu, hv)
    assert np.array_equal(hu.numpy().astype(np.float64), x) and np.array_equal(hv.numpy().astype(np.float64), -x)


def test_init_from_host_and_device(rd, oracle_mod):
    x = f32(inp.uniform_field(12, 32, 64))
    ka = 0.75
    ref = oracle_mod.run(*oracle_mod.init_state(x, ka), inp.default_params(), 10)
    for src in (torch.from_numpy(x).float(), torch.from_numpy(x).float().cuda()):
        g = rd.Grid(32, 64, inp.default_params(), dtype=F32)
        g.init(src, ka).run(10)
        u, v = (t.double().cpu().numpy() for t in g.state())
        assert normwise(u, ref[0]) < 1e-6 and normwise(v, ref[1]) < 1e-6


def test_smooth_noise_1024_T1000(rd, oracle_mod):
    """Image-style workload: 1024^2 FP32, blurred-noise image, compared after 1000 steps, in
    the AUTO shape and in the shapes the benchmark's autotuner picks for it (graph replay)."""
    x = f32(inp.smooth_noise(0, 1024, 1024))
    ref_u, ref_v = oracle_mod.run(x, x, inp.default_params(), 1000, nthreads=cpu_threads())
    first = None
    for variant, k, rows in (("auto", 0, 0), ("temporal", 3, 8), ("temporal", 4, 8), ("temporal", 4, 16)):
        u, v = gpu_run(rd, x, x, inp.default_params(), 1000, F32, variant, k, rows=rows)
        assert normwise(u, ref_u) <= 1e-5 and normwise(v, ref_v) <= 1e-5, (variant, k, rows)
        if first is None:
            first = (u, v)
        assert np.array_equal(u, first[0]) and np.array_equal(v, first[1]), (variant, k, rows)


@pytest.mark.parametrize("T,M", [(500, 1024), (1000, 2048)])
def test_slow_growth_4096_light_cone(rd, oracle_mod, T, M):
    """4096^2 centred-patch workload in the launch configuration the benchmark times.

    A 16 x 16 patch influences only cells within distance T, so the centre M x M
    window equals the same patch run on an M x M torus (M >= 16 + 2T), and every
    cell outside it follows the cell map from (0, 0)."""
    N = 4096
    x = f32(inp.mid_patch(0, N, N))
    u, v = gpu_run(rd, x, x, inp.default_params(), T, F32, "auto")
    xs = f32(inp.mid_patch(0, M, M))
    assert np.array_equal(xs, x[(N - M) // 2:(N + M) // 2, (N - M) // 2:(N + M) // 2])
    ref_u, ref_v = oracle_mod.run(xs, xs, inp.default_params(), T, nthreads=cpu_threads())
    o = (N - M) // 2
    assert normwise(u[o:o + M, o:o + M], ref_u) <= 1e-5
    assert normwise(v[o:o + M, o:o + M], ref_v) <= 1e-5
    far = np.ones((N, N), bool)
    far[o:o + M, o:o + M] = False
    assert np.all(u[far] == u[0, 0]) and np.all(v[far] == v[0, 0])
    bu, bv = oracle_mod.scalar_map(0.0, 0.0, inp.default_params(), T)
    assert abs(u[0, 0] - bu[-1]) <= 1e-5 * max(1, abs(bu[-1])) and abs(v[0, 0] - bv[-1]) <= 1e-5 * max(1, abs(bv[-1]))


def test_full_size_random_sampled_cells(rd, oracle_mod):
    """4096^2 fully random state, T = 48: sampled cells against the oracle run on the
    (2T+3)^2 periodic window centred on each cell (exact at the centre)."""
    N, T = 4096, 48
    x = f32(inp.uniform_field(0, N, N))
    u, v = gpu_run(rd, x, x, inp.default_params(), T, F32, "auto")
    rng = np.random.default_rng(1)
    W = 2 * T + 3
    for _ in range(12):
        i, j = rng.integers(0, N, size=2)
        rows = (np.arange(W) + i - W // 2) % N
        cols = (np.arange(W) + j - W // 2) % N
        win = x[np.ix_(rows, cols)]
        ou, ov = oracle_mod.run(win, win, inp.default_params(), T)
        c = W // 2
        assert abs(u[i, j] - ou[c, c]) <= 1e-4 * max(1.0, abs(ou[c, c]))
        assert abs(v[i, j] - ov[c, c]) <= 1e-4 * max(1.0, abs(ov[c, c]))


def test_temporal_matches_step1_at_full_size_bitwise(rd):
    N = 4096
    x = f32(inp.mid_patch(3, N, N)) + f32(0.05 * inp.uniform_field(4, N, N))
    a = gpu_run(rd, x, x, inp.default_params(), 24, F32, "temporal", 4)
    b = gpu_run(rd, x, x, inp.default_params(), 24, F32, "step1")
    c = gpu_run(rd, x, x, inp.default_params(), 24, F32, "temporal2", 8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(c[0], b[0]) and np.array_equal(c[1], b[1])


def test_misaligned_views_use_generic_or_fail_loudly(rd, oracle_mod):
    base = torch.zeros(1 + 16 * 32, dtype=F32, device="cuda")
    u = base[1:].view(16, 32)  # 4-byte offset: not 16-byte aligned
    v = torch.zeros((16, 32), dtype=F32, device="cuda")
    x = f32(inp.uniform_field(2, 16, 32))
    u.copy_(torch.from_numpy(x)); v.copy_(torch.from_numpy(x))
    with pytest.raises(rd.RDCNNError):
        rd.run(u, v, inp.default_params(), 5, variant="temporal")
    u.copy_(torch.from_numpy(x)); v.copy_(torch.from_numpy(x))
    rd.run(u, v, inp.default_params(), 5, variant="auto")
    ref = oracle_mod.run(x, x, inp.default_params(), 5)
    assert normwise(u.double().cpu().numpy(), ref[0]) < 1e-6


def test_launch_counter_counts(rd):
    before = rd.launch_count()
    gpu_run(rd, np.zeros((8, 8)), np.zeros((8, 8)), inp.default_params(), 12, F32, "temporal", 4)
    assert rd.launch_count() - before >= 3


def test_wide_variant_rejects_unsupported_planes(rd):
    g = rd.Grid(16, 20, None, dtype=F32)  # NM = 20: not a multiple of 8
    g.set_state(torch.zeros((16, 20), device="cuda"), torch.zeros((16, 20), device="cuda"))
    with pytest.raises(rd.RDCNNError):
        g.run(4, variant="temporal_wide", k=2)
    g.run(4, variant="temporal", k=2)  # the 4-value lane still runs
    g.close()
    g = rd.Grid(16, 16, None, dtype=F64)
    g.set_state(torch.zeros((16, 16), device="cuda", dtype=F64), torch.zeros((16, 16), device="cuda", dtype=F64))
    with pytest.raises(rd.RDCNNError):
        g.run(4, variant="temporal_wide", k=2)
    g.close()


@pytest.mark.parametrize("variant,k", [("generic", 0), ("step1", 0), ("temporal", 4)])  # FP64: k <= 4
def test_degenerate_genes(rd, oracle_mod, variant, k):
    """dt = 0 leaves the state bitwise unchanged; Du = Dv = 0 decouples the cells, each then
    following the oracle's scalar map (FP64, cell by cell)."""
    x = inp.uniform_field(21, 24, 40)
    y = inp.uniform_field(22, 24, 40)
    still = dict(inp.default_params(), dt=0.0)
    u, v = gpu_run(rd, x, y, still, 64, F64, variant, k)
    assert np.array_equal(u, x) and np.array_equal(v, y)
    apart = dict(inp.default_params(), Du=0.0, Dv=0.0)
    u, v = gpu_run(rd, x, y, apart, 50, F64, variant, k)
    for i, j in ((0, 0), (5, 17), (23, 39), (11, 3)):
        su, sv = oracle_mod.scalar_map(x[i, j], y[i, j], apart, 50)
        assert abs(u[i, j] - su[-1]) <= 1e-12 and abs(v[i, j] - sv[-1]) <= 1e-12


@pytest.mark.parametrize("shape", [(1, 64), (57, 4), (1, 4), (2, 8)])
def test_single_row_and_column_tori(rd, oracle_mod, shape):
    """One-row (or few-column) tori: a cell is its own north and south neighbour; the temporal
    pipeline's halo rows all wrap to the same rows."""
    x = inp.uniform_field(23, *shape)
    ref = oracle_mod.run(x, -x, inp.default_params(), 33)
    for variant, k in (("step1", 0), ("temporal", 3), ("temporal", 4)):
        u, v = gpu_run(rd, x, -x, inp.default_params(), 33, F64, variant, k)
        assert normwise(u, ref[0]) <= 1e-12 and normwise(v, ref[1]) <= 1e-12, (variant, k)
