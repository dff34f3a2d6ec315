"""Reverse-time adjoint on the GPU vs the oracle adjoint (itself pinned to
finite differences on the CPU), vs finite differences of the GPU forward, and
through torch.autograd.

Tolerances: FP64 kernels 1e-8..1e-10 relative (rounding order only); FP32
kernels 1e-4 relative for the gene-gradient vector (the stated gradient
target), with the FP64 oracle started from the same FP32-rounded state.
"""
import numpy as np
import pytest
import torch

import rdcnn_inputs as inp
from _util import cpu_threads, f32, gpu_run, normwise

pytestmark = pytest.mark.gpu

F32, F64 = torch.float32, torch.float64
NAMES = ("Du", "Dv", "a", "b", "eps", "c")


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _gpu_adjoint(rd, u0, v0, params, T, gu, gv, dtype, nck=0):
    g = rd.Grid(u0.shape[0], u0.shape[1], params, dtype=dtype)
    du, dv, gp = g.adjoint(T, _dev(u0, dtype), _dev(v0, dtype), _dev(gu, dtype), _dev(gv, dtype), nck)
    torch.cuda.synchronize()
    return du.double().cpu().numpy(), dv.double().cpu().numpy(), np.array([gp[k] for k in NAMES])


@pytest.mark.parametrize("nck", [0, 1, 7, 50])
def test_f64_adjoint_matches_oracle(rd, oracle_mod, nck):
    nn, nm, T = 24, 40, 50
    params = inp.default_params()
    x = inp.uniform_field(1, nn, nm)
    y = inp.uniform_field(2, nn, nm)
    wu = inp.uniform_field(3, nn, nm)
    wv = inp.uniform_field(4, nn, nm)
    du, dv, g = _gpu_adjoint(rd, x, y, params, T, wu, wv, F64, nck)
    ou, ov, og = oracle_mod.adjoint(x, y, params, T, wu, wv, n_checkpoints=nck)
    assert normwise(du, ou) < 1e-10 and normwise(dv, ov) < 1e-10
    np.testing.assert_allclose(g, og, rtol=1e-9, atol=1e-12)


def test_f64_adjoint_vs_gpu_finite_differences(rd):
    nn, nm, T = 16, 32, 30
    params = {"dt": 0.05, "a": 0.2, "b": 0.7, "eps": 0.3, "c": 0.5, "Du": 0.11, "Dv": 0.37}
    x = inp.uniform_field(5, nn, nm)
    y = inp.uniform_field(6, nn, nm)
    wu = inp.uniform_field(7, nn, nm)
    wv = inp.uniform_field(8, nn, nm)
    _, _, g = _gpu_adjoint(rd, x, y, params, T, wu, wv, F64)

    def loss(p):
        u, v = gpu_run(rd, x, y, p, T, F64, "temporal", 3)
        return float(np.sum(wu * u) + np.sum(wv * v))

    for k, name in enumerate(NAMES):
        h = 1e-5 * max(1.0, abs(params[name]))
        pp = dict(params); pp[name] += h
        pm = dict(params); pm[name] -= h
        fd = (loss(pp) - loss(pm)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * max(1.0, abs(fd)), (name, g[k], fd)


def test_adjoint_without_reaction_is_forward_of_costate(rd):
    """Self-adjointness of the periodic Laplacian: with no reaction the adjoint sweep
    equals the forward sweep applied to the co-state, bit for bit."""
    nn, nm, T = 32, 64, 21
    params = inp.default_params(Du=0.13, Dv=0.21)
    x = f32(inp.uniform_field(9, nn, nm))
    wu = f32(inp.uniform_field(10, nn, nm))
    wv = f32(inp.uniform_field(11, nn, nm))
    g = rd.Grid(nn, nm, params, dtype=F32, reaction="none")
    du, dv, gp = g.adjoint(T, _dev(x, F32), _dev(x, F32), _dev(wu, F32), _dev(wv, F32))
    fu, fv = gpu_run(rd, wu, wv, params, T, F32, "step1", reaction="none")
    assert np.array_equal(du.double().cpu().numpy(), fu) and np.array_equal(dv.double().cpu().numpy(), fv)
    assert all(gp[k] == 0.0 for k in ("a", "b", "eps", "c"))


def _mse_seed(uT, target):
    return 2.0 * (uT - target) / uT.size


@pytest.mark.parametrize("T,gtol", [(200, 1e-3), (2000, 1e-4)])
def test_f32_checkerboard_mse_512(rd, oracle_mod, T, gtol):
    """512^2 FP32, MSE(u_T, checkerboard of period 32), sqrt(T) checkpoints.

    Gene gradient: ||g_gpu - g_ref|| / ||g_ref|| <= 1e-4 at the workload's horizon T = 2000
    against the FP64 oracle adjoint (which is pinned to FP64 finite differences).  The
    vector norm is the measure: single entries can be nearly cancelled sums (dL/db is
    ~1e-4 of ||g|| at T = 200).  At T = 200 the field is mid-transient and the FP32
    trajectory itself is ill-conditioned (FP64 co-state along an FP32 trajectory:
    7e-5 on the CPU, 2.4e-4 with the GPU's rounding order), so that horizon gets 1e-3.
    State gradient: the FP32 forward trajectory differs from the FP64 one by rounding, and
    dL/du0 is sensitive to it: an FP64 co-state swept along the FP32 trajectory is already
    ~2e-3 away from the FP64 reference, while the FP32 co-state arithmetic itself adds ~1e-7
    (measured on the CPU); the GPU measured 2.4e-3 / 2.5e-3 (u0 / v0) at T = 200 and
    3.6e-3 / 3.9e-3 at T = 2000.  The bound below is therefore 5e-3 normwise."""
    N = 512
    params = inp.default_params()
    x = f32(inp.uniform_field(0, N, N))
    target = inp.checkerboard(0, N, N)
    uT, _ = gpu_run(rd, x, x, params, T, F32, "auto")
    gu = f32(_mse_seed(uT, target))
    du, dv, g = _gpu_adjoint(rd, x, x, params, T, gu, 0 * gu, F32)
    ou, ov, og = oracle_mod.adjoint(x, x, params, T, gu, 0 * gu, nthreads=cpu_threads())
    assert np.linalg.norm(g - og) <= gtol * np.linalg.norm(og), dict(zip(NAMES, np.abs(g - og)))
    assert normwise(du, ou) <= 5e-3 and normwise(dv, ov) <= 5e-3


def test_f32_adjoint_short_horizon_is_tight(rd, oracle_mod):
    """Over a short horizon the FP32 and FP64 trajectories agree to ~1e-7, so the FP32
    adjoint must match the FP64 oracle closely: this isolates the adjoint arithmetic."""
    N, T = 256, 20
    params = inp.default_params()
    x = f32(inp.uniform_field(3, N, N))
    gu = f32(inp.uniform_field(4, N, N)) / (N * N)
    gv = f32(inp.uniform_field(5, N, N)) / (N * N)
    du, dv, g = _gpu_adjoint(rd, x, x, params, T, gu, gv, F32)
    ou, ov, og = oracle_mod.adjoint(x, x, params, T, gu, gv)
    assert normwise(du, ou) <= 1e-5 and normwise(dv, ov) <= 1e-5
    np.testing.assert_allclose(g, og, rtol=1e-5, atol=1e-6 * np.linalg.norm(og))


def test_f64_adjoint_full_size_512_T2000(rd, oracle_mod):
    """The adjoint workload at full size (512^2, T = 2000, sqrt(T) = 45 checkpoints) in the
    FP64 instantiation of the same kernels: rounding-order agreement with the oracle."""
    N, T = 512, 2000
    params = inp.default_params()
    x = inp.uniform_field(0, N, N)
    target = inp.checkerboard(0, N, N)
    uT, _ = oracle_mod.run(x, x, params, T, nthreads=cpu_threads())
    gu = _mse_seed(uT, target)
    du, dv, g = _gpu_adjoint(rd, x, x, params, T, gu, 0 * gu, F64)
    ou, ov, og = oracle_mod.adjoint(x, x, params, T, gu, 0 * gu, nthreads=cpu_threads())
    assert normwise(du, ou) <= 1e-8 and normwise(dv, ov) <= 1e-8
    np.testing.assert_allclose(g, og, rtol=1e-8, atol=1e-10 * np.linalg.norm(og))


def test_autograd_function_gradcheck_f64(rd):
    from torch.autograd import gradcheck

    nn, nm, T = 6, 8, 5
    u0 = _dev(inp.uniform_field(12, nn, nm), F64).requires_grad_()
    v0 = _dev(inp.uniform_field(13, nn, nm), F64).requires_grad_()
    p = inp.default_params()
    theta = torch.tensor([p[k] for k in NAMES], dtype=F64, device="cuda", requires_grad=True)
    f = lambda a, b, t: rd.RDCNNFunction.apply(a, b, t, T, p["dt"])  # noqa: E731
    assert gradcheck(f, (u0, v0, theta), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_autograd_end_to_end_fit_step(rd):
    """One gradient step on Du, Dv through RDCNNFunction lowers an MSE loss."""
    N, T = 64, 60
    p = inp.default_params()
    x = _dev(f32(inp.uniform_field(0, N, N)), F32)
    target = _dev(inp.checkerboard(0, N, N), F32)
    theta = torch.tensor([p[k] for k in NAMES], dtype=F64, device="cuda", requires_grad=True)
    uT, _ = rd.RDCNNFunction.apply(x, x, theta, T, p["dt"])
    loss = torch.mean((uT - target) ** 2)
    loss.backward()
    assert torch.isfinite(theta.grad).all()
    with torch.no_grad():
        th2 = theta - 1e-3 * theta.grad / theta.grad.norm()
    u2, _ = rd.RDCNNFunction.apply(x, x, th2, T, p["dt"])
    assert torch.mean((u2 - target) ** 2).item() < loss.item()


# ----------------------------------------------------------------------------- zero-flux boundary

ZF_SHAPES = [(24, 40), (9, 6), (33, 130), (1, 8)]


@pytest.mark.parametrize("shape", ZF_SHAPES, ids=[f"{a}x{b}" for a, b in ZF_SHAPES])
@pytest.mark.parametrize("nck", [0, 7])
def test_f64_zeroflux_adjoint_matches_oracle(rd, oracle_mod, shape, nck):
    """Zero flux: mirrored halos for the co-state and for the state rows the reverse pass
    reads; the oracle adjoint (pinned to central differences of the zero-flux forward)."""
    nn, nm = shape
    T = 37
    params = inp.default_params(Du=0.17, Dv=0.4)
    x = inp.uniform_field(61, nn, nm)
    y = inp.uniform_field(62, nn, nm)
    wu = inp.uniform_field(63, nn, nm)
    wv = inp.uniform_field(64, nn, nm)
    g = rd.Grid(nn, nm, params, dtype=F64, boundary="zeroflux")
    du, dv, gp = g.adjoint(T, _dev(x, F64), _dev(y, F64), _dev(wu, F64), _dev(wv, F64), nck)
    torch.cuda.synchronize()
    ou, ov, og = oracle_mod.adjoint(x, y, params, T, wu, wv, n_checkpoints=nck, boundary=oracle_mod.ZEROFLUX)
    assert normwise(du.cpu().numpy(), ou) < 1e-10 and normwise(dv.cpu().numpy(), ov) < 1e-10
    np.testing.assert_allclose(np.array([gp[k] for k in NAMES]), og, rtol=1e-9, atol=1e-12)


def test_f32_zeroflux_adjoint_short_horizon(rd, oracle_mod):
    N, T = 200, 20
    params = inp.default_params()
    x = f32(inp.uniform_field(65, N, N))
    gu = f32(inp.uniform_field(66, N, N)) / (N * N)
    gv = f32(inp.uniform_field(67, N, N)) / (N * N)
    g = rd.Grid(N, N, params, dtype=F32, boundary="zeroflux")
    du, dv, gp = g.adjoint(T, _dev(x, F32), _dev(x, F32), _dev(gu, F32), _dev(gv, F32))
    torch.cuda.synchronize()
    ou, ov, og = oracle_mod.adjoint(x, x, params, T, gu, gv, boundary=oracle_mod.ZEROFLUX)
    assert normwise(du.double().cpu().numpy(), ou) <= 1e-5 and normwise(dv.double().cpu().numpy(), ov) <= 1e-5
    got = np.array([gp[k] for k in NAMES])
    np.testing.assert_allclose(got, og, rtol=1e-5, atol=1e-6 * np.linalg.norm(og))


def test_zeroflux_adjoint_without_reaction_is_forward_of_costate(rd):
    """The zero-flux Laplacian is symmetric too: with no reaction the adjoint sweep equals
    the zero-flux forward sweep of the co-state, bit for bit."""
    nn, nm, T = 32, 64, 21
    params = inp.default_params(Du=0.13, Dv=0.21)
    x = f32(inp.uniform_field(68, nn, nm))
    wu = f32(inp.uniform_field(69, nn, nm))
    wv = f32(inp.uniform_field(70, nn, nm))
    g = rd.Grid(nn, nm, params, dtype=F32, reaction="none", boundary="zeroflux")
    du, dv, gp = g.adjoint(T, _dev(x, F32), _dev(x, F32), _dev(wu, F32), _dev(wv, F32))
    fu, fv = gpu_run(rd, wu, wv, params, T, F32, "step1", reaction="none", boundary="zeroflux")
    assert np.array_equal(du.double().cpu().numpy(), fu) and np.array_equal(dv.double().cpu().numpy(), fv)
    assert all(gp[k] == 0.0 for k in ("a", "b", "eps", "c"))


def test_zeroflux_autograd_gradcheck_f64(rd):
    from torch.autograd import gradcheck

    nn, nm, T = 6, 8, 5
    u0 = _dev(inp.uniform_field(71, nn, nm), F64).requires_grad_()
    v0 = _dev(inp.uniform_field(72, nn, nm), F64).requires_grad_()
    p = inp.default_params()
    theta = torch.tensor([p[k] for k in NAMES], dtype=F64, device="cuda", requires_grad=True)
    f = lambda a, b, t: rd.RDCNNFunction.apply(a, b, t, T, p["dt"], 0, "zeroflux")  # noqa: E731
    assert gradcheck(f, (u0, v0, theta), eps=1e-6, atol=1e-7, rtol=1e-5)


CENN_ADJ = {"dt": 0.1, "a": 0.0, "b": 0.0, "eps": 0.0, "c": 1.3, "Du": -0.2, "Dv": 0.0}
CENN_SHAPES = [(24, 40), (9, 6), (33, 130)]


@pytest.mark.parametrize("boundary", ["periodic", "zeroflux"])
@pytest.mark.parametrize("shape", CENN_SHAPES, ids=[f"{a}x{b}" for a, b in CENN_SHAPES])
def test_f64_cenn_adjoint_matches_oracle(rd, oracle_mod, shape, boundary):
    """Chua-Yang cell: the reverse step gates the fed-back co-state by the output function's
    slope; the oracle adjoint is pinned to central differences of the CeNN forward map."""
    nn, nm = shape
    T = 31
    x = 1.7 * inp.uniform_field(81, nn, nm)
    y = inp.uniform_field(82, nn, nm)
    wu = inp.uniform_field(83, nn, nm)
    wv = inp.uniform_field(84, nn, nm)
    g = rd.Grid(nn, nm, CENN_ADJ, dtype=F64, reaction="cenn", boundary=boundary)
    du, dv, gp = g.adjoint(T, _dev(x, F64), _dev(y, F64), _dev(wu, F64), _dev(wv, F64), 5)
    torch.cuda.synchronize()
    bc = oracle_mod.ZEROFLUX if boundary == "zeroflux" else oracle_mod.PERIODIC
    ou, ov, og = oracle_mod.adjoint(x, y, CENN_ADJ, T, wu, wv, n_checkpoints=5, reaction=oracle_mod.CENN,
                                    boundary=bc)
    assert normwise(du.cpu().numpy(), ou) < 1e-10 and normwise(dv.cpu().numpy(), ov) < 1e-10
    got = np.array([gp[k] for k in NAMES])
    np.testing.assert_allclose(got, og, rtol=1e-9, atol=1e-12)
    assert np.all(got[1:5] == 0.0)


def test_f32_cenn_adjoint_short_horizon(rd, oracle_mod):
    N, T = 256, 20
    x = f32(1.7 * inp.uniform_field(85, N, N))
    y = f32(inp.uniform_field(86, N, N))
    gu = f32(inp.uniform_field(87, N, N)) / (N * N)
    gv = f32(inp.uniform_field(88, N, N)) / (N * N)
    g = rd.Grid(N, N, CENN_ADJ, dtype=F32, reaction="cenn")
    du, dv, gp = g.adjoint(T, _dev(x, F32), _dev(y, F32), _dev(gu, F32), _dev(gv, F32))
    torch.cuda.synchronize()
    ou, ov, og = oracle_mod.adjoint(x, y, CENN_ADJ, T, gu, gv, reaction=oracle_mod.CENN)
    assert normwise(du.double().cpu().numpy(), ou) <= 1e-5 and normwise(dv.double().cpu().numpy(), ov) <= 1e-5
    got = np.array([gp[k] for k in NAMES])
    np.testing.assert_allclose(got, og, rtol=1e-5, atol=1e-6 * np.linalg.norm(og))


def test_cenn_autograd_fit_step(rd):
    """Template learning through RDCNNFunction: one gradient step on the CeNN feedback
    weights (Du, c) lowers the distance to a target state produced by other weights."""
    N, T = 48, 30
    x = _dev(f32(1.5 * inp.uniform_field(89, N, N)), F32)
    w = _dev(f32(0.2 * inp.uniform_field(90, N, N)), F32)
    true = dict(CENN_ADJ, c=1.1, Du=0.15)
    target, _ = rd.RDCNNFunction.apply(x, w, torch.tensor([true[k] for k in NAMES], dtype=F64, device="cuda"),
                                       T, 0.1, 0, "periodic", "cenn")
    theta = torch.tensor([CENN_ADJ[k] for k in NAMES], dtype=F64, device="cuda", requires_grad=True)
    uT, _ = rd.RDCNNFunction.apply(x, w, theta, T, 0.1, 0, "periodic", "cenn")
    loss = torch.mean((uT - target.detach()) ** 2)
    loss.backward()
    assert torch.isfinite(theta.grad).all() and theta.grad[1:5].abs().max().item() == 0.0
    with torch.no_grad():
        th2 = theta - 1e-2 * theta.grad / theta.grad.norm()
    u2, _ = rd.RDCNNFunction.apply(x, w, th2, T, 0.1, 0, "periodic", "cenn")
    assert torch.mean((u2 - target) ** 2).item() < loss.item()


@pytest.mark.parametrize("dtype,k", [(F32, 2), (F32, 5), (F32, 8), (F64, 1), (F64, 3), (F64, 4)],
                         ids=["f32-k2", "f32-k5", "f32-k8", "f64-k1", "f64-k3", "f64-k4"])
@pytest.mark.parametrize("model", [("fhn", "periodic"), ("fhn", "zeroflux"), ("cenn", "zeroflux")])
def test_adjoint_depths_match_oracle(rd, oracle_mod, dtype, k, model):
    """The handle's tune k sets the recompute / reverse depth (one halo lane while k <= V, two
    above); every depth gives the oracle's adjoint (T not a multiple of k: ragged launches)."""
    reaction, boundary = model
    nn, nm, T = 40, 64, 27
    gene = CENN_ADJ if reaction == "cenn" else inp.default_params(Du=0.12, Dv=0.3)
    scale = 1.7 if reaction == "cenn" else 1.0
    x = scale * inp.uniform_field(91, nn, nm)
    y = inp.uniform_field(92, nn, nm)
    wu = inp.uniform_field(93, nn, nm) / (nn * nm)
    wv = inp.uniform_field(94, nn, nm) / (nn * nm)
    if dtype == F32:
        x, y, wu, wv = f32(x), f32(y), f32(wu), f32(wv)
    g = rd.Grid(nn, nm, gene, dtype=dtype, reaction=reaction, boundary=boundary)
    g.set_tune(k=k)
    du, dv, gp = g.adjoint(T, _dev(x, dtype), _dev(y, dtype), _dev(wu, dtype), _dev(wv, dtype), 3)
    torch.cuda.synchronize()
    rx = oracle_mod.CENN if reaction == "cenn" else oracle_mod.FHN
    bc = oracle_mod.ZEROFLUX if boundary == "zeroflux" else oracle_mod.PERIODIC
    ou, ov, og = oracle_mod.adjoint(x, y, gene, T, wu, wv, n_checkpoints=3, reaction=rx, boundary=bc)
    tol, gtol = (1e-10, 1e-9) if dtype == F64 else (1e-5, 1e-5)
    assert normwise(du.double().cpu().numpy(), ou) <= tol and normwise(dv.double().cpu().numpy(), ov) <= tol
    got = np.array([gp[n] for n in NAMES])
    np.testing.assert_allclose(got, og, rtol=gtol, atol=gtol * np.linalg.norm(og))


# ---------------------------------------------------------------------------- recorded forward (tape)

TAPE_MODELS = [("fhn", "periodic"), ("fhn", "zeroflux"), ("cenn", "periodic")]


def _tape_grid(rd, reaction, boundary, dtype, nn=40, nm=64):
    gene = CENN_ADJ if reaction == "cenn" else inp.default_params(Du=0.12, Dv=0.3)
    return rd.Grid(nn, nm, gene, dtype=dtype, reaction=reaction, boundary=boundary), gene


@pytest.mark.parametrize("dtype", [F32, F64], ids=["f32", "f64"])
@pytest.mark.parametrize("nck", [0, 4, 31], ids=["sqrtT", "nck4", "all"])
def test_run_record_is_run_and_tape_holds_the_states(rd, dtype, nck):
    """rdcnn_run_record leaves the bits rdcnn_run leaves, and tape slot i holds the state at
    step i*S of that run (S = ceil(T / n)); n >= T keeps every state."""
    nn, nm, T = 40, 64, 31
    x = inp.uniform_field(51, nn, nm)
    y = inp.uniform_field(52, nn, nm)
    if dtype == F32:
        x, y = f32(x), f32(y)
    g, gene = _tape_grid(rd, "fhn", "periodic", dtype, nn, nm)
    g.set_state(_dev(x, dtype), _dev(y, dtype))
    tape = g.run_record(T, nck)
    torch.cuda.synchronize()
    n = int(np.ceil(np.sqrt(T))) if nck == 0 else min(nck, T)
    S = -(-T // n)
    nseg = -(-T // S)
    esz = 4 if dtype == F32 else 8
    plane = -(-(nn * nm * esz) // 256) * 256
    assert tape.numel() >= nseg * 2 * plane
    ref_u, ref_v = gpu_run(rd, x, y, gene, T, dtype)
    assert np.array_equal(g.u.double().cpu().numpy(), ref_u) and np.array_equal(g.v.double().cpu().numpy(), ref_v)
    raw = tape.view(torch.uint8)
    for i in sorted({0, 1, nseg // 2, nseg - 1}):
        su = raw[2 * i * plane:2 * i * plane + nn * nm * esz].view(dtype).reshape(nn, nm)
        sv = raw[(2 * i + 1) * plane:(2 * i + 1) * plane + nn * nm * esz].view(dtype).reshape(nn, nm)
        eu, ev = gpu_run(rd, x, y, gene, i * S, dtype)
        assert np.array_equal(su.double().cpu().numpy(), eu) and np.array_equal(sv.double().cpu().numpy(), ev), i


@pytest.mark.parametrize("dtype", [F32, F64], ids=["f32", "f64"])
@pytest.mark.parametrize("nck", [0, 5, 27], ids=["sqrtT", "nck5", "all"])
@pytest.mark.parametrize("model", TAPE_MODELS, ids=["fhn-torus", "fhn-zeroflux", "cenn-torus"])
def test_adjoint_tape_equals_adjoint(rd, oracle_mod, dtype, nck, model):
    """The adjoint from a recorded tape gives rdcnn_adjoint's bits (same checkpoints, same
    launch sequence of the reverse sweep), and the oracle's adjoint within the parity bar."""
    reaction, boundary = model
    nn, nm, T = 40, 64, 27
    scale = 1.7 if reaction == "cenn" else 1.0
    x = scale * inp.uniform_field(61, nn, nm)
    y = inp.uniform_field(62, nn, nm)
    wu = inp.uniform_field(63, nn, nm) / (nn * nm)
    wv = inp.uniform_field(64, nn, nm) / (nn * nm)
    if dtype == F32:
        x, y, wu, wv = f32(x), f32(y), f32(wu), f32(wv)
    g, gene = _tape_grid(rd, reaction, boundary, dtype, nn, nm)
    du, dv, gp = g.adjoint(T, _dev(x, dtype), _dev(y, dtype), _dev(wu, dtype), _dev(wv, dtype), nck)
    g.set_state(_dev(x, dtype), _dev(y, dtype))
    tape = g.run_record(T, nck)
    tu, tv, tp = g.adjoint_tape(T, tape, _dev(wu, dtype), _dev(wv, dtype), nck)
    torch.cuda.synchronize()
    assert torch.equal(du, tu) and torch.equal(dv, tv)
    assert all(gp[k] == tp[k] for k in NAMES), (gp, tp)
    rx = oracle_mod.CENN if reaction == "cenn" else oracle_mod.FHN
    bc = oracle_mod.ZEROFLUX if boundary == "zeroflux" else oracle_mod.PERIODIC
    ou, ov, og = oracle_mod.adjoint(x, y, gene, T, wu, wv, n_checkpoints=nck, reaction=rx, boundary=bc)
    tol, gtol = (1e-10, 1e-9) if dtype == F64 else (1e-5, 1e-5)
    assert normwise(tu.double().cpu().numpy(), ou) <= tol and normwise(tv.double().cpu().numpy(), ov) <= tol
    got = np.array([tp[n] for n in NAMES])
    np.testing.assert_allclose(got, og, rtol=gtol, atol=gtol * np.linalg.norm(og))


def test_adjoint_tape_full_size_f32(rd, oracle_mod):
    """The benchmark's adjoint workload (512^2, T = 2000) from a full tape (every state kept,
    nothing rebuilt) against the sqrt(T)-checkpoint adjoint: the same co-state bits."""
    N, T = 512, 2000
    p = inp.default_params()
    x = _dev(f32(inp.uniform_field(0, N, N)), F32)
    target = _dev(inp.checkerboard(0, N, N), F32)
    g = rd.Grid(N, N, p, dtype=F32)
    g.set_state(x, x)
    tape = g.run_record(T, T)
    gu = (2.0 * (g.u - target) / g.u.numel()).contiguous()
    du, dv, gp = g.adjoint_tape(T, tape, gu, torch.zeros_like(gu), T)
    del tape
    ru, rv, rp = g.adjoint(T, x, x, gu, torch.zeros_like(gu))
    torch.cuda.synchronize()
    assert torch.equal(du, ru) and torch.equal(dv, rv)
    a = np.array([gp[k] for k in NAMES])
    b = np.array([rp[k] for k in NAMES])
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)


@pytest.mark.parametrize("T", [0, 1, 2, 3, 9])
@pytest.mark.parametrize("nck", [0, 1, 100], ids=["sqrtT", "one", "all"])
def test_tape_short_horizons(rd, T, nck):
    """Horizons of 0 .. 9 steps through the recorded forward and the tape adjoint: the same
    bits as rdcnn_run and rdcnn_adjoint (T = 0 leaves the state and passes the co-state
    through with a zero gene gradient)."""
    nn, nm = 16, 32
    x = inp.uniform_field(81, nn, nm)
    y = inp.uniform_field(82, nn, nm)
    wu = inp.uniform_field(83, nn, nm)
    wv = inp.uniform_field(84, nn, nm)
    params = inp.default_params(Du=0.11, Dv=0.37)
    g = rd.Grid(nn, nm, params, dtype=F64)
    g.set_state(_dev(x, F64), _dev(y, F64))
    tape = g.run_record(T, nck)
    ru, rv = gpu_run(rd, x, y, params, T, F64)
    assert np.array_equal(g.u.cpu().numpy(), ru) and np.array_equal(g.v.cpu().numpy(), rv)
    du, dv, gp = g.adjoint_tape(T, tape, _dev(wu, F64), _dev(wv, F64), nck)
    eu, ev, ep = g.adjoint(T, _dev(x, F64), _dev(y, F64), _dev(wu, F64), _dev(wv, F64), nck)
    torch.cuda.synchronize()
    assert torch.equal(du, eu) and torch.equal(dv, ev)
    assert all(gp[k] == ep[k] for k in NAMES)
    if T == 0:
        assert np.array_equal(du.cpu().numpy(), wu) and all(gp[k] == 0.0 for k in NAMES)
