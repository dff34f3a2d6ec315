"""Out-of-bounds detection without a sanitizer: every buffer the library touches
is carved out of one device arena whose gaps (guard bands, 4 KiB each) hold a
fixed byte pattern (0xFF: a NaN in every floating format).  After each run the
guard bands must be unchanged (no stray write), and the results must equal the
same run on ordinary torch buffers bit for bit (a stray read of a guard value
would have put a NaN into them).  Ragged grid sizes, every forward variant,
both boundaries, every dtype, the batched sweep and the adjoint."""
import ctypes

import numpy as np
import pytest
import torch

import rdcnn_inputs as inp
from _util import f32

pytestmark = pytest.mark.gpu

GUARD = 4096
FILL = 0xFF
DT = {torch.float32: 0, torch.float64: 1, torch.bfloat16: 2, torch.float16: 3}
VARIANT = {"auto": 0, "step1": 1, "temporal": 2, "generic": 3, "temporal2": 4, "temporal_wide": 5}


class Arena:
    """One device byte buffer; take() hands out 256-byte aligned regions separated by guards."""

    def __init__(self, sizes):
        total = GUARD
        self.offs = []
        for n in sizes:
            self.offs.append(total)
            total += (n + 255) // 256 * 256 + GUARD
        self.buf = torch.full((total,), FILL, dtype=torch.uint8, device="cuda")
        self.sizes = list(sizes)

    def ptr(self, i):
        return self.buf.data_ptr() + self.offs[i]

    def view(self, i, shape, dtype):
        n = int(np.prod(shape)) * torch.tensor([], dtype=dtype).element_size()
        return self.buf[self.offs[i]:self.offs[i] + n].view(dtype).view(*shape)

    def guards_intact(self):
        mask = torch.ones_like(self.buf, dtype=torch.bool)
        for o, n in zip(self.offs, self.sizes):
            mask[o:o + n] = False
        return bool((self.buf[mask] == FILL).all().item())


@pytest.fixture(scope="module")
def L():
    from paper_2102_10340_gb300 import _lib

    return _lib


def _handle(L, nn, nm, params, dtype, reaction, boundary):
    lib = L.load()
    h = ctypes.c_void_p()
    ps = L.params_struct(params)
    rc = lib.rdcnn_create(ctypes.byref(h), nn, nm, ctypes.byref(ps), boundary, DT[dtype], reaction)
    assert rc >= 0, L.last_error()
    return lib, h


SHAPES = [(37, 68), (5, 8), (1, 4), (129, 260), (66, 32)]
CASES = [(torch.float32, "temporal", 8), (torch.float32, "temporal", 3), (torch.float32, "step1", 0),
         (torch.float32, "generic", 0), (torch.float32, "temporal2", 5), (torch.float32, "temporal_wide", 4),
         (torch.float64, "temporal", 4), (torch.float64, "temporal2", 2), (torch.float64, "step1", 0),
         (torch.bfloat16, "temporal", 8), (torch.bfloat16, "step1", 0), (torch.float16, "temporal", 2)]


@pytest.mark.parametrize("boundary", [0, 1], ids=["torus", "zeroflux"])
@pytest.mark.parametrize("dtype,variant,k", CASES, ids=[f"{str(d)[6:]}-{v}{k}" for d, v, k in CASES])
def test_forward_variants_stay_in_bounds(L, dtype, variant, k, boundary):
    from paper_2102_10340_gb300 import rdcnn as rd

    params = inp.default_params()
    T = 23
    for nn, nm in SHAPES:
        if variant == "temporal_wide" and nm % 8:
            continue
        vec = 2 if dtype == torch.float64 else 4
        if variant != "generic" and nm % vec:
            continue
        x = torch.from_numpy(inp.uniform_field(nn + nm, nn, nm)).to("cuda", dtype)
        lib, h = _handle(L, nn, nm, params, dtype, 0, boundary)
        wsb = ctypes.c_size_t()
        assert lib.rdcnn_workspace_bytes(h, ctypes.byref(wsb)) == 0
        esz = x.element_size()
        ar = Arena([nn * nm * esz, nn * nm * esz, wsb.value])
        u, v = ar.view(0, (nn, nm), dtype), ar.view(1, (nn, nm), dtype)
        u.copy_(x)
        v.copy_(0.5 * x)
        assert lib.rdcnn_bind(h, ctypes.c_void_p(ar.ptr(0)), ctypes.c_void_p(ar.ptr(1)),
                              ctypes.c_void_p(ar.ptr(2)), wsb.value, None) == 0
        rc = lib.rdcnn_run(h, T, VARIANT[variant], k)
        torch.cuda.synchronize()
        lib.rdcnn_destroy(h)
        assert rc == 0, (nn, nm, L.last_error())
        assert ar.guards_intact(), (nn, nm)
        ref = rd.Grid(nn, nm, params, dtype=dtype, boundary="zeroflux" if boundary else "periodic")
        ref.set_state(x, 0.5 * x)
        ref.run(T, variant=variant, k=k)
        ru, rv = ref.state()
        torch.cuda.synchronize()
        assert torch.equal(u, ru) and torch.equal(v, rv), (nn, nm)
        ref.close()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64, torch.bfloat16], ids=["f32", "f64", "bf16"])
def test_batched_sweep_stays_in_bounds(L, dtype):
    from paper_2102_10340_gb300 import rdcnn as rd

    shapes = [(37, 64), (5, 8), (1, 4), (130, 132)]
    esz = torch.tensor([], dtype=dtype).element_size()
    sizes = []
    for nn, nm in shapes:
        sizes += [nn * nm * esz] * 4
    tab_bytes = ctypes.c_size_t()
    lib = L.load()
    inst = (L.Instance * len(shapes))()
    genes = [inp.default_params(Du=0.1 + 0.02 * i) for i in range(len(shapes))]
    for i, (nn, nm) in enumerate(shapes):
        inst[i] = L.Instance(nn, nm, L.params_struct(genes[i]), 0, 0, 0, 0)
    assert lib.rdcnn_batch_workspace_bytes(inst, len(shapes), DT[dtype], None, ctypes.byref(tab_bytes)) == 0
    ar = Arena(sizes + [tab_bytes.value])
    ref = rd.Batch([{"nn": a, "nm": b, "params": genes[i]} for i, (a, b) in enumerate(shapes)], dtype=dtype,
                   boundary="zeroflux")
    for i, (nn, nm) in enumerate(shapes):
        x = torch.from_numpy(inp.uniform_field(300 + i, nn, nm)).to("cuda", dtype)
        ar.view(4 * i, (nn, nm), dtype).copy_(x)
        ar.view(4 * i + 1, (nn, nm), dtype).copy_(x)
        ref.set_state(i, x, x)
        inst[i] = L.Instance(nn, nm, L.params_struct(genes[i]), ar.ptr(4 * i), ar.ptr(4 * i + 1),
                             ar.ptr(4 * i + 2), ar.ptr(4 * i + 3))
    tune = L.Tune(3, 0)
    rc = lib.rdcnn_batch_run_model(inst, len(shapes), 17, DT[dtype], 0, 1, ctypes.byref(tune),
                                   ctypes.c_void_p(ar.ptr(4 * len(shapes))), tab_bytes.value, None)
    torch.cuda.synchronize()
    assert rc == 0, L.last_error()
    assert ar.guards_intact()
    ref.set_tune(k=3)
    ref.run(17)
    torch.cuda.synchronize()
    for i, (nn, nm) in enumerate(shapes):
        assert torch.equal(ar.view(4 * i, (nn, nm), dtype), ref.state(i)[0]), i
        assert torch.equal(ar.view(4 * i + 1, (nn, nm), dtype), ref.state(i)[1]), i


@pytest.mark.parametrize("reaction,boundary", [(0, 0), (0, 1), (2, 1)], ids=["fhn-torus", "fhn-zf", "cenn-zf"])
def test_adjoint_stays_in_bounds(L, reaction, boundary):
    from paper_2102_10340_gb300 import rdcnn as rd

    nn, nm, T = 33, 68, 29
    gene = ({"dt": 0.1, "a": 0.0, "b": 0.0, "eps": 0.0, "c": 1.3, "Du": -0.2, "Dv": 0.0} if reaction == 2
            else inp.default_params())
    lib, h = _handle(L, nn, nm, gene, torch.float32, reaction, boundary)
    wsb = ctypes.c_size_t()
    assert lib.rdcnn_adjoint_workspace_bytes(h, T, 4, ctypes.byref(wsb)) == 0
    pb = nn * nm * 4
    ar = Arena([pb] * 6 + [wsb.value])
    planes = [ar.view(i, (nn, nm), torch.float32) for i in range(6)]
    for i in range(4):
        planes[i].copy_(torch.from_numpy(f32(inp.uniform_field(400 + i, nn, nm))).cuda())
    g = (ctypes.c_double * 6)()
    rc = lib.rdcnn_adjoint(h, T, *[ctypes.c_void_p(ar.ptr(i)) for i in range(4)], 4, ctypes.c_void_p(ar.ptr(4)),
                           ctypes.c_void_p(ar.ptr(5)), g, ctypes.c_void_p(ar.ptr(6)), wsb.value)
    torch.cuda.synchronize()
    lib.rdcnn_destroy(h)
    assert rc == 0, L.last_error()
    assert ar.guards_intact()
    ref = rd.Grid(nn, nm, gene, dtype=torch.float32, reaction=["fhn", "none", "cenn"][reaction],
                  boundary="zeroflux" if boundary else "periodic")
    du, dv, gp = ref.adjoint(T, *[p.clone() for p in planes[:4]], 4)
    torch.cuda.synchronize()
    assert torch.equal(planes[4], du) and torch.equal(planes[5], dv)
    names = ("Du", "Dv", "a", "b", "eps", "c")
    assert [g[i] for i in range(6)] == [gp[n] for n in names]
