"""rdcnn_run_static: the entry point for callers that cannot allocate device memory.

Such callers (a plug-in inside a host that owns the whole device memory pool,
or a C/Fortran driver that only receives device pointers) cannot hand
rdcnn_bind a scratch workspace; rdcnn_run_static takes its ping-pong planes
from a fixed device array inside the library instead.  Here it is called
through the C ABI on two calls in a row that share that array, and each
result is compared bit for bit with rdcnn_run (caller-provided workspace, the
same kernels) and with the FP64 oracle within the forward parity tolerance.

The cases cover the vectorised temporal path (FP32 and FP64), the generic
path (NM not a multiple of 4, and planes that are not 16-byte aligned), odd
and even launch counts (an odd count ends in the array and is copied back),
and a grid whose plane is exactly the 8 MiB limit, which puts the second
plane at the very end of the array.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

import rdcnn_inputs as inp
from _util import cpu_threads, f32, gpu_run, normwise

pytestmark = pytest.mark.gpu

TOL = {torch.float32: 1e-5, torch.float64: 1e-12}  # forward parity bars against the oracle

# (nn, nm, dtype, T, k, offset in elements of the planes' start, launches)
CASES = [
    (512, 512, torch.float32, 37, 0, 0, "vector, odd"),
    (1024, 2048, torch.float32, 16, 8, 0, "vector, plane = 8 MiB, even"),
    (130, 66, torch.float32, 20, 0, 0, "generic (NM % 4 != 0), even"),
    (130, 66, torch.float32, 21, 0, 0, "generic, odd"),
    (96, 128, torch.float32, 13, 4, 1, "generic (unaligned planes), odd"),
    (256, 256, torch.float64, 31, 4, 0, "FP64 vector, even"),
    (200, 64, torch.float64, 9, 2, 0, "FP64 vector, odd"),
]


def _plane(x, dtype, offset):
    """A device plane holding x, starting `offset` elements into its allocation."""
    n = x.size
    buf = torch.zeros(n + offset, dtype=dtype, device="cuda")
    view = buf[offset:offset + n].view(x.shape)
    view.copy_(torch.from_numpy(x).to("cuda", dtype))
    return buf, view


def _run_static(L, lib, u, v, params, T, k):
    ps = L.params_struct(params)
    code = L.F32 if u.dtype == torch.float32 else L.F64
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.rdcnn_run_static(u.shape[0], u.shape[1], ctypes.byref(ps), code, L.REACTION_FHN,
                              ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                              T, k, ctypes.c_void_p(stream))
    assert rc == L.OK, L.last_error()


@pytest.mark.parametrize("nn,nm,dtype,T,k,offset,what", CASES, ids=[c[-1] for c in CASES])
def test_run_static_matches_run_and_oracle_on_two_calls(rd, oracle_mod, nn, nm, dtype, T, k, offset, what):
    from paper_2102_10340_gb300 import _lib as L

    lib = rd.load()
    params = inp.default_params()
    for call, seed in enumerate((11, 12)):  # two calls in a row share the static array
        x = inp.uniform_field(seed, nn, nm)
        x = f32(x) if dtype == torch.float32 else x
        ref_u, ref_v = gpu_run(rd, x, -x, params, T, dtype, "auto" if k == 0 else "temporal", k)
        bu, u = _plane(x, dtype, offset)
        bv, v = _plane(-x, dtype, offset)
        _run_static(L, lib, u, v, params, T, k)
        torch.cuda.synchronize()
        gu, gv = u.double().cpu().numpy(), v.double().cpu().numpy()
        assert np.array_equal(gu, ref_u) and np.array_equal(gv, ref_v), (what, call)
        ou, ov = oracle_mod.run(x, -x, params, T, nthreads=cpu_threads())
        assert normwise(gu, ou) <= TOL[dtype] and normwise(gv, ov) <= TOL[dtype], (what, call)
        # nothing outside the planes was written
        if offset:
            assert float(bu[0]) == 0.0 and float(bv[0]) == 0.0


def test_run_static_limit_is_exactly_half_the_array(rd):
    from paper_2102_10340_gb300 import _lib as L

    lib = rd.load()
    ps = L.params_struct(inp.default_params())
    # one FP32 cell past 8 MiB per plane: rejected on the host before any GPU work
    rc = lib.rdcnn_run_static(1, (8 << 20) // 4 + 1, ctypes.byref(ps), L.F32, L.REACTION_FHN,
                              ctypes.c_void_p(256), ctypes.c_void_p(512), 10, 0, None)
    assert rc == L.EINVAL and "static scratch" in L.last_error()
    # 2048 x 2048 FP32 needs 32 MiB of scratch, twice the fixed array
    rc = lib.rdcnn_run_static(2048, 2048, ctypes.byref(ps), L.F32, L.REACTION_FHN,
                              ctypes.c_void_p(256), ctypes.c_void_p(512), 10, 0, None)
    assert rc == L.EINVAL and "static scratch" in L.last_error()
