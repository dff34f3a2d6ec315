"""rdcnn_run_static: the entry point for callers that cannot allocate device memory.

Such callers (a plug-in inside a host that owns the whole device memory pool,
or a C/Fortran driver that only receives device pointers) cannot hand
rdcnn_bind a scratch workspace; rdcnn_run_static takes its ping-pong planes
from a fixed device array inside the library instead.  Here it is called
through the C ABI and compared with rdcnn_run (caller-provided workspace) on
two calls in a row that share that array.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

import rdcnn_inputs as inp
from _util import f32, gpu_run, normwise

pytestmark = pytest.mark.gpu

TOL = 1e-5  # FP32 normwise tolerance used by the forward parity tests


def test_run_static_matches_run_on_two_calls(rd):
    from paper_2102_10340_gb300 import _lib as L

    lib = rd.load()
    params = inp.default_params()
    ps = L.params_struct(params)
    for nn, nm, T, seed in ((512, 512, 37, 1), (300, 64, 20, 2)):
        x = f32(inp.uniform_field(seed, nn, nm))
        ref_u, ref_v = gpu_run(rd, x, x, params, T, torch.float32, "auto")
        u = torch.from_numpy(x).float().cuda().contiguous()
        v = torch.from_numpy(x).float().cuda().contiguous()
        stream = torch.cuda.current_stream().cuda_stream
        rc = lib.rdcnn_run_static(nn, nm, ctypes.byref(ps), L.F32, L.REACTION_FHN,
                                  ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                  T, 0, ctypes.c_void_p(stream))
        assert rc == L.OK, L.last_error()
        torch.cuda.synchronize()
        gu, gv = u.double().cpu().numpy(), v.double().cpu().numpy()
        assert np.all(np.isfinite(gu)) and np.all(np.isfinite(gv))
        assert normwise(gu, ref_u) <= TOL and normwise(gv, ref_v) <= TOL


def test_run_static_rejects_grid_beyond_its_scratch(rd):
    from paper_2102_10340_gb300 import _lib as L

    lib = rd.load()
    ps = L.params_struct(inp.default_params())
    # 2048 x 2048 FP32 needs 32 MiB of scratch, twice the fixed array; rejected before GPU work
    rc = lib.rdcnn_run_static(2048, 2048, ctypes.byref(ps), L.F32, L.REACTION_FHN,
                              ctypes.c_void_p(256), ctypes.c_void_p(512), 10, 0, None)
    assert rc == L.EINVAL
    assert "static scratch" in L.last_error()
