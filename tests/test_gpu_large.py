"""A grid past 2^31 cells (49152 x 49152 FP32, ~48 GB on the device with the
input): plane offsets beyond 32-bit range.  The input is drawn on the device
from a seeded generator; light-cone windows (a cell after T steps depends
only on cells within T of it) are read back and run by the oracle, at the
first and the last cells of the grid, where the offsets are largest.
Device memory: the input and four planes, 5 x 9.7 GB."""
import numpy as np
import pytest
import torch

import rdcnn_inputs as inp
from _util import normwise

pytestmark = pytest.mark.gpu

N = 49152  # N * N = 2 415 919 104 > 2^31
W, T = 48, 8


def test_grid_past_2_31_cells(rd, oracle_mod):
    gen = torch.Generator(device="cuda")
    gen.manual_seed(20210219)
    x = torch.rand((N, N), generator=gen, device="cuda", dtype=torch.float32).mul_(2.0).sub_(1.0)
    corners = [(0, 0), (N - W, N - W), (N // 2 - W // 2, 7 * N // 8)]
    xw = [x[r:r + W, c:c + W].double().cpu().numpy() for r, c in corners]
    params = inp.default_params()
    g = rd.Grid(N, N, params, dtype=torch.float32)
    for variant, k in (("temporal", 8), ("step1", 0)):
        g.init(x, 1.0)  # u = v = x
        g.run(T, variant=variant, k=k)
        torch.cuda.synchronize()
        for (r, c), xin in zip(corners, xw):
            ru, rv = oracle_mod.run(xin, xin, params, T)
            gu = g.u[r + T:r + W - T, c + T:c + W - T].double().cpu().numpy()
            gv = g.v[r + T:r + W - T, c + T:c + W - T].double().cpu().numpy()
            assert normwise(gu, ru[T:W - T, T:W - T]) <= 1e-5, (variant, r, c)
            assert normwise(gv, rv[T:W - T, T:W - T]) <= 1e-5, (variant, r, c)
    g.close()
