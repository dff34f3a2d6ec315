"""Programmatic dependent launch changes only when a kernel is scheduled, never
what it computes: the same runs in a process with RDCNN_PDL=0 (plain launches)
give the same bits, for the single-grid variants (plain and graph-replayed),
the batched sweep and the adjoint."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SCRIPT = r"""
import sys
import numpy as np
import torch
import rdcnn_inputs as inp
from paper_2102_10340_gb300 import rdcnn as rd

out = {}
x = inp.uniform_field(5, 96, 128)
for variant, k, T in (("temporal", 8, 37), ("temporal", 3, 3 * 64 * 3 + 2), ("step1", 0, 150),
                      ("generic", 0, 9), ("temporal2", 4, 21), ("temporal_wide", 4, 22)):
    g = rd.Grid(96, 128, None)
    xt = torch.from_numpy(x).float().cuda()
    g.set_state(xt, 0.5 * xt)
    g.run(T, variant=variant, k=k)
    u, v = g.state()
    out[f"{variant}{k}_u"] = u.cpu().numpy()
    out[f"{variant}{k}_v"] = v.cpu().numpy()
    g.close()
specs = [{"nn": 40, "nm": 64, "params": inp.default_params(Du=0.2)},
         {"nn": 128, "nm": 132, "params": inp.default_params(a=0.1)}]
b = rd.Batch(specs, dtype=torch.float32, boundary="zeroflux")
for i, s in enumerate(specs):
    y = torch.from_numpy(inp.uniform_field(20 + i, s["nn"], s["nm"])).float()
    b.set_state(i, y, y)
b.set_tune(k=4)
b.run(45)
for i in range(len(specs)):
    out[f"batch{i}_u"] = b.state(i)[0].cpu().numpy()
g = rd.Grid(64, 64, None, dtype=torch.float32)
z = torch.from_numpy(inp.uniform_field(30, 64, 64)).float().cuda()
du, dv, gp = g.adjoint(40, z, z, z / 4096, 0 * z)
out["adj_du"] = du.cpu().numpy()
out["adj_g"] = np.array([gp[k] for k in ("Du", "Dv", "a", "b", "eps", "c")])
np.savez(sys.argv[1], **out)
"""


def _run(tmp_path, pdl: str):
    path = str(tmp_path / f"pdl{pdl}.npz")
    env = dict(os.environ, RDCNN_PDL=pdl,
               PYTHONPATH=os.pathsep.join([ROOT, HERE, os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, "-c", SCRIPT, path], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(path)


def test_pdl_and_plain_launches_give_the_same_bits(tmp_path):
    a = _run(tmp_path, "1")
    b = _run(tmp_path, "0")
    assert sorted(a.files) == sorted(b.files)
    for name in a.files:
        assert np.array_equal(a[name], b[name]), name
