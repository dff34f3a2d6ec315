"""Small helpers shared by the GPU tests (no method arithmetic here)."""
import os

import numpy as np


def normwise(got, ref) -> float:
    """||got - ref||_2 / ||ref||_2 (the relative error measure used by the parity tests)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def cpu_threads() -> int:
    return max(1, os.cpu_count() or 1)


def gpu_run(rd, u0, v0, params, T, dtype, variant="auto", k=0, reaction="fhn", rows=0,
            boundary="periodic"):
    """Run T steps on the GPU through the C ABI; returns float64 numpy (u_T, v_T)."""
    import torch

    u0 = np.asarray(u0)
    g = rd.Grid(u0.shape[0], u0.shape[1], params, dtype=dtype, reaction=reaction, boundary=boundary)
    if rows:
        g.set_tune(k=k, rows=rows)
    g.set_state(torch.from_numpy(np.ascontiguousarray(u0)).to("cuda", dtype),
                torch.from_numpy(np.ascontiguousarray(v0)).to("cuda", dtype))
    g.run(T, variant=variant, k=k)
    u, v = g.state()
    torch.cuda.synchronize()
    out = u.double().cpu().numpy(), v.double().cpu().numpy()
    g.close()
    return out


def f32(a):
    """Round once to float32 and return as float64 (the values both sides start from)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)
