"""Seeded synthetic inputs for the RD-CNN workloads.

This module is shared by the CPU oracle (``oracle/``), the tests and the
benchmark.  It holds none of the method's arithmetic: it only draws the
initial images x, the loss targets and the per-instance genes of a sweep.
All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64) in
float64; callers that run in FP32 round the result once and hand the SAME
rounded values to both the GPU path and the oracle.

Workload recipes (sizes and distributions of the paper's experiments):

* ``uniform_field``  -- fully random initial state, x ~ U[-1, 1]
  (Sec. II.A, "typ=2": all cells random).
* ``mid_patch``      -- zero field with a random square in the middle
  (Sec. II.A, "typ=1"; 16 x 16 for the 4096^2 slow-growth workload, 11 x 11
  is the paper's own size).
* ``smooth_noise``   -- stand-in for the paper's test image (Sec. II.A,
  "typ=3"; the image file itself is not available): U[0, 1] blurred with a
  periodic Gaussian of sigma = 8 px, then min-max rescaled to [-1, 1].
* ``checkerboard``   -- +/-1 target of period 32 px with seeded offsets, the
  loss target for the adjoint workload.
* ``sweep_instances``-- genes of a (Du, Dv) / FHN-coefficient sweep in the
  spirit of Sec. III.A (per-instance grid size and parameters).
"""
from __future__ import annotations

import numpy as np

# Sec. II.A, get_init_state() defaults: a=-0.3, b=1.3, eps=-0.1, c=1, Du=0.06, Dv=1, dt=0.1, ka=1
DEFAULT_GENE = {"dt": 0.1, "a": -0.3, "b": 1.3, "eps": -0.1, "c": 1.0, "Du": 0.06, "Dv": 1.0}
DEFAULT_KA = 1.0


def default_params(**overrides) -> dict:
    p = dict(DEFAULT_GENE)
    p.update(overrides)
    return p


def uniform_field(seed: int, nn: int, nm: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(nn, nm))


def mid_patch(seed: int, nn: int, nm: int, patch: int = 16) -> np.ndarray:
    """Zeros with a patch x patch block of U[-1, 1] at rows/cols [N/2 - patch/2, N/2 + patch/2)."""
    x = np.zeros((nn, nm))
    rng = np.random.default_rng(seed)
    block = rng.uniform(-1.0, 1.0, size=(patch, patch))
    r0 = nn // 2 - patch // 2
    c0 = nm // 2 - patch // 2
    rr = (np.arange(patch) + r0) % nn
    cc = (np.arange(patch) + c0) % nm
    x[np.ix_(rr, cc)] = block
    return x


def patch_origin(nn: int, nm: int, patch: int = 16):
    return nn // 2 - patch // 2, nm // 2 - patch // 2


def smooth_noise(seed: int, nn: int, nm: int, sigma: float = 8.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.0, 1.0, size=(nn, nm))
    ky = np.fft.fftfreq(nn)[:, None]
    kx = np.fft.fftfreq(nm)[None, :]
    gain = np.exp(-2.0 * (np.pi * sigma) ** 2 * (kx * kx + ky * ky))
    blurred = np.real(np.fft.ifft2(np.fft.fft2(w) * gain))
    lo, hi = blurred.min(), blurred.max()
    if hi <= lo:
        return np.zeros((nn, nm))
    return 2.0 * (blurred - lo) / (hi - lo) - 1.0


def checkerboard(seed: int, nn: int, nm: int, period: int = 32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    p, q = rng.integers(0, period, size=2)
    half = period // 2
    i = (np.arange(nn)[:, None] + p) // half
    j = (np.arange(nm)[None, :] + q) // half
    return np.where((i + j) % 2 == 0, 1.0, -1.0)


def fourier_mode(nn: int, nm: int, p: int, q: int) -> np.ndarray:
    i = np.arange(nn)[:, None]
    j = np.arange(nm)[None, :]
    return np.cos(2.0 * np.pi * (p * i / nn + q * j / nm))


def sweep_instances(seed: int = 0, n: int = 256, sizes=(128, 256, 512, 1024), dt: float = 0.1,
                    jitter: float = 0.2):
    """Per-instance grid sizes and genes for a batched parameter sweep.

    Grid side N_i uniform over ``sizes``; Du, Dv ~ U[0.01, 0.25]; a, b, eps, c
    each the default value times U[1 - jitter, 1 + jitter]; dt shared.  The
    initial image of instance i is ``uniform_field(seed + i, N_i, N_i)``.
    """
    rng = np.random.default_rng(seed)
    side = rng.choice(np.asarray(sizes), size=n)
    du = rng.uniform(0.01, 0.25, size=n)
    dv = rng.uniform(0.01, 0.25, size=n)
    scale = rng.uniform(1.0 - jitter, 1.0 + jitter, size=(n, 4))
    out = []
    g = DEFAULT_GENE
    for k in range(n):
        params = {"dt": dt, "a": g["a"] * scale[k, 0], "b": g["b"] * scale[k, 1],
                  "eps": g["eps"] * scale[k, 2], "c": g["c"] * scale[k, 3],
                  "Du": float(du[k]), "Dv": float(dv[k])}
        out.append({"nn": int(side[k]), "nm": int(side[k]), "params": params, "x_seed": seed + k})
    return out
