"""Parameter-space search over the gene, the use the paper makes of a fast
simulator in Sec. III: sweep the (Du, Dv) plane to find slow growth, dynamic
patterns or dull homogeneous states (Sec. III.A), or the (a, b) plane for
image-processing behaviour (Sec. III.B).

All candidate genes run together as one :class:`Batch` (one launch per k
steps for every instance); at each checkpoint the on-device statistics of
``rdcnn_batch_summary`` are taken (8 numbers per instance, no grid leaves the
GPU).  Each run is then labelled from its statistics:

* ``dull``        -- homogeneous at the end: var(u) <= ``flat``;
* ``patterns``    -- the gradient-active area covers at least ``full`` of the grid;
* ``slow growth`` -- the active area grew by at least ``growth`` x between the
  first and last checkpoint but stays below ``full``;
* ``static``      -- anything else (structure that neither spreads nor fades).

The paper sorts these behaviours by eye from plots; the labels here are
heuristics over measured numbers, documented so they can be re-tuned.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rdcnn as rd

EDGE = rd.SUMMARY_FIELDS.index("edge_frac")
VAR_U = rd.SUMMARY_FIELDS.index("var_u")


def classify(traj: np.ndarray, flat: float = 1e-6, full: float = 0.5, growth: float = 1.5) -> list:
    """Label runs from statistics trajectories of shape (n, checkpoints, 8)."""
    traj = np.asarray(traj)
    labels = []
    for t in traj:
        first, last = t[0], t[-1]
        if last[VAR_U] <= flat:
            labels.append("dull")
        elif last[EDGE] >= full:
            labels.append("patterns")
        elif last[EDGE] >= growth * max(first[EDGE], 1e-12):
            labels.append("slow growth")
        else:
            labels.append("static")
    return labels


def sweep(genes, N: int = 256, T: int = 2000, init: str = "patch", checkpoints: int = 4, seed: int = 0,
          dtype=torch.float32, threshold: float = 0.05, tune: dict | None = None, device="cuda",
          reaction: str = "fhn", boundary: str = "periodic"):
    """Run every gene in ``genes`` (list of dicts) on an N x N grid for T steps (torus, or zero
    flux with ``boundary="zeroflux"``; ``reaction="cenn"`` sweeps Chua-Yang cells, whose
    offset plane v starts equal to the input like u).

    init: "patch" (16 x 16 U[-1, 1] square in the middle, the paper's typ=1 shape) or
    "random" (all cells U[-1, 1], typ=2), drawn from ``seed`` (same start for every gene).
    Returns {"genes", "times", "stats" (n, checkpoints + 1, 8), "labels"}.
    """
    import rdcnn_inputs as inp

    if init == "patch":
        x = inp.mid_patch(seed, N, N, patch=min(16, N))
    elif init == "random":
        x = inp.uniform_field(seed, N, N)
    else:
        raise ValueError("init must be 'patch' or 'random'")
    xt = torch.from_numpy(np.asarray(x)).to(dtype)
    batch = rd.Batch([{"nn": N, "nm": N, "params": g} for g in genes], dtype=dtype, device=device,
                     reaction=reaction, boundary=boundary)
    for i in range(len(genes)):
        batch.set_state(i, xt, xt)
    if tune:
        batch.set_tune(**tune)
    cuts = np.linspace(0, T, checkpoints + 1).round().astype(int)
    stats = [batch.summary(threshold).numpy()]
    for a, b in zip(cuts[:-1], cuts[1:]):
        if b > a:
            batch.run(int(b - a))
        stats.append(batch.summary(threshold).numpy())
    traj = np.stack(stats, axis=1)
    return {"genes": list(genes), "times": cuts.tolist(), "stats": traj, "labels": classify(traj[:, 1:])}


def du_dv_grid(du_values, dv_values, base: dict | None = None) -> list:
    """Genes on a (Du, Dv) grid around ``base`` (default: the paper's defaults)."""
    base = dict(base or rd.DEFAULT_PARAMS)
    return [dict(base, Du=float(du), Dv=float(dv)) for du in du_values for dv in dv_values]


def ab_grid(a_values, b_values, base: dict | None = None) -> list:
    """Genes on an (a, b) grid around ``base``: the plane Sec. III.B searches for
    image-processing (edge-detecting) behaviour."""
    base = dict(base or rd.DEFAULT_PARAMS)
    return [dict(base, a=float(a), b=float(b)) for a in a_values for b in b_values]
