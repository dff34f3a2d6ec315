"""Labelling rules of the parameter search (host logic, no GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _traj(edges, var_last=0.1):
    t = np.zeros((len(edges), 8))
    t[:, 7] = edges
    t[:, 1] = 0.1
    t[-1, 1] = var_last
    return t


def test_classify_rules():
    from paper_2102_10340_gb300 import search

    trajs = np.stack([_traj([0.01, 0.02, 0.05, 0.08]),        # grows, stays small -> slow growth
                      _traj([0.30, 0.55, 0.60, 0.62]),        # fills the grid -> patterns
                      _traj([0.02, 0.01, 0.0, 0.0], 1e-9),    # fades to uniform -> dull
                      _traj([0.05, 0.05, 0.05, 0.05])])       # neither -> static
    assert search.classify(trajs) == ["slow growth", "patterns", "dull", "static"]


def test_du_dv_grid():
    from paper_2102_10340_gb300 import search

    g = search.du_dv_grid([0.3, 0.5], [0.8, 1.0])
    assert [(x["Du"], x["Dv"]) for x in g] == [(0.3, 0.8), (0.3, 1.0), (0.5, 0.8), (0.5, 1.0)]
    assert all(x["a"] == -0.3 and x["dt"] == 0.1 for x in g)


def test_ab_grid():
    from paper_2102_10340_gb300 import search

    g = search.ab_grid([-0.3, 0.0], [1.0, 1.3], base={"dt": 0.05, "a": 9.0, "b": 9.0, "eps": -0.1, "c": 1.0,
                                                      "Du": 0.06, "Dv": 1.0})
    assert [(x["a"], x["b"]) for x in g] == [(-0.3, 1.0), (-0.3, 1.3), (0.0, 1.0), (0.0, 1.3)]
    assert all(x["dt"] == 0.05 and x["Du"] == 0.06 for x in g)
