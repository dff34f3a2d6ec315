"""Graph replay inside rdcnn_run (launch-bound grids: cells x k <= 2^23 and at
least 64 full-depth launches): a run that replays captured launch groups must
give the bits of the same run split into calls too short to use a graph, the
launch counter must count the replayed kernels, and a changed gene, launch
shape or binding must not reuse a stale graph."""
import numpy as np
import pytest
import torch

import rdcnn_inputs as inp

pytestmark = pytest.mark.gpu


def _grid(rd, x, params, dtype=torch.float32, **kw):
    g = rd.Grid(x.shape[0], x.shape[1], params, dtype=dtype, **kw)
    xt = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)
    g.set_state(xt, 0.5 * xt)
    return g


@pytest.mark.parametrize("variant,k", [("step1", 0), ("temporal", 2), ("temporal", 4), ("generic", 0),
                                       ("temporal_wide", 3), ("temporal2", 4)])
def test_graph_run_equals_short_calls(rd, variant, k):
    x = inp.uniform_field(11, 96, 128)
    T = 3 * 64 * max(k, 1) + 5  # several graph groups plus a ragged tail
    a = _grid(rd, x, None)
    n0 = rd.launch_count()
    a.run(T, variant=variant, k=k)
    torch.cuda.synchronize()
    launches = rd.launch_count() - n0
    kk = max(k, 1)
    assert launches == -(-T // kk)  # one kernel per k steps, replayed or not
    b = _grid(rd, x, None)
    left = T
    while left > 0:  # calls of at most 60 launches never use a graph
        step = min(left, 60 * kk)
        b.run(step, variant=variant, k=k)
        left -= step
    assert torch.equal(a.u, b.u) and torch.equal(a.v, b.v)
    a.close(); b.close()


def test_graph_follows_gene_shape_and_model_changes(rd):
    x = inp.uniform_field(12, 64, 64)
    g = _grid(rd, x, None)
    g.run(400, variant="temporal", k=4)  # captures
    other = dict(inp.default_params(), Du=0.09, c=0.8)
    g.set_params(other)
    g.set_state(torch.from_numpy(x).cuda().float(), 0.5 * torch.from_numpy(x).cuda().float())
    g.run(400, variant="temporal", k=4)
    ref = _grid(rd, x, other)
    ref.run(400, variant="step1")
    assert torch.equal(g.u, ref.u) and torch.equal(g.v, ref.v)
    g.set_state(torch.from_numpy(x).cuda().float(), 0.5 * torch.from_numpy(x).cuda().float())
    g.run(400, variant="temporal", k=2)  # another depth: another graph
    assert torch.equal(g.u, ref.u) and torch.equal(g.v, ref.v)
    z = _grid(rd, x, None, boundary="zeroflux", dtype=torch.bfloat16)
    z.run(300, variant="step1")
    w = _grid(rd, x, None, boundary="zeroflux", dtype=torch.bfloat16)
    for _ in range(10):
        w.run(30, variant="step1")
    assert torch.equal(z.u, w.u) and torch.equal(z.v, w.v)
    for h in (g, ref, z, w):
        h.close()


@pytest.mark.parametrize("variant,k", [("temporal", 4), ("step1", 0), ("temporal2", 6)])
def test_run_captured_into_a_caller_graph(rd, variant, k):
    """rdcnn_run inside the caller's own stream capture (torch.cuda.graph): the library skips
    its graph replay, records its programmatically serialised launches into the caller's
    graph, and replaying that graph twice equals two direct runs, bit for bit."""
    x = inp.uniform_field(21, 96, 128)
    T = 3 * 64 * 4 + 6  # long enough for the library's own graph path outside a capture
    a = _grid(rd, x, None)
    a.run(8, variant=variant, k=k)  # warm-up outside the capture (module load, shape queries)
    xt = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", torch.float32)
    a.set_state(xt, 0.5 * xt)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        a.run(T, variant=variant, k=k)
    torch.cuda.synchronize()
    assert torch.equal(a.u, xt)  # capturing runs nothing
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    b = _grid(rd, x, None)
    b.run(T, variant=variant, k=k)
    b.run(T, variant=variant, k=k)
    torch.cuda.synchronize()
    assert torch.equal(a.u, b.u) and torch.equal(a.v, b.v)
