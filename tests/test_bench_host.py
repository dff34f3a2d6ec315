"""Host-side logic of bench.py that needs no GPU: the multi-rank timing
reduction (max over ranks, under gloo with world size 2), the weak-scaling
throughput formula, and the reference arm's rank behaviour."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 150.0][rank]
        out[rank] = bench.max_over_ranks(local_ms, world)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        assert out[0] == 150.0 and out[1] == 150.0


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_replica_throughput_is_weak_scaling_aggregate():
    import bench

    one = bench.replica_throughput(4096 * 4096, 1000, 3, 1, 1.5)
    two = bench.replica_throughput(4096 * 4096, 1000, 3, 2, 1.5)
    assert two == pytest.approx(2 * one)
    assert one == pytest.approx(4096 * 4096 * 3000 / 1.5 / 1e9)


def test_reference_arm_nonzero_rank_exits_without_work(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_contract_line(monkeypatch, capsys):
    import json

    import bench

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0", "--grid", "64", "--T", "50"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "config", "cpu_baseline", "e2e"):
        assert key in line
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_followon_summary_ends_the_line_and_carries_the_ratios():
    """The JSON line ends with a compact `followon` object that repeats the companion figures
    (single step, batched and adjoint ratios, gradient errors), so that a reader of the line's
    tail sees them; built here from a hand-made line (no GPU)."""
    import json

    import bench

    line = {"value": 1450.0, "roofline": {"frac": 0.49},
            "single_step_kernel": {"gcell_s": 392.0, "frac": 0.94},
            "batched": {"value": 1330.0, "plain_fwd_value": 260.0, "vs_plain_fwd": 5.1},
            "adjoint": {"adjoint_ms": 10.8, "plain_fwd_ms": 2.9, "adjoint_over_fwd": 3.7,
                        "all_states": {"adjoint_over_fwd": 2.9}, "every_state": {"adjoint_over_fwd": 2.7},
                        "tape": {"sqrt": {"record_over_fwd": 1.0, "backward_over_fwd": 2.7},
                                 "all": {"record_over_fwd": 0.95, "backward_over_fwd": 1.8}},
                        "gradient_check": {
                            "short_horizon": {"T": 100,
                                              "fp32": {"dLdu0_dir_rel_err": 3e-4, "dLdv0_dir_rel_err": 1e-5,
                                                       "gene_rel_err": 3e-7},
                                              "fp64": {"dLdu0_dir_rel_err": 8e-7, "dLdv0_dir_rel_err": 3e-8,
                                                       "gene_rel_err": 9e-9}},
                            "workload_horizon": {"T": 2000,
                                                 "fp32": {"gene_rel_err": 3e-6, "dLdu0_vs_fp64_adjoint": 4e-3},
                                                 "fp64": {"gene_rel_err": 4e-6}}}}}
    line["followon"] = bench.followon_summary(line)
    text = json.dumps(line)
    tail = text[text.rindex('"followon"'):]
    assert list(json.loads(text))[-1] == "followon"
    f = json.loads(text)["followon"]
    assert f["batched"]["vs_plain_fwd"] == 5.1 and f["single_step"]["frac_hbm"] == 0.94
    assert f["adjoint"]["tape_sqrt"]["backward_over_fwd"] == 2.7 and f["adjoint"]["tape_all"]["backward_over_fwd"] == 1.8
    assert f["adjoint"]["grad_err_fp64"]["T100_dLdu0_dir_rel_err"] == 8e-7
    assert f["adjoint"]["grad_err_fp32"]["T2000_dLdu0_vs_fp64"] == 4e-3
    assert len(tail) < 1500  # small enough to survive a truncated log tail
