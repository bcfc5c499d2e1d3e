"""The multi-rank host logic of bench.py on CPU: two gloo ranks (one per replica on a GPU
box) synchronise with the barrier, agree on the slowest rank's time, and report the
whole-job throughput of weak scaling; under torchrun only rank 0 runs the reference arm."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "HEAR_DIST_BACKEND": "gloo"})
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    ms = 100.0 + 50.0 * rank                       # rank 1 is the slow one
    d.barrier()
    slowest = d.max(ms)
    value = bench.replica_value(d.world, 10, 4, slowest)
    d.barrier()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"world": d.world, "rank": d.rank, "slowest": slowest, "value": value}, f)
    d.close()


def test_two_gloo_ranks_agree_on_the_slowest_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    for r, g in enumerate(got):
        assert g["world"] == 2 and g["rank"] == r
        assert g["slowest"] == 150.0                 # the max over ranks, seen by both
        assert g["value"] == pytest.approx(2 * 10 * 4 / 0.150)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload, steps, warmup, gpus = "small", 1, 0, 2
    bench.main_reference(Args())                    # returns at once, without work
    assert capsys.readouterr().out == ""


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "1")
    d = bench.Dist()
    assert d.pg is None and d.max(3.5) == 3.5
    assert bench.replica_value(1, 20, 1, 1000.0) == pytest.approx(20.0)


def test_bench_command_lines_parse(monkeypatch):
    """the driver's command lines and the options the profiles pin"""
    sys.path.insert(0, ROOT)
    import bench
    for argv in (["bench.py"], ["bench.py", "--gpus", "8", "--steps", "20", "--warmup", "3"],
                 ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                 ["bench.py", "--fc-form", "32,1", "--simd-rows", "0,2", "--no-served"]):
        monkeypatch.setattr(sys, "argv", argv)
        a = bench.parse()
        assert a.gpus >= 1 and a.steps >= 1 and a.warmup >= 0
    assert a.fc_form == "32,1" and [bench.SIMD_ROWS[int(i)] for i in a.simd_rows.split(",")][1][0] == "large"


def test_slot_batched_roofline_count():
    """the algorithmic multiply-pipe work of the slot-batched network: three partial products
    per (row, input, residue) of each FC, at the level the layer runs"""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2104_09164_gb300.workloads import make_workload
    w = make_workload("small")
    n = 1 << w.log_n
    primes = [1 << 40] * 8                       # only the count of limbs matters
    got = bench.simd_mad_lanes(primes, w.layers, 7, n)
    want = 128 * 2048 * 2 * n * 3 * 8 + 2 * 128 * 2 * n * 3 * 6    # FC1 at level 7, FC2 at level 5
    assert got == want
