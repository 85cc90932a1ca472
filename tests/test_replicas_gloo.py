"""Multi-GPU path of bench.py (independent replicas: each rank decodes its
own streams and no data moves between ranks): per-rank workloads and the
max-over-ranks aggregation, run as two gloo ranks on CPU; and the reference
arm's output line."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    a = bench.parse_args(["--width", "64", "--height", "48", "--frames", "3", "--seed", "5"])
    gop = bench.make_workload(a, rank)  # replicas decode different streams
    # rank r "took" 10 + 5 r ms for 3 steps of a 3-frame GOP
    value, ms = bench.replica_value(10.0 + 5.0 * rank, 3 * gop.n_frames, 64 * 48 / bench.FULLHD_PX, dist)
    q.put((rank, value, ms, int(gop.iframe.y_idx[:4].sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_aggregate_max_time():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, v0, ms0, s0), (r1, v1, ms1, s1) = out
    assert ms0 == ms1 == 15.0  # max over ranks
    expect = 2 * 9 * (64 * 48 / (1920 * 1080)) / 0.015
    assert abs(v0 - expect) < 1e-9 and abs(v1 - expect) < 1e-9
    assert s0 != s1  # each rank has its own seeded stream


def test_single_process_value():
    import bench

    v, ms = bench.replica_value(20.0, 30, 1.0)
    assert ms == 20.0 and abs(v - 1500.0) < 1e-9


def test_reference_arm_nonzero_rank_exits_without_work(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(bench.parse_args(["--impl", "reference"])) == 0


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    """Rank 0 of the reference arm times the oracle on the same workload and
    prints one JSON line with the contract's keys."""
    import json

    import bench

    monkeypatch.setenv("RANK", "0")
    a = bench.parse_args(["--impl", "reference", "--width", "48", "--height", "32", "--frames", "3",
                          "--steps", "1", "--warmup", "1"])
    assert bench.run_reference(a) == 0
    lines = [x for x in capsys.readouterr().out.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"]
