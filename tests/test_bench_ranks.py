"""Host-side logic of the multi-GPU bench (replicas, one process per GPU),
run as two gloo ranks on the CPU: every rank sees the slowest rank's step
time, the whole-job value counts the units of all ranks, and the reference
arm prints from rank 0 only."""

import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_max, value = bench.job_timing(10.0 + 5.0 * rank, 1000.0, world)
    out.put((rank, ms_max, value))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value in res:
        assert ms_max == 15.0
        assert value == pytest.approx(1000.0 * 2 / 0.015)


def test_single_process_timing_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_timing(4.0, 8.0, 1) == (4.0, 8.0 / 0.004)


def test_reference_arm_prints_from_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(bench.parse(["--impl", "reference"]))
    assert buf.getvalue() == ""


def test_reference_arm_times_the_whole_oracle_step(monkeypatch):
    """The reference arm (rank 0, N = 1) prints one JSON line whose value is
    element pairs per second of the oracle's whole step (the scope of one
    GPU step), on the small level-1 workload here."""
    import json

    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(bench.parse(["--impl", "reference", "--steps", "2", "--warmup", "1",
                                         "--workload", "sphere_L1_eps4_ka1"]))
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2
    assert line["value"] > 0 and line["unit"] == bench.UNIT
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["value"] == line["value"]
    # value = element pairs of the steps over their summed time
    assert line["value"] == pytest.approx(2 * 80 * 80 / (2 * line["ms_per_step"] / 1e3), rel=1e-3)
