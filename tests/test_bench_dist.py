"""bench.py's multi-rank logic on CPU: two gloo ranks (127.0.0.1) take the
slowest rank's time, report whole-job throughput over all replicas, and only
rank 0 runs the reference arm."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        t = bench.max_over_ranks(times[r], dist, "cpu")
        out[r] = (r, w, lr, t, bench.job_throughput(w, 1000, 10, t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_replicas():
    world = 2
    times = [0.5, 2.0]
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        rr, w, lr, t, v = res[r]
        assert (rr, w, lr) == (r, world, r)
        assert t == 2.0
        assert v == world * 1000 * 10 / 2.0


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(1.25, None, "cpu") == 1.25
    assert bench.job_throughput(1, 100, 4, 2.0) == 200.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup, gpus = 1, 0, 2

    bench.run_reference(Args)
    assert capsys.readouterr().out == ""


@pytest.mark.slow
def test_reference_arm_line(monkeypatch, capsys):
    """The reference arm's JSON line: the oracle timed on its sample, with the keys the driver reads."""
    import json
    monkeypatch.setenv("RANK", "0")

    class Args:
        steps, warmup, gpus = 1, 0, 1

    bench.run_reference(Args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["ms_per_step"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
