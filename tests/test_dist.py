"""The bench's multi-rank path on the CPU: two ranks over gloo.  Each rank
draws its own batch (no data-path collective), the job time is the slowest
rank's, the whole-job value counts every rank's cells, and only rank 0 runs
the reference arm."""
import contextlib
import io
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2506_22935_gb300 import inputs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank's own inputs
        phi = inputs.random_phases(bench.rank_seed(rank), 2, 64)
        got = [None] * world
        dist.all_gather_object(got, phi[0, :4].tolist())
        # the job's time is the slowest rank's
        local_ms = 10.0 + 5.0 * rank
        job_ms = bench.reduce_max_ms(local_ms, dist, torch.device("cpu"))
        value = bench.weak_value(world, 1e9, 3, job_ms)
        out.put((rank, got, job_ms, value))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, job_ms, value in res:
        assert job_ms == 15.0                      # max over ranks
        assert value == pytest.approx(2 * 1e9 * 3 / 0.015 / 1e9)
        assert not np.allclose(got[0], got[1])     # independent batches per rank


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})())
    assert buf.getvalue() == ""


def test_reference_arm_prints_the_contract_line(monkeypatch):
    """Rank 0 of the reference arm prints one JSON line with the metric, the
    oracle as cpu_baseline and a zero-copy e2e block (small oracle budget)."""
    import json
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(bench, "_oracle_budget_cols", lambda seconds: 4)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(type("A", (), {"steps": 1, "warmup": 3, "gpus": 1})())
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
