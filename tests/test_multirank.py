"""The multi-rank path of the benchmark on CPU (two gloo ranks): every rank solves its own
disjoint batch (seeds offset by rank, no collective on the data path), and the whole-job
figures are the slowest rank's time and the sum of all ranks' work.  The reference arm runs
on rank 0 only; other ranks leave without work."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Qs, _ = bench._instances(rank, sizes=(24,), seeds=3)
        ms, work = 10.0 * (rank + 1), 1000.0 * (rank + 1)
        ms_max, work_all = bench.aggregate_ranks(ms, work, dist, "cpu")
        digests = [float(np.sum(Q * np.arange(Q.size).reshape(Q.shape))) for Q in Qs]
        out.put((rank, ms_max, work_all, digests))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_aggregate():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, work_all, _ in res:
        assert ms_max == 20.0                 # the slowest rank
        assert work_all == 3000.0             # work of both ranks
    d0, d1 = res[0][3], res[1][3]
    assert len(d0) == len(d1) == 3
    assert not set(d0) & set(d1)              # disjoint instances: seeds offset by rank


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), dict(gpus=2, steps=1, warmup=0))()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""      # no line, no work on rank 1


def test_reference_arm_line_has_the_contract_keys(monkeypatch, capsys):
    """Rank 0 prints one JSON line with the keys of the benchmark contract (a short oracle
    sample per step here)."""
    import json
    import bench
    orig = bench.cpu_baseline
    monkeypatch.setattr(bench, "cpu_baseline", lambda budget_s=0.0, threads=None: orig(budget_s=0.2, threads=2))
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    args = type("A", (), dict(gpus=1, steps=1, warmup=1))()
    assert bench.run_reference(args) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["ms_per_step"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 2
    assert isinstance(line["cpu_baseline"]["cpu_model"], str) and line["cpu_baseline"]["cpu_model"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert "workload" in line["config"]
