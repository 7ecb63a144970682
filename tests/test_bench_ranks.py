"""The N > 1 bench path on the CPU: two gloo ranks (replicas of the
benchmark box); the whole-job rate takes every rank's units over the slowest
rank's time, and the reference arm's non-zero ranks exit without work."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms_local = 10.0 * (rank + 1)            # rank 1 is the slow one
    rate, ms_max = bench.whole_job_rate(1000, ms_local, ws)
    bench.barrier(ws)
    out[rank] = (rate, ms_max)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_by_the_slowest_rank():
    ws, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
    for r in range(ws):
        rate, ms_max = out[r]
        assert ms_max == 20.0
        assert rate == pytest.approx(1000 * ws / 20e-3)


def test_reference_arm_nonzero_rank_exits_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        gpus, steps, warmup, n = 2, 1, 0, 8
    assert bench.run_reference(Args()) == 0


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """Rank 0 of the reference arm times the oracle on a bounded sample and
    prints one JSON line with the contract's keys."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")

    class Args:
        gpus, steps, warmup, n = 1, 1, 0, 8
    assert bench.run_reference(Args()) in (0, None)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    for k in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config"):
        assert k in line, k
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"]
