"""The bench's host logic on CPU: replicas in a gloo process group (world
size 2), where each rank's timed quantities are reduced to the maximum over
ranks, so the slowest rank defines the step and the whole-job rate is the
units of all ranks over that time; and the reference arm's JSON line."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, local, w = bench.dist_env()
    assert (r, local, w) == (rank, rank, world)
    # rank 0 is slower at the first quantity, rank 1 at the second
    got = bench.max_over_ranks([2.0 - rank, 1.0 + 3 * rank, 7.5], torch.device("cpu"), world)
    dist.barrier()
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write(",".join("%.3f" % x for x in got))
    dist.destroy_process_group()


def test_max_over_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        assert (tmp_path / ("rank%d.txt" % r)).read_text() == "2.000,4.000,7.500"


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([1.0, 2.0], None, 1) == [1.0, 2.0]


def test_reference_arm_non_zero_rank_exits_quietly(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(None) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle timed on the host, no GPU)
    prints exactly one JSON line with the contract's keys, on the same
    metric, unit and config as the GPU arm."""
    import json
    import subprocess
    import sys
    import bench
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2", "--warmup", "1",
           "--b-log2", "10", "--batches", "4", "--lookups-log2", "12", "--queries-log2", "10"]
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "M updates/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert "workload" in line["config"] and line["config"]["b"] == 1024 and line["config"]["batches"] == 4
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
