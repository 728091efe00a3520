"""The bench's N > 1 host logic on CPU: replicas in a gloo process group
(world size 2).  Each rank's timed quantities are reduced to the maximum
over ranks, so the slowest rank defines the step, and the whole-job rate is
the units of all ranks over that time."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


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
