"""The multi-rank logic of bench.py on CPU (gloo, world size 2).

Each rank assembles its own replica (weak scaling, no collective on the data
path); the only collectives are the barrier and the max-over-ranks reduction
of the step time, which these tests exercise without a GPU.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist
    r, local, w = bench.dist_init("gloo")
    assert (r, local, w) == (rank, rank, world)
    bench.barrier()
    slowest = bench.max_over_ranks(0.25 * (rank + 1))
    out.put((rank, slowest, bench.aggregate_throughput(1000, w, slowest)))
    bench.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [0.5, 0.5]          # the slower rank sets the time
    assert [g[2] for g in got] == [4000.0, 4000.0]    # 2 ranks x 1000 units / 0.5 s


def test_single_process_helpers():
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.aggregate_throughput(10, 1, 2.0) == 5.0


def test_reference_arm_non_zero_rank_exits_without_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"]) == 0


def test_warmup_floor():
    with pytest.raises(SystemExit):
        bench.main(["--warmup", "2"])
