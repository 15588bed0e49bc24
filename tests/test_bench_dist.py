"""bench.py's multi-process timing (weak scaling: max step time over ranks,
sum of the work of all ranks), run with two gloo processes on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, flop = bench.aggregate(10.0 + 5.0 * rank, 1e9 * (rank + 1), world)
    out.put((rank, ms, flop))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_max_time_sum_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, flop in res:
        assert ms == 15.0          # the slower rank sets the time
        assert flop == 3e9         # the work of both ranks


def test_single_process_passthrough():
    import bench
    assert bench.aggregate(7.0, 2.0, 1) == (7.0, 2.0)


def test_reference_arm_only_rank0_prints(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out == ""
