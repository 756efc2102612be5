"""The N > 1 bench path on CPU: world_size-2 gloo ranks.  Each rank runs a
replica ("replicas only": no data-path collective); the whole-job value is the
units of all ranks divided by the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    units = 1000.0 * (rank + 1)            # uneven replicas
    ms = 10.0 * (rank + 1)
    bench.barrier()
    value, max_ms = bench.aggregate(units, ms)
    out[rank] = (value, max_ms)
    dist.destroy_process_group()


def test_aggregate_world2_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        value, max_ms = res[r]
        assert max_ms == pytest.approx(20.0)
        assert value == pytest.approx(3000.0 / 0.020)


def test_reference_arm_other_ranks_exit_cleanly(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload = "burgers2d_small"
        steps = 1
        warmup = 1
        gpus = 2
    assert bench.run_reference(A()) == 0
