"""bench.py's multi-rank plumbing (Replicas) on two CPU processes over gloo:
the N-GPU run is N replicas of the whole step (the path does not shard), so
both ranks must see the slowest rank's time and the whole job's throughput
(units of every rank over that time)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    reps = bench.Replicas("gloo")
    reps.barrier()
    ms = reps.max_ms(10.0 * (rank + 1))          # rank 1 is the slow one
    value = reps.throughput(1e9, ms)
    reps.barrier()
    reps.close()
    q.put((rank, reps.world, ms, value))


def test_two_replicas_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0], codes
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, world, ms, value in res:
        assert world == 2
        assert ms == pytest.approx(20.0)
        assert value == pytest.approx(2 * 1e9 / 0.020)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE"):
        os.environ.pop(k, None)
    reps = bench.Replicas("gloo")
    assert reps.world == 1 and reps.max_ms(7.5) == 7.5 and reps.throughput(1e6, 2.0) == pytest.approx(5e8)
    reps.close()
