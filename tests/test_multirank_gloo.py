"""Host-side multi-rank logic of bench.py on two gloo ranks (CPU, 127.0.0.1).

Instances are independent, so N GPUs run N replicas with no data-path collective; the only
cross-rank steps are the barrier around the timed region and the max over ranks of the
elapsed time, which these tests exercise without a GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    bench.barrier()
    t = bench.max_over_ranks(10.0 + 5.0 * rank)
    bench.barrier()
    dist.destroy_process_group()
    q.put((rank, ws, r, local, t))


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_barrier(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, local, t in res:
        assert ws == world and r == rank and local == rank
        assert t == 10.0 + 5.0 * (world - 1)


def test_single_process_defaults():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_env() == (1, 0, 0)
        assert bench.max_over_ranks(3.5) == 3.5
    finally:
        os.environ.update(env)
