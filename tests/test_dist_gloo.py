"""The N > 1 plumbing of bench.py (rendezvous, barrier, max/sum over ranks)
on CPU with the gloo backend, world size 2."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w = bench.dist_init("gloo")
    bench.dist_barrier()
    mx = bench.dist_max(float(10 + r))            # each rank's "elapsed ms"
    sm = bench.dist_sum(float(100 * (r + 1)))     # each rank's units
    q.put((r, w, mx, sm))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_and_sum():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, mx, sm in out:
        assert w == 2 and mx == 11.0 and sm == 300.0
