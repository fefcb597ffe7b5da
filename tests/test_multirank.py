"""Host logic of the multi-rank bench on CPU: two gloo ranks on 127.0.0.1.

The multi-GPU mode of the library is replicas (one independent sequence per
rank, no collective on the data path); what the ranks share is the bench's
bookkeeping: the max-over-ranks time, the sum-over-ranks work, the barrier,
and a distinct seeded sequence per rank.  These run here as two spawned
processes with the gloo backend.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    mx = bench.max_over_ranks(10.0 * (rank + 1), world, None)
    sm = bench.sum_over_ranks(float(rank + 1), world, None)
    bench.barrier(world)
    seq, _ = bench.make_sequence("tiny", seed_offset=rank)
    dist.destroy_process_group()
    q.put((rank, r, w, mx, sm, float(seq.astype("float64").sum()), seq.shape))


def test_two_gloo_ranks_reduce_and_get_distinct_sequences():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, r, w, mx, sm, _, shape in out:
        assert (r, w) == (rank, 2)
        assert mx == 20.0            # the slowest rank's time
        assert sm == 3.0             # work of all ranks
        assert shape == (16, 64, 64)
    assert out[0][5] != out[1][5]    # each replica registers its own sequence
    del torch
