"""Multi-rank host logic on CPU (gloo, world size 2): sharding of independent
slices and the max-over-ranks timing that bench.py uses for N > 1."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1812_01307_gb300 import dist as D  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, lr, w = D.env_rank()
    start, stop = D.shard(64, r, w)
    elapsed = 1.0 + r             # rank 1 is the slow one
    mx = D.max_over_ranks(elapsed)
    units = D.sum_over_ranks(stop - start)
    D.barrier()
    q.put((r, lr, w, start, stop, mx, units))
    dist.destroy_process_group()


def test_two_ranks_gloo():
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
    (r0, lr0, w0, s0, e0, mx0, u0), (r1, lr1, w1, s1, e1, mx1, u1) = out
    assert (r0, r1, w0, w1, lr1) == (0, 1, 2, 2, 1)
    assert (s0, e0, s1, e1) == (0, 32, 32, 64)      # disjoint, covering
    assert mx0 == mx1 == 2.0                        # max over ranks
    assert u0 == u1 == 64.0


@pytest.mark.parametrize("n,w", [(10, 3), (7, 7), (3, 5), (64, 8)])
def test_shard_covers_items(n, w):
    got = [D.shard(n, r, w) for r in range(w)]
    assert got[0][0] == 0 and got[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
    sizes = [b - a for a, b in got]
    assert max(sizes) - min(sizes) <= 1


def test_single_process_identity():
    assert D.max_over_ranks(3.5) == 3.5
    assert D.env_rank() == (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
                            int(os.environ.get("WORLD_SIZE", "1")))
