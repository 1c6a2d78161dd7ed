"""Multi-rank host logic on CPU (gloo, world size 2, 127.0.0.1): the batched
workload is split over ranks with no data exchange (every rank computes the
same split locally), and bench.py's reductions over ranks (max of the times,
sum of the work) give the whole-job numbers."""
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORLD = 2


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    import paper_2604_09517_gb300 as hpl

    d = bench.Dist()
    d.init("gloo")
    try:
        # reductions used for the whole-job value: slowest rank, total work
        assert d.max(float(rank)) == world - 1
        assert d.sum(1.0) == world
        n = hpl.batch_sizes(1, 4096)
        kind = np.array([0 if s < 2048 else 1 for s in range(4096)], dtype=np.uint8)
        owner = hpl.batch_shard(n, kind, world)
        assert owner.min() >= 0 and owner.max() < world
        mine = np.nonzero(owner == rank)[0]
        # every system is solved by exactly one rank
        assert d.sum(float(mine.size)) == 4096
        # all ranks computed the same split (a position-weighted checksum)
        h = float(np.sum((owner.astype(np.int64) + 1) * (np.arange(4096) % 9973)))
        assert d.max(h) == h and -d.max(-h) == h
        # balanced estimated work: FP64 systems weigh 64x per flop
        w = np.where(kind == 0, 64.0, 1.0) * n.astype(np.float64) ** 3
        share = float(w[mine].sum())
        assert d.max(share) <= 1.01 * d.sum(share) / world
        # both kinds are spread over the ranks
        assert 0 < int(np.sum(kind[mine] == 0)) < 2048 and 0 < int(np.sum(kind[mine] == 1)) < 2048
    finally:
        d.close()


def test_batched_split_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    from paper_2604_09517_gb300 import _build
    _build.build()                          # once, before the ranks load the library
    mp.spawn(_worker, args=(WORLD, _free_port()), nprocs=WORLD, join=True)


def test_batch_shard_edge_cases():
    import paper_2604_09517_gb300 as hpl
    assert list(hpl.batch_shard([5], [0], 4)) == [0]
    assert hpl.batch_shard([], [], 3).size == 0
    owner = hpl.batch_shard([512, 512, 512, 32], [0, 0, 0, 1], 3)
    assert sorted(owner[:3]) == [0, 1, 2] and owner[3] == 0
    try:
        hpl.batch_shard([5], [0], 0)
        raise AssertionError("world 0 accepted")
    except hpl.HplError:
        pass
