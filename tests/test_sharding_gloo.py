"""Multi-rank host logic of the sub-cube sharding, on CPU with the gloo backend
(world size 2): ranks get distinct seeded cubes or disjoint sub-cubes, and the
timing reduction takes the maximum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2003_07358_gb300 import sharding as sh  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    info = sh.rank_info()
    seed_off, cubes = sh.replicate_cubes(4, info)
    mine = sh.split_subcubes(4, info)
    t = sh.max_over_ranks(1.0 + rank, dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, (seed_off, cubes, mine, t))
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (s0, c0, m0, t0), (s1, c1, m1, t1) = res
    assert s0 != s1 and c0 == c1 == [0, 1, 2, 3]          # weak scaling: distinct cubes, full work each
    assert sorted(m0 + m1) == [0, 1, 2, 3] and not set(m0) & set(m1)
    assert t0 == t1 == 2.0                                  # max over ranks
    assert sh.weak_scaling_value(5, world, 2.0) == 5.0


def test_single_rank_defaults():
    info = sh.rank_info({})
    assert (info.rank, info.world, info.local) == (0, 1, 0)
    assert sh.split_subcubes(3, info) == [0, 1, 2]
    assert sh.max_over_ranks(3.5, None) == 3.5
