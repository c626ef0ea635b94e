"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks.

Ranks register independent problems (weak scaling): each gets its own
generator seed, the job time is the slowest rank's, and the job value counts
the units of all ranks.  No data-path collective is involved."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms = 10.0 + 5.0 * rank                     # rank 1 is the slow one
    ms_max = bench.slowest_rank_ms(ms, w, "cpu")
    out[rank] = (r, w, bench.rank_seed(r), ms_max, bench.job_value(1e6, w, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    seeds = {res[r][2] for r in res}
    assert len(seeds) == 2                               # independent problems
    for r in res:
        assert res[r][0] == r and res[r][1] == world
        assert res[r][3] == 15.0                         # the slowest rank's time on every rank
        assert abs(res[r][4] - 2 * 1e6 / 0.015) < 1e-6   # units of both ranks over that time


def test_single_rank_is_identity():
    import bench
    assert bench.slowest_rank_ms(12.5, 1, "cpu") == 12.5
    assert bench.job_value(100.0, 1, 1000.0) == 100.0
