"""Multi-rank host logic (replicas only) on two gloo ranks on the CPU: every
rank gets a distinct seed, batch shards cover each problem exactly once, the
step time is the maximum over ranks and the whole-job rate counts every
rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1811_09909_gb300 import replicas  # noqa: E402


def test_shard_covers_every_unit_once():
    for n in (0, 1, 5, 64, 65):
        for world in (1, 2, 3, 8):
            seen = []
            sizes = []
            for r in range(world):
                lo, hi = replicas.shard(n, r, world)
                seen.extend(range(lo, hi))
                sizes.append(hi - lo)
            assert seen == list(range(n))
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def test_single_process_defaults():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.whole_job_rate(1000, 1, 2.0) == 500000.0
    assert replicas.replica_seed(2, 0) == 2 and replicas.replica_seed(2, 1) != 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = replicas.rank_info()
        ms = 10.0 + 5.0 * r                       # rank 1 is the slow one
        dist.barrier()
        mx = replicas.max_over_ranks(ms, dist)
        lo, hi = replicas.shard(64, r, w)
        out[r] = (r, w, lr, mx, lo, hi, replicas.replica_seed(2, r),
                  replicas.whole_job_rate(1000, w, mx))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        rr, w, lr, mx, lo, hi, seed, rate = res[r]
        assert (rr, w, lr) == (r, 2, r)
        assert mx == 15.0                          # the slowest rank's time on every rank
        assert rate == pytest.approx(1000 * 2 / 15e-3)
    assert (res[0][4], res[0][5], res[1][4], res[1][5]) == (0, 32, 32, 64)
    assert res[0][6] != res[1][6]
