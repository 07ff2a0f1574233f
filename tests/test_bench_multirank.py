"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, no collective on the data path; only
the timing is reduced).  Each rank runs its own circuits, the step time is the maximum over ranks,
and the reported value counts the units of every rank over that time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    bench.init_ranks()                                 # gloo here: no GPU
    assert dist.is_initialized() and dist.get_backend() == "gloo"
    try:
        r, w, local = bench.dist_env()
        t = bench.max_over_ranks(1.5 + rank)          # rank 0 took 1.5 s, rank 1 took 2.5 s
        units = bench.sum_over_ranks(3.0 + rank)      # rank 0 did 3 units, rank 1 did 4
        out[rank] = (r, w, local, t, tuple(bench.rank_seeds(r)), units)
    finally:
        bench.finish_ranks()
        assert not dist.is_initialized()


def test_two_gloo_ranks_reduce_the_step_time_and_split_the_seeds():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, w, local, t, seeds, units) in res.items():
        assert (r, w, local) == (rank, world, rank)
        assert t == pytest.approx(2.5)                  # max over ranks
        assert units == pytest.approx(7.0)              # sum over ranks
    assert not set(res[0][4]) & set(res[1][4])          # each rank its own circuits
    import bench
    assert bench.aggregate_rate(512, 5, world, 2.5) == pytest.approx(512 * 5 * 2 / 2.5)


def test_single_process_is_unchanged():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.sum_over_ranks(3.25) == 3.25
    assert bench.rank_seeds(0) == list(range(1, bench.SEEDS_PER_D + 1))


def test_all_core_oracle_sample_finishes_the_circuits_it_starts():
    """The batched workload's CPU baseline: spawned workers, one circuit each; every circuit started is
    finished and counted, and a zero budget still runs one circuit per worker."""
    import bench
    shapes = [(4, 3, 4, 1), (5, 3, 5, 2), (4, 2, 4, 3)]
    rate, wall, done = bench.cpu_oracle_pool_sample(shapes, 3, 27, 60.0, 2)
    assert done == 3 and wall > 0 and rate == pytest.approx((4 + 5 + 4) / wall)
    _rate, _wall, done = bench.cpu_oracle_pool_sample(shapes, 3, 27, 0.0, 2)
    assert done == 2
