"""The multi-GPU host logic on CPU: two gloo ranks, each projecting its own
shard of points with the FP64 oracle (the arithmetic the GPUs run is tested
elsewhere), then the same collectives the benchmark uses -- the broadcast of
rank 0's plan choice and the maximum of the ranks' times -- and the job
throughput of a weak-scaling run; the row-range split of one caller's X with
landmarks broadcast from rank 0 once per version."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2201_00701_gb300 import sharding, workloads  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import oracle
    assert sharding.env_ranks() == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = workloads.mixture30_d16(n=n, shard=rank)
        out = oracle.project(w.X, w.hi, w.lo, w.k, w.boost, w.adjust, threads=1)
        # a rank-specific "time": the maximum must be the slowest rank's
        t_mine = 1.0 + rank
        t_max, other = sharding.max_over_ranks([t_mine, -rank])
        assert t_max == float(world) and other == 0.0
        assert sharding.broadcast_choice(10 * rank + 7) == 7
        value = sharding.job_throughput(n, world, 3, t_max)
        assert value == pytest.approx(world * n * 3 / world)
        np.save(os.path.join(outdir, f"x{rank}.npy"), w.X)
        np.save(os.path.join(outdir, f"o{rank}.npy"), out)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world, n = 2, 400
    mp.spawn(_rank_main, args=(world, _free_port(), n, str(tmp_path)), nprocs=world, join=True)
    import oracle
    xs = [np.load(tmp_path / f"x{r}.npy") for r in range(world)]
    outs = [np.load(tmp_path / f"o{r}.npy") for r in range(world)]
    # shards are different points of the same mixture, same landmarks
    assert not np.array_equal(xs[0], xs[1])
    assert len({r.tobytes() for r in np.concatenate(xs)}) == world * n
    # no cross-rank dependence: projecting the union at once gives the same
    w = workloads.mixture30_d16(n=n, shard=0)
    whole = oracle.project(np.concatenate(xs), w.hi, w.lo, w.k, w.boost, w.adjust, threads=1)
    assert np.array_equal(np.concatenate(outs), whole)


def _row_range_main(rank, world, port, n, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # one X, known to every rank; the landmarks only to rank 0
        w = workloads.mixture10_d8(n=n)
        hi = torch.from_numpy(w.hi.copy()) if rank == 0 else torch.zeros(w.L, w.d)
        lo = torch.from_numpy(w.lo.copy()) if rank == 0 else torch.zeros(w.L, 2)
        sync = sharding.LandmarkSync()
        assert sync.sync(1, hi, lo)
        assert not sync.sync(1 if rank == 0 else 5, hi, lo)   # rank 0's version decides
        assert sync.broadcasts == 1
        assert np.array_equal(hi.numpy(), w.hi) and np.array_equal(lo.numpy(), w.lo)
        # a new version on rank 0 is broadcast again
        if rank == 0:
            hi += 0.5
        assert sync.sync(2, hi, lo) and sync.broadcasts == 2
        assert np.array_equal(hi.numpy(), w.hi + np.float32(0.5))
        a, b = sharding.row_range(n, world, rank)
        out = oracle.project(w.X[a:b], hi.numpy(), lo.numpy(), w.k, w.boost, w.adjust,
                             threads=1)
        np.save(os.path.join(outdir, f"r{rank}.npy"), out)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_row_ranges_and_landmark_broadcast(tmp_path):
    """Two gloo ranks take their row ranges of one X and rank 0's landmarks
    (broadcast once per version); the outputs concatenated in rank order
    equal one projection of the whole X."""
    world, n = 2, 301
    mp.spawn(_row_range_main, args=(world, _free_port(), n, str(tmp_path)), nprocs=world,
             join=True)
    import oracle
    w = workloads.mixture10_d8(n=n)
    parts = [np.load(tmp_path / f"r{r}.npy") for r in range(world)]
    assert [len(p) for p in parts] == [151, 150]
    whole = oracle.project(w.X, w.hi + np.float32(0.5), w.lo, w.k, w.boost, w.adjust, threads=1)
    assert np.array_equal(np.concatenate(parts), whole)


def test_row_range_partition():
    for n in (0, 1, 7, 1000, 1_000_003):
        for world in (1, 2, 3, 8):
            ranges = [sharding.row_range(n, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.row_range(10, 2, 2)


def test_single_process_fallbacks():
    assert sharding.max_over_ranks([2.5, 1.0]) == [2.5, 1.0]
    assert sharding.broadcast_choice(3) == 3
    assert sharding.job_throughput(1000, 1, 10, 2.0) == 5000.0
    hi, lo = torch.ones(4, 8), torch.ones(4, 2)
    sync = sharding.LandmarkSync()
    assert sync.sync(3, hi, lo) and not sync.sync(3, hi, lo) and sync.broadcasts == 0
