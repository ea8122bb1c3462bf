"""Host logic of the multi-GPU run (one process per GPU), on the CPU.

The parameter instances are independent, so ranks split them with no collective
on the data path (weak scaling).  Two gloo ranks check that the split is
disjoint and complete, that solving each rank's block separately gives exactly
the single-process result (the oracle's Algorithm 4 per instance), and that the
step time is reduced as the maximum over ranks.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_2311_13862_gb300 import inputs, ranks


def test_shard_blocks_are_disjoint_and_cover_the_job():
    rows = np.arange(24)
    for world in (1, 2, 3, 4, 6):
        per = len(rows) // world
        got = np.concatenate([ranks.shard(rows, per, r, world) for r in range(world)])
        assert np.array_equal(got, rows)
    with pytest.raises(ValueError):
        ranks.shard(rows, 5, 0, 4)       # 20 != 24 rows
    with pytest.raises(ValueError):
        ranks.shard(rows, 12, 2, 2)      # rank out of range


def test_rank_info_and_job_rate():
    assert ranks.rank_info({}) == ranks.RankInfo(0, 1, 0)
    assert ranks.rank_info({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == ranks.RankInfo(1, 2, 1)
    with pytest.raises(ValueError):
        ranks.rank_info({"RANK": "2", "WORLD_SIZE": "2"})
    # 256 solves per rank on 4 ranks in 40 ms per step: 25,600 solves/s for the job
    assert ranks.job_rate(256, 4, 40.0) == pytest.approx(25600.0)
    with pytest.raises(ValueError):
        ranks.job_rate(1, 1, 0.0)
    assert ranks.max_over_ranks(3.5) == 3.5  # no process group: the value itself


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle as O

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = inputs.small()
        per = 3
        mu = ranks.shard(inputs.test_mu(w, per * world), per, rank, world)
        op = O.assemble(w.grid, w.blocks)
        res = O.solve_batch(op, mu, warm=O.WARM_ZERO, tol=1e-10, n_threads=1)
        # rank-dependent "step times": the reduction must return the slowest
        ms = ranks.max_over_ranks(10.0 + 5.0 * rank, "cpu")
        parts = [None] * world
        dist.all_gather_object(parts, (rank, mu, res.u, res.iters, ms))
        if rank == 0:
            np.savez(os.path.join(out_dir, "parts.npz"),
                     ranks=np.array([p[0] for p in parts]), mu=np.concatenate([p[1] for p in parts]),
                     u=np.concatenate([p[2] for p in parts]), iters=np.concatenate([p[3] for p in parts]),
                     ms=np.array([p[4] for p in parts]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_the_parameters_and_reduce_the_time():
    mp = pytest.importorskip("torch.multiprocessing")
    import oracle as O

    O.lib()  # compile the oracle once before the ranks load it
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), d), nprocs=world, join=True,
                           start_method="spawn")
        got = np.load(os.path.join(d, "parts.npz"))
    w = inputs.small()
    mu_all = inputs.test_mu(w, 3 * world)
    assert np.array_equal(got["ranks"], np.arange(world))
    assert np.array_equal(got["mu"], mu_all)          # disjoint blocks, in rank order, covering the job
    ref = O.solve_batch(O.assemble(w.grid, w.blocks), mu_all, warm=O.WARM_ZERO, tol=1e-10, n_threads=1)
    assert np.array_equal(got["u"], ref.u)            # per-instance solves: splitting changes nothing
    assert np.array_equal(got["iters"], ref.iters)
    assert np.all(got["ms"] == 15.0)                  # every rank sees the slowest rank's time
