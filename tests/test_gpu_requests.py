"""Uneven batches: requests on several grids in one call (each grid's batch on its own
stream), per-request latency from the GPU timer, and the tile autotuner."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2311_13862_gb300 import inputs, rbws

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2311_13862_gb300 import build
    build.build()


GRIDS = [((24, 24, 24), (3, 3, 3)), ((32, 28, 20), (3, 3, 3)), ((16, 16, 16), (3, 3, 3))]


@pytest.mark.parametrize("precision,tol", [(rbws.FP64, 1e-12), (rbws.FP32_IR, 1e-10)])
def test_mixed_grid_requests_match_oracle(precision, tol):
    ops = [O.assemble(g, b) for g, b in GRIDS]
    probs = [rbws.Problem(g, b) for g, b in GRIDS]
    mus_all = inputs.log_uniform(91, 12, 27, 0.1, 10.0)
    which = [0, 1, 2, 1, 0, 2, 2, 0, 1, 1, 0, 2]  # interleaved grids
    handles = [probs[k].h for k in which]
    outs = [torch.empty(probs[k].n, dtype=torch.float64, device="cuda") for k in which]
    rc, it, rel, st, lat = rbws.rbws_solve_requests(handles, list(mus_all), outs, tol, rbws.WARM_ZERO,
                                                    rbws.rbws_options_default(precision=precision))
    assert rc == 0 and np.all(st == 0)
    assert np.all(lat > 0) and np.all(np.isfinite(lat))
    for r, k in enumerate(which):
        u = outs[r].cpu().numpy()
        true_rel = np.linalg.norm(np.ones(ops[k].n) - ops[k].matvec(mus_all[r], u)) / np.sqrt(ops[k].n)
        assert true_rel < tol
        if precision == rbws.FP64:
            ref = O.pcg(ops[k], mus_all[r], tol=1e-12)
            assert np.linalg.norm(u - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
            assert abs(it[r] - ref.iters) <= 2
    for P in probs:
        P.close()


def test_autotune_picks_a_valid_tile_and_caches_it(tmp_path):
    grid, blocks = (64, 48, 40), (2, 2, 1)
    op = O.assemble(grid, blocks)
    cache = tmp_path / "tiles.txt"
    mu = inputs.log_uniform(92, 8, 4, 0.1, 10.0)
    with rbws.Problem(grid, blocks) as P:
        tx, ty, zc, ms, sched = rbws.rbws_autotune(P.h, 8, cache)
        assert tx in (4, 8, 16, 32) and 64 <= tx * ty <= 256 and zc >= 1 and ms > 0 and sched in (0, 1, 2, 3)
        assert cache.read_text().split()[1:4] == [str(tx), str(ty), str(zc)]
        again = rbws.rbws_autotune(P.h, 8, cache)  # read back from the cache
        assert again[:3] == (tx, ty, zc) and again[4] == sched
        u = torch.empty((8, P.n), dtype=torch.float64, device="cuda")
        rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, 1e-10, rbws.WARM_ZERO, u,
                                                rbws.rbws_options_default(precision=rbws.FP32_IR))
        assert rc == 0 and np.all(st == 0)
        uh = u.cpu().numpy()
    for b in range(8):
        assert np.linalg.norm(np.ones(op.n) - op.matvec(mu[b], uh[b])) / np.sqrt(op.n) < 1e-10


@pytest.mark.parametrize("sched", [0, 1, 2, 3])
def test_each_fp32_schedule_reaches_the_fp64_residual(tmp_path, sched):
    """Forces each FP32 iteration schedule through an autotuner cache entry (0: 44 bytes per
    DoF with register prefetch, 1: 32 bytes with recomputed A p, 2: 44 bytes with the TMA-fed
    stencil phase, 3: 32 bytes in s-form with both phases TMA-fed) and checks the solutions
    with the oracle's FP64 operator."""
    grid, blocks = (64, 40, 36), (2, 2, 1)
    op = O.assemble(grid, blocks)
    B = 6
    mu = inputs.log_uniform(93, B, 4, 0.1, 10.0)
    cache = tmp_path / "tiles.txt"
    cache.write_text("%dx%dx%d/B%d/fp32 16 8 16 1.0 %d\n" % (grid + (B, sched)))
    with rbws.Problem(grid, blocks) as P:
        assert rbws.rbws_autotune(P.h, B, cache)[:3] == (16, 8, 16)
        u = torch.empty((B, P.n), dtype=torch.float64, device="cuda")
        rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, 1e-10, rbws.WARM_ZERO, u,
                                                rbws.rbws_options_default(precision=rbws.FP32_IR))
        assert rc == 0 and np.all(st == 0)
        uh = u.cpu().numpy()
    ref = O.solve_batch(op, mu, warm=O.WARM_ZERO, tol=1e-13)
    for b in range(B):
        assert np.linalg.norm(np.ones(op.n) - op.matvec(mu[b], uh[b])) / np.sqrt(op.n) < 1e-10
    assert np.all(np.linalg.norm(uh - ref.u, axis=1) / np.linalg.norm(ref.u, axis=1) < 1e-8)
    print("schedule", sched, "iterations", it.tolist())
