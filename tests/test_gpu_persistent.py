"""The persistent FP64 PCG: one cooperative launch runs the start, the iterations and the
true-residual checks with restarts (Algorithm 1 inside Algorithm 4) of every instance, with
the convergence loop on the device.  It runs the same phase bodies as the graph-captured
path, in the same order per instance, so its results must be bitwise those of that path; it
also takes the batches of several grids in one launch, and its grid barriers are bounded."""
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


@pytest.mark.parametrize("precond,warm", [(rbws.PREC_JACOBI, rbws.WARM_GALERKIN), (rbws.PREC_NONE, rbws.WARM_ZERO),
                                          (rbws.PREC_JACOBI, rbws.WARM_ZERO)])
def test_persistent_equals_the_graph_path_and_the_oracle(precond, warm):
    grid, blocks = (40, 33, 28), (2, 2, 1)
    w = inputs.small(grid=grid, blocks=blocks, n_max=8, n_train=24, n_test=12)
    op = O.assemble(grid, blocks)
    mu = inputs.test_mu(w)
    B = len(mu)
    with rbws.Problem(grid, blocks) as P:
        rbws.rbws_offline_greedy(P.h, inputs.train_mu(w), w.n_max, 0.0, 1e-12)
        out = {}
        for pers in (0, 1):
            u = torch.empty((B, P.n), dtype=torch.float64, device="cuda")
            opt = rbws.rbws_options_default(precond=precond, persistent=pers)
            rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, 1e-11, warm, u, opt)
            assert rc == 0 and np.all(st == 0)
            out[pers] = (u.cpu().numpy(), it, rel)
    (u0, it0, rel0), (u1, it1, rel1) = out[0], out[1]
    assert np.array_equal(it0, it1) and np.array_equal(rel0, rel1)
    assert np.array_equal(u0, u1)
    pre = O.PREC_JACOBI if precond == rbws.PREC_JACOBI else O.PREC_NONE
    for b in range(0, B, 3):
        ref = O.pcg(op, mu[b], precond=pre, tol=1e-13)
        assert np.linalg.norm(u1[b] - ref.u) <= 1e-9 * np.linalg.norm(ref.u)


def test_persistent_residual_history_equals_the_graph_path():
    grid, blocks = (24, 20, 16), (2, 1, 1)
    mu = inputs.log_uniform(301, 4, 2, 0.1, 10.0)
    with rbws.Problem(grid, blocks) as P:
        h = {}
        for pers in (0, 1):
            u = torch.empty((4, P.n), dtype=torch.float64, device="cuda")
            rc, it, rel, st, hist = rbws.rbws_solve_batch_history(P.h, mu, 1e-12, rbws.WARM_ZERO, u, 200,
                                                                  rbws.rbws_options_default(persistent=pers))
            assert rc == 0
            h[pers] = hist
    assert np.array_equal(np.nan_to_num(h[0], nan=-1.0), np.nan_to_num(h[1], nan=-1.0))


def test_one_launch_for_uneven_grids_matches_the_oracle():
    grids = [((24, 24, 24), (3, 3, 3)), ((32, 28, 20), (3, 3, 3)), ((16, 16, 16), (3, 3, 3))]
    ops = [O.assemble(g, b) for g, b in grids]
    probs = [rbws.Problem(g, b) for g, b in grids]
    try:
        mus = inputs.log_uniform(302, 12, 27, 0.1, 10.0)
        which = [0, 1, 2, 1, 0, 2, 2, 0, 1, 1, 0, 2]
        handles = [probs[k].h for k in which]
        res = {}
        for pers in (0, 1):
            outs = [torch.empty(probs[k].n, dtype=torch.float64, device="cuda") for k in which]
            rc, it, rel, st, lat = rbws.rbws_solve_requests(handles, list(mus), outs, 1e-12, rbws.WARM_ZERO,
                                                            rbws.rbws_options_default(persistent=pers))
            assert rc == 0 and np.all(st == 0) and np.all(lat > 0)
            res[pers] = (it, [o.cpu().numpy() for o in outs])
        # one launch takes one CTA shape for every grid (that of the smallest), so its partial
        # sums are grouped differently from the per-grid launches: equal to rounding, not bitwise
        assert np.all(np.abs(res[0][0] - res[1][0]) <= 1)
        for r, k in enumerate(which):
            u = res[1][1][r]
            assert np.linalg.norm(u - res[0][1][r]) <= 1e-11 * np.linalg.norm(u)
            ref = O.pcg(ops[k], mus[r], tol=1e-12)  # the same tolerance: iterations within 2
            assert abs(int(res[1][0][r]) - ref.iters) <= 2
            assert np.linalg.norm(u - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
    finally:
        for P in probs:
            P.close()


def test_persistent_barrier_wait_runs_out_and_the_problem_stays_usable():
    grid, blocks = (32, 24, 20), (2, 2, 1)
    op = O.assemble(grid, blocks)
    mu = inputs.log_uniform(303, 4, 4, 0.1, 10.0)
    with rbws.Problem(grid, blocks) as P:
        u = torch.empty((4, P.n), dtype=torch.float64, device="cuda")
        with pytest.raises(rbws.RbwsError) as ei:
            rbws.rbws_solve_batch(P.h, mu, 1e-12, rbws.WARM_ZERO, u,
                                  rbws.rbws_options_default(persistent=1, wait_cycles=8))
        assert ei.value.status == rbws.ERR_DEVICE_TIMEOUT
        rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, 1e-12, rbws.WARM_ZERO, u,
                                                rbws.rbws_options_default(persistent=1))
        assert rc == 0 and np.all(st == 0)
        uh = u.cpu().numpy()
    for b in range(4):
        ref = O.pcg(op, mu[b], tol=1e-13)
        assert np.linalg.norm(uh[b] - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
