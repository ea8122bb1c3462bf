"""Bounded device-side waits.  Every mbarrier wait of the TMA-fed FP32 kernels has a budget
(rbws_options.wait_cycles).  A budget of a few cycles makes the first wait of every CTA run
out; each kernel then flags the timeout, lets its copies in flight land and returns, and the
call returns RBWS_ERR_DEVICE_TIMEOUT.  The test then checks that the context and the problem
are still usable: a normal solve on the same problem matches the oracle."""
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


@pytest.mark.parametrize("precond", [rbws.PREC_MG, rbws.PREC_JACOBI])
def test_a_short_wait_budget_times_out_and_the_problem_stays_usable(precond):
    grid, blocks = (64, 32, 24), (2, 2, 1)
    op = O.assemble(grid, blocks)
    mu = inputs.log_uniform(95, 4, 4, 0.1, 10.0)
    with rbws.Problem(grid, blocks) as P:
        u = torch.empty((4, P.n), dtype=torch.float64, device="cuda")
        short = rbws.rbws_options_default(precision=rbws.FP32_IR, precond=precond, wait_cycles=8)
        with pytest.raises(rbws.RbwsError) as ei:
            rbws.rbws_solve_batch(P.h, mu, 1e-10, rbws.WARM_ZERO, u, short)
        assert ei.value.status == rbws.ERR_DEVICE_TIMEOUT
        with pytest.raises(rbws.RbwsError) as ei:  # negative budgets are rejected
            rbws.rbws_solve_batch(P.h, mu, 1e-10, rbws.WARM_ZERO, u,
                                  rbws.rbws_options_default(precision=rbws.FP32_IR, wait_cycles=-1))
        assert ei.value.status == rbws.ERR_INVALID_ARG
        normal = rbws.rbws_options_default(precision=rbws.FP32_IR, precond=precond)
        rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, 1e-10, rbws.WARM_ZERO, u, normal)
        assert rc == 0 and np.all(st == 0)
        uh = u.cpu().numpy()
    ref = O.solve_batch(op, mu, warm=O.WARM_ZERO, tol=1e-13)
    for b in range(4):
        assert np.linalg.norm(np.ones(op.n) - op.matvec(mu[b], uh[b])) / np.sqrt(op.n) < 1e-10
    assert np.all(np.linalg.norm(uh - ref.u, axis=1) / np.linalg.norm(ref.u, axis=1) < 1e-8)
