"""Float-float reliable updates of the mixed-precision iteration (ru_mode 2, the default on
grids with nx % 4 == 0).  The update r <- r - A d, u <- u + d in pairs of floats is pinned
against the oracle's FP64 CSR residual of u0 + d: its error must sit at float-float level
(about 1e-14 of |A| |u|), far below what FP32 arithmetic could reach (about 1e-7), so a
dropped low part or a wrong sign fails.  Then full solves with float-float and with FP64
updates both reach the oracle's FP64 solutions."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle as O
from oracle import batch as OB
from paper_2311_13862_gb300 import inputs, rbws

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2311_13862_gb300 import build
    build.build()


@pytest.mark.parametrize("grid,blocks,lo,hi", [((24, 20, 12), (2, 2, 1), 0.1, 10.0),
                                               ((36, 20, 16), (3, 3, 3), 0.01, 100.0),
                                               ((64, 64, 64), (2, 2, 1), 0.1, 10.0)])
def test_float_float_update_matches_the_oracle_residual(grid, blocks, lo, hi):
    op = O.assemble(grid, blocks)
    B = 3
    mu = inputs.log_uniform(97, B, op.Q, lo, hi)
    # u0: the oracle's solutions rounded to FP32 (the magnitudes a solve meets); d: a correction
    U = np.stack([O.pcg(op, mu[b], tol=1e-6).u for b in range(B)])
    u0 = U.astype(np.float32).astype(np.float64)
    d = (1e-3 * np.abs(U).max() * inputs.random_field(98, (B, op.n))).astype(np.float32)
    with rbws.Problem(grid, blocks) as P:
        u_out = torch.empty((B, op.n), dtype=torch.float64, device="cuda")
        r_out = torch.empty_like(u_out)
        rbws.rbws_update_ff(P.h, mu, torch.from_numpy(u0).cuda(), torch.from_numpy(d).cuda(), u_out, r_out)
        ug, rg = u_out.cpu().numpy(), r_out.cpu().numpy()
    ut = u0 + d.astype(np.float64)  # the sum of two floats, rounded once
    # u = hi + lo goes to FP64 with integer operations: within one unit in the last place
    assert np.all(np.abs(ug - ut) <= 2.0 ** -52 * np.abs(ut))
    for b in range(B):
        val = op.values(mu[b])
        absA = sp.csr_matrix((np.abs(val), op.col, op.row_ptr))
        r_ref = np.ones(op.n) - op.matvec(mu[b], ut[b])
        scale = absA @ (np.abs(u0[b]) + np.abs(d[b]).astype(np.float64)) + 1.0
        err = np.abs(rg[b] - r_ref) / scale
        print("%s: max |r_ff - r_csr| / (|A|(|u0|+|d|) + |f|) = %.2e" % (grid, err.max()))
        assert err.max() <= 1e-13


@pytest.mark.parametrize("precond", [rbws.PREC_MG, rbws.PREC_JACOBI])
def test_float_float_and_fp64_updates_reach_the_oracle_solution(precond):
    grid, blocks = (48, 40, 36), (2, 2, 1)
    mu = inputs.log_uniform(99, 6, 4, 0.1, 10.0)
    U_ref = OB.reference_solutions(grid, mu, blocks=blocks, tol=1e-13, processes=2)[0]
    its = {}
    with rbws.Problem(grid, blocks) as P:
        u = torch.empty((6, P.n), dtype=torch.float64, device="cuda")
        for mode in (1, 2):
            opt = rbws.rbws_options_default(precision=rbws.FP32_IR, precond=precond, ru_mode=mode)
            rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, 1e-10, rbws.WARM_ZERO, u, opt)
            assert rc == 0 and np.all(st == 0)
            es = OB.error_summary(grid, mu, u.cpu().numpy(), U_ref, blocks=blocks)
            assert es["true_relres_max"] < 1e-10, mode
            assert es["relL2_max"] <= 1e-8, mode
            its[mode] = it
    print("iterations, FP64 updates", its[1].tolist(), "float-float updates", its[2].tolist())
    assert np.all(np.abs(its[1] - its[2]) <= 2)
