"""The mu-interleaved layout [nz][ny][nx][B] of the operator apply (an alternative the
autotuner times against the planar layout of the solvers): against the oracle's CSR, and
bit for bit against the planar apply transposed (the same terms in the same order)."""
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


@pytest.mark.parametrize("grid,blocks,B", [((9, 7, 5), (2, 1, 1), 3), ((33, 17, 20), (2, 2, 2), 37),
                                           ((64, 64, 64), (2, 2, 1), 64)])
def test_interleaved_apply_matches_csr_and_planar(grid, blocks, B):
    op = O.assemble(grid, blocks)
    mu = inputs.log_uniform(401, B, op.Q, 0.01, 100.0)
    x = inputs.random_field(402, (B, op.n))
    with rbws.Problem(grid, blocks) as P:
        for prec, dt, tol in ((rbws.FP64, torch.float64, 1e-14), (rbws.FP32_IR, torch.float32, 1e-5)):
            xp = torch.from_numpy(x).cuda().to(dt)
            yp = torch.empty_like(xp)
            rbws.rbws_apply_operator(P.h, mu, xp, yp, prec)
            xi = xp.t().contiguous()  # [n][B]
            yi = torch.empty_like(xi)
            rbws.rbws_apply_operator_interleaved(P.h, mu, xi, yi, prec)
            assert torch.equal(yi.t().contiguous(), yp)
            ref = np.stack([op.matvec(mu[b], xp[b].cpu().double().numpy()) for b in range(B)])
            scale = np.abs(ref).max(axis=1, keepdims=True)
            assert np.max(np.abs(yi.t().cpu().double().numpy() - ref) / scale) <= tol


def test_autotune_layout_times_both_layouts():
    with rbws.Problem((64, 64, 64), (2, 2, 1)) as P:
        for prec in (rbws.FP32_IR, rbws.FP64):
            tp, ti, lay = rbws.rbws_autotune_layout(P.h, 256, prec)
            print("64^3, 256 instances, %s: planar %.3f ms, interleaved %.3f ms" %
                  ("fp32" if prec == rbws.FP32_IR else "fp64", tp, ti))
            assert tp > 0 and ti > 0 and lay == (1 if ti < tp else 0)
