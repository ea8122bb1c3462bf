"""The residual-manifold experiment of Sec. 5: the singular values of the residuals of the
RB-initialised PCG after k iterations (a POD of the residual snapshots), GPU against oracle."""
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


def pod_values(R):
    """Singular values of the snapshot matrix (rows = residuals), largest first, relative."""
    s = np.linalg.svd(np.asarray(R), compute_uv=False)
    return s / s[0]


def test_residual_pod_matches_oracle():
    grid, blocks = (24, 20, 18), (2, 2, 1)
    w = inputs.small(grid=grid, blocks=blocks, n_max=6, n_train=24, n_test=16)
    op = O.assemble(grid, blocks)
    mus = inputs.test_mu(w)
    ref_basis = O.greedy(op, inputs.train_mu(w), w.n_max, snapshot_tol=1e-12)
    f = np.ones(op.n)
    with rbws.Problem(grid, blocks) as P:
        rbws.rbws_offline_greedy(P.h, inputs.train_mu(w), w.n_max, 0.0, 1e-12)
        for k in (0, 3, 8):
            u = torch.empty((len(mus), P.n), dtype=torch.float64, device="cuda")
            rbws.rbws_solve_batch(P.h, mus, 1e-15, rbws.WARM_GALERKIN, u,
                                  rbws.rbws_options_default(max_iters=k))
            au = torch.empty_like(u)
            rbws.rbws_apply_operator(P.h, mus, u, au)
            R = (torch.ones_like(u) - au).cpu().numpy()
            Rref = []
            for mu in mus:
                u0 = ref_basis.W.T @ O.rb_solve(ref_basis.ANq, ref_basis.fN, mu)
                uk = O.pcg(op, mu, u0=u0, tol=1e-15, max_iters=k).u
                Rref.append(f - op.matvec(mu, uk))
            got, exp = pod_values(R), pod_values(np.array(Rref))
            assert np.allclose(got[:10], exp[:10], rtol=1e-6, atol=1e-12), (k, got[:10], exp[:10])
