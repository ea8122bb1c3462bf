"""Full-size workloads: the 128^3 high-contrast octant problem (FP32 PCG inside FP64
refinement, RB warm start, N <= 40, 64 parameters) and a 96^3 grid with 27 blocks.  Every GPU
solution's true residual is recomputed by the oracle's CSR operator in FP64; sampled
instances are compared with the oracle's own FP64 solution."""
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


def true_relres(op, mu, u):
    return np.linalg.norm(np.ones(op.n) - op.matvec(mu, u)) / np.sqrt(op.n)


def test_octants_128_high_contrast_fp32_refinement():
    w = inputs.WORKLOADS["c3"]
    op = O.assemble(w.grid, w.blocks)
    mu = inputs.test_mu(w)
    with rbws.Problem(w.grid, w.blocks) as P:
        N, sel, eta = rbws.rbws_offline_greedy(P.h, inputs.train_mu(w), w.n_max, 0.0, 1e-12)
        assert N == w.n_max and np.all(np.isfinite(eta))
        u = torch.empty((len(mu), P.n), dtype=torch.float64, device="cuda")
        rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, w.tol, rbws.WARM_GALERKIN, u,
                                                rbws.rbws_options_default(precision=rbws.FP32_IR))
        assert rc == 0 and np.all(st == 0), st
        u64 = torch.empty_like(u[:4])
        rc64, it64, rel64, st64 = rbws.rbws_solve_batch(P.h, mu[:4], 1e-12, rbws.WARM_GALERKIN, u64)
        assert rc64 == 0
        uh, u64h = u.cpu().numpy(), u64.cpu().numpy()
    for b in range(0, len(mu), 8):
        r = true_relres(op, mu[b], uh[b])
        assert r < w.tol and r == pytest.approx(rel[b], rel=1e-5)
    # error of the mixed-precision solutions against FP64 solves: bounded by cond(A) * tol
    err = np.linalg.norm(uh[:4] - u64h, axis=1) / np.linalg.norm(u64h, axis=1)
    print("c3 iterations mean %.1f max %d; rel-L2 vs FP64 %s" % (it.mean(), it.max(), np.array2string(err, precision=2)))
    assert np.all(err < 1e-5)
    # one instance against the oracle's own FP64 PCG
    ref = O.pcg(op, mu[0], tol=1e-11)
    assert np.linalg.norm(uh[0] - ref.u) / np.linalg.norm(ref.u) < 1e-5
    assert np.linalg.norm(u64h[0] - ref.u) / np.linalg.norm(ref.u) < 1e-9


def test_grid_96_with_27_blocks():
    w = inputs.WORKLOADS["c5-96"]
    op = O.assemble(w.grid, w.blocks)
    mu = inputs.test_mu(w, 16)
    with rbws.Problem(w.grid, w.blocks) as P:
        N, sel, eta = rbws.rbws_offline_greedy(P.h, inputs.train_mu(w, 64), 20, 0.0, 1e-12)
        u = torch.empty((len(mu), P.n), dtype=torch.float64, device="cuda")
        for prec in (rbws.FP32_IR, rbws.FP64):
            rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, w.tol, rbws.WARM_GALERKIN, u,
                                                    rbws.rbws_options_default(precision=prec))
            assert rc == 0 and np.all(st == 0)
            uh = u.cpu().numpy()
            for b in (0, 7, 15):
                assert true_relres(op, mu[b], uh[b]) < w.tol


def test_plain_method_16cube_two_halves():
    """The plain method at 16^3: greedy RB (N <= 10) over 64 training parameters, then 8 test
    parameters solved by plain CG (no preconditioner) to rel-res 1e-12 from zero and from the
    RB warm start, against the oracle doing the same."""
    w = inputs.WORKLOADS["c1"]
    op = O.assemble(w.grid, w.blocks)
    ref_basis = O.greedy(op, inputs.train_mu(w), w.n_max)
    mu = inputs.test_mu(w)
    opt = rbws.rbws_options_default(precond=rbws.PREC_NONE)
    with rbws.Problem(w.grid, w.blocks) as P:
        N, sel, eta = rbws.rbws_offline_greedy(P.h, inputs.train_mu(w), w.n_max, 0.0, 1e-12)
        assert N == ref_basis.N
        u = torch.empty((len(mu), P.n), dtype=torch.float64, device="cuda")
        res = {}
        for name, warm in [("zero", rbws.WARM_ZERO), ("warm", rbws.WARM_GALERKIN)]:
            rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, w.tol, warm, u, opt)
            assert rc == 0 and np.all(st == 0)
            res[name] = (it, u.cpu().numpy())
    z = O.solve_batch(op, mu, warm=O.WARM_ZERO, precond=O.PREC_NONE, tol=w.tol)
    g = O.solve_batch(op, mu, warm=O.WARM_GALERKIN, basis=ref_basis, precond=O.PREC_NONE, tol=w.tol)
    assert np.all(np.abs(res["zero"][0] - z.iters) <= 2)
    assert np.all(np.abs(res["warm"][0] - g.iters) <= 2)
    for (it, u), ref in ((res["zero"], z), (res["warm"], g)):
        assert np.all(np.linalg.norm(u - ref.u, axis=1) / np.linalg.norm(ref.u, axis=1) <= 1e-10)
    assert res["warm"][0].mean() < res["zero"][0].mean()
    print("16^3 plain CG iterations: zero", res["zero"][0].tolist(), "warm", res["warm"][0].tolist())
