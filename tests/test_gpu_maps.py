"""Explicit subdomain maps (Eq. 1 with kappa = mu_q on an arbitrary map of subdomains): the
CUDA operator, solves and checkpoints against the oracle assembled from the same map."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2311_13862_gb300 import inputs, rbws

pytestmark = pytest.mark.gpu

GRIDS = [(16, 16, 16), (37, 29, 21), (40, 36, 32)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2311_13862_gb300 import build
    build.build()


def rel_l2(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("precision", [rbws.FP64, rbws.FP32_IR])
def test_apply_with_an_inclusion_map_matches_csr(grid, precision):
    m = inputs.inclusion_map(grid, 5)
    op = O.assemble(grid, submap=m, Q=3)
    B = 3
    mu = inputs.log_uniform(81, B, 3, 0.01, 100.0)
    x = inputs.random_field(82, (B, op.n))
    ref = np.stack([op.matvec(mu[b], x[b]) for b in range(B)])
    dt = torch.float64 if precision == rbws.FP64 else torch.float32
    with rbws.Problem(grid, subdomain_map=m, Q=3) as P:
        xd = torch.from_numpy(x).to(dt).cuda()
        yd = torch.empty_like(xd)
        rbws.rbws_apply_operator(P.h, mu, xd, yd, precision)
        y = yd.double().cpu().numpy()
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.max(np.abs(y - ref) / scale) <= (1e-14 if precision == rbws.FP64 else 2e-6)


def test_block_rule_given_as_a_map_is_bitwise_the_block_problem():
    grid, blocks = (37, 41, 29), (3, 3, 3)
    m = O.block_map(grid, blocks)
    mu = inputs.log_uniform(83, 2, 27, 0.1, 10.0)
    x = torch.from_numpy(inputs.random_field(84, (2, grid[0] * grid[1] * grid[2]))).cuda()
    ys = []
    for kw in (dict(blocks=blocks), dict(subdomain_map=m, Q=27)):
        with rbws.Problem(grid, **kw) as P:
            y = torch.empty_like(x)
            rbws.rbws_apply_operator(P.h, mu, x, y, rbws.FP64)
            ys.append(y.cpu().numpy())
    assert np.array_equal(ys[0], ys[1])


def test_greedy_and_warm_start_with_an_inclusion_map_match_oracle():
    grid = (16, 16, 16)
    m = inputs.inclusion_map(grid, 5)
    op = O.assemble(grid, submap=m, Q=3)
    mus = inputs.log_uniform(85, 24, 3, 0.1, 10.0)
    mu = inputs.log_uniform(86, 4, 3, 0.1, 10.0)
    ref_basis = O.greedy(op, mus, 6)
    ref = O.solve_batch(op, mu, warm=O.WARM_GALERKIN, basis=ref_basis, tol=1e-12)
    with rbws.Problem(grid, subdomain_map=m, Q=3) as P:
        N, sel, eta = rbws.rbws_offline_greedy(P.h, mus, 6, 0.0, 1e-12)
        assert N == ref_basis.N and list(sel[:N]) == list(ref_basis.selected)
        assert np.allclose(eta, ref_basis.eta_hist, rtol=1e-6, atol=1e-12)
        u = torch.empty((len(mu), P.n), dtype=torch.float64, device="cuda")
        rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, 1e-12, rbws.WARM_GALERKIN, u,
                                                rbws.rbws_options_default())
        u = u.cpu().numpy()
    assert rc == 0 and np.all(st == 0)
    assert np.all(np.abs(it - ref.iters) <= 2), (it, ref.iters)
    assert np.all(rel_l2(u, ref.u) <= 1e-10)


def test_fp32_refinement_with_a_map_reaches_the_fp64_residual():
    grid = (40, 36, 32)
    m = inputs.inclusion_map(grid, 7)
    op = O.assemble(grid, submap=m, Q=3)
    mu = inputs.log_uniform(87, 3, 3, 0.01, 100.0)
    with rbws.Problem(grid, subdomain_map=m, Q=3) as P:
        u = torch.empty((len(mu), P.n), dtype=torch.float64, device="cuda")
        rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, 1e-10, rbws.WARM_ZERO, u,
                                                rbws.rbws_options_default(precision=rbws.FP32_IR))
        u = u.cpu().numpy()
    assert rc == 0 and np.all(st == 0)
    for b in range(len(mu)):
        true_rel = np.linalg.norm(np.ones(op.n) - op.matvec(mu[b], u[b])) / np.sqrt(op.n)
        assert true_rel < 1e-10


def test_checkpoint_keeps_the_map(tmp_path):
    grid = (16, 16, 16)
    m = inputs.inclusion_map(grid, 5)
    mus = inputs.log_uniform(85, 16, 3, 0.1, 10.0)
    mu = inputs.log_uniform(88, 2, 3, 0.1, 10.0)
    x = torch.from_numpy(inputs.random_field(89, (2, 16 ** 3))).cuda()
    path = str(tmp_path / "map.rbws")
    with rbws.Problem(grid, subdomain_map=m, Q=3) as P:
        rbws.rbws_offline_greedy(P.h, mus, 4, 0.0, 1e-12)
        y1 = torch.empty_like(x)
        rbws.rbws_apply_operator(P.h, mu, x, y1, rbws.FP64)
        c1 = rbws.rbws_reduced_solve(P.h, mu)
        rbws.rbws_save(P.h, path)
    with rbws.Problem.load(path) as P2:
        assert P2.Q == 3
        y2 = torch.empty_like(x)
        rbws.rbws_apply_operator(P2.h, mu, x, y2, rbws.FP64)
        c2 = rbws.rbws_reduced_solve(P2.h, mu)
    assert torch.equal(y1, y2)
    assert np.array_equal(c1, c2)
