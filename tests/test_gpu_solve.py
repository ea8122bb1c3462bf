"""Parity of the batched CUDA PCG / RB warm start (Algorithms 1 and 4, Sec. 2.3) with the
oracle: solutions to rel-L2 1e-10 (both solved to 1e-12), iteration counts within 2."""
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


def solve(P, mu, tol, warm, **opt):
    u = torch.empty((len(mu), P.n), dtype=torch.float64, device="cuda")
    o = rbws.rbws_options_default(**opt)
    rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, tol, warm, u, o)
    return rc, it, rel, st, u.cpu().numpy()


def rel_l2(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.mark.parametrize("grid,blocks", [((9, 7, 5), (2, 1, 1)), ((16, 16, 16), (2, 1, 1)),
                                         ((33, 17, 20), (2, 2, 2)), ((37, 41, 29), (3, 3, 3))])
@pytest.mark.parametrize("precond", [rbws.PREC_NONE, rbws.PREC_JACOBI])
def test_zero_start_matches_oracle(grid, blocks, precond):
    op = O.assemble(grid, blocks)
    mu = inputs.log_uniform(51, 5, op.Q, 0.1, 10.0)
    ref = O.solve_batch(op, mu, warm=O.WARM_ZERO, precond=precond, tol=1e-12)
    with rbws.Problem(grid, blocks) as P:
        rc, it, rel, st, u = solve(P, mu, 1e-12, rbws.WARM_ZERO, precond=precond)
    assert rc == 0 and np.all(st == 0)
    assert np.all(rel < 1e-12)
    assert np.all(np.abs(it - ref.iters) <= 2), (it, ref.iters)
    assert np.all(rel_l2(u, ref.u) <= 1e-10)


def test_galerkin_warm_start_matches_oracle():
    w = inputs.small(grid=(24, 20, 18), blocks=(2, 2, 1), n_max=8, n_train=24, n_test=6)
    op = O.assemble(w.grid, w.blocks)
    basis = O.greedy(op, inputs.train_mu(w), w.n_max)
    mu = inputs.test_mu(w)
    ref = O.solve_batch(op, mu, warm=O.WARM_GALERKIN, basis=basis, tol=1e-12)
    with rbws.Problem(w.grid, w.blocks) as P:
        rbws.rbws_set_basis(P.h, basis.W, basis.ANq, basis.fN)
        c = rbws.rbws_reduced_solve(P.h, mu)
        for b in range(len(mu)):
            cr = O.rb_solve(basis.ANq, basis.fN, mu[b])
            assert np.linalg.norm(c[b] - cr) <= 1e-12 * np.linalg.norm(cr)
        rc, it, rel, st, u = solve(P, mu, 1e-12, rbws.WARM_GALERKIN)
    assert rc == 0 and np.all(st == 0)
    assert np.all(np.abs(it - ref.iters) <= 2), (it, ref.iters)
    assert np.all(rel_l2(u, ref.u) <= 1e-10)


def test_warm_start_exact_for_one_subdomain():
    # p = 1: the one-vector basis reproduces u(mu) = u(1)/mu, so no iteration is needed
    op = O.assemble((12, 10, 9), (1, 1, 1))
    basis = O.greedy(op, np.array([[1.0], [3.0]]), 2, snapshot_tol=1e-13)
    with rbws.Problem((12, 10, 9), (1, 1, 1)) as P:
        rbws.rbws_set_basis(P.h, basis.W, basis.ANq, basis.fN)
        rc, it, rel, st, u = solve(P, np.array([[0.3], [7.0]]), 1e-10, rbws.WARM_GALERKIN)
    assert rc == 0 and np.all(it == 0) and np.all(rel < 1e-10)


def test_max_iters_reports_warning_and_status():
    op = O.assemble((16, 16, 16), (2, 1, 1))
    with rbws.Problem((16, 16, 16), (2, 1, 1)) as P:
        rc, it, rel, st, u = solve(P, np.array([[1.0, 5.0]]), 1e-12, rbws.WARM_ZERO, max_iters=5)
    assert rc == rbws.RBWS_WARN_NOT_CONVERGED and st[0] == 1 and it[0] == 5
    ref = O.pcg(op, [1.0, 5.0], tol=1e-12, max_iters=5, max_restarts=0)
    assert rel[0] == pytest.approx(np.linalg.norm(np.ones(op.n) - op.matvec([1.0, 5.0], ref.u))
                                   / np.sqrt(op.n), rel=1e-6)


def test_warm_mode_without_basis_is_an_error():
    with rbws.Problem((8, 8, 8), (2, 1, 1)) as P:
        with pytest.raises(rbws.RbwsError, match="NO_BASIS"):
            solve(P, np.array([[1.0, 2.0]]), 1e-10, rbws.WARM_GALERKIN)


@pytest.mark.parametrize("grid,blocks", [((40, 36, 32), (2, 2, 2)),   # 4-node kernels, ragged tiles
                                         ((33, 17, 20), (2, 2, 2)),   # nx % 4 != 0: 1-node kernels
                                         ((64, 48, 40), (2, 2, 1)),   # 4-node kernels, full tiles
                                         ((16, 16, 16), (2, 1, 1))])
def test_fp32_refinement_reaches_fp64_residual(grid, blocks):
    op = O.assemble(grid, blocks)
    mu = inputs.log_uniform(61, 4, op.Q, 0.01, 100.0)
    ref = O.solve_batch(op, mu, warm=O.WARM_ZERO, tol=1e-13)
    with rbws.Problem(grid, blocks) as P:
        rc, it, rel, st, u = solve(P, mu, 1e-10, rbws.WARM_ZERO, precision=rbws.FP32_IR)
    assert rc == 0 and np.all(st == 0)
    for b in range(len(mu)):
        true_rel = np.linalg.norm(np.ones(op.n) - op.matvec(mu[b], u[b])) / np.sqrt(op.n)
        assert true_rel < 1e-10
        assert rel[b] == pytest.approx(true_rel, rel=1e-6)
    # error against the FP64 oracle is bounded by cond(A) * 1e-10
    assert np.all(rel_l2(u, ref.u) <= 1e-7)


def test_reruns_are_bitwise_deterministic():
    grid, blocks = (33, 17, 20), (2, 2, 2)
    mu = inputs.log_uniform(71, 3, 8, 0.1, 10.0)
    with rbws.Problem(grid, blocks) as P:
        a = solve(P, mu, 1e-11, rbws.WARM_ZERO)
        b = solve(P, mu, 1e-11, rbws.WARM_ZERO)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[4], b[4])


@pytest.mark.parametrize("grid,blocks,n_max", [((16, 16, 16), (2, 1, 1), 6), ((24, 20, 18), (2, 2, 1), 8)])
def test_msrb_preconditioned_start_matches_oracle(grid, blocks, n_max):
    """RB-preconditioned arm: Galerkin start, then PCG with the MSRB preconditioner
    (Algorithm 3, same W at every iteration).  Iteration counts within 2; converged
    solutions agree to 1e-10; non-converged ones report the same status."""
    w = inputs.small(grid=grid, blocks=blocks, n_max=n_max, n_train=24, n_test=4)
    op = O.assemble(w.grid, w.blocks)
    basis = O.greedy(op, inputs.train_mu(w), w.n_max)
    mu = inputs.test_mu(w)
    ref = O.solve_batch(op, mu, warm=O.WARM_GALERKIN, basis=basis, precond=O.PREC_MSRB, tol=1e-12,
                        max_iters=400)
    with rbws.Problem(w.grid, w.blocks) as P:
        rbws.rbws_set_basis(P.h, basis.W, basis.ANq, basis.fN)
        rc, it, rel, st, u = solve(P, mu, 1e-12, rbws.WARM_GALERKIN, precond=rbws.PREC_MSRB, max_iters=400)
    assert np.array_equal(st, ref.status), (st, ref.status)
    conv = st == 0
    assert np.all(np.abs(it[conv] - ref.iters[conv]) <= 2), (it, ref.iters)
    if conv.any():
        assert np.all(rel_l2(u[conv], ref.u[conv]) <= 1e-10)


def test_msrb_without_basis_is_an_error():
    with rbws.Problem((8, 8, 8), (2, 1, 1)) as P:
        with pytest.raises(rbws.RbwsError, match="NO_BASIS"):
            solve(P, np.array([[1.0, 2.0]]), 1e-10, rbws.WARM_ZERO, precond=rbws.PREC_MSRB)


def test_checkpoint_round_trip(tmp_path):
    """rbws_save after the offline stage (greedy + network), rbws_load in a new problem: the
    online solves are bitwise identical."""
    w = inputs.small(grid=(20, 16, 12), blocks=(2, 2, 1), n_max=6, n_train=16, n_test=4)
    mu = inputs.test_mu(w)
    path = tmp_path / "offline.rbws"
    with rbws.Problem(w.grid, w.blocks) as P:
        rbws.rbws_offline_greedy(P.h, inputs.train_mu(w), w.n_max)
        rbws.rbws_train_surrogate(P.h, inputs.surrogate_mu(w, 256), hidden=32, epochs=20, batch=64,
                                  mu_lo=w.mu_lo, mu_hi=w.mu_hi)
        a = {m: solve(P, mu, 1e-10, m) for m in (rbws.WARM_GALERKIN, rbws.WARM_LEARNED)}
        rbws.rbws_save(P.h, path)
    with rbws.Problem.load(path) as P2:
        b = {m: solve(P2, mu, 1e-10, m) for m in (rbws.WARM_GALERKIN, rbws.WARM_LEARNED)}
    for m in a:
        assert np.array_equal(a[m][1], b[m][1]) and np.array_equal(a[m][4], b[m][4])
