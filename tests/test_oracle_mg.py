"""Pins of the oracle's multigrid V-cycle (Algorithm 2) and MGCG against facts fixed by the
mathematics: interpolation of linear functions, the Kronecker form of Galerkin coarse
operators for constant coefficients, symmetry and definiteness of the V-cycle, exactness of
the one-level cycle, direct solves, and mesh-independent iteration counts."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from oracle import mg
from paper_2311_13862_gb300 import inputs


@pytest.mark.parametrize("n", [7, 8, 9, 16])
def test_prolongation_interpolates_linear_functions(n):
    h = 1.0 / (n + 1)
    P = mg.prolongation_1d(n)
    m = n // 2
    assert P.shape == (n, m)
    xc = 2 * h * np.arange(1, m + 1)           # coarse nodes sit at fine nodes 2J
    xf = h * np.arange(1, n + 1)
    # g(x) = x vanishes on the lower boundary: exact at every fine node left of the last
    # coarse node; g(x) = 1 - x vanishes on the upper one: exact right of the first
    up = P @ xc
    assert np.allclose(up[: 2 * m], xf[: 2 * m], rtol=0, atol=1e-15)
    down = P @ (1 - xc)
    assert np.allclose(down[1:], 1 - xf[1:], rtol=0, atol=1e-15)


def test_galerkin_coarse_operator_has_the_kronecker_form():
    """Constant kappa: A = (T (x) I (x) I)/h^2 + ... with T = tridiag(-1, 2, -1).  Then
    P^T A P = sum over axes of (P^T T P) (x) (P^T P) (x) (P^T P) / h^2, built here from 1D
    factors only (independently of the 3D assembly and of the hierarchy code)."""
    grid = (10, 9, 8)
    m = 1.7
    op = O.assemble(grid, (1, 1, 1))
    H = mg.Hierarchy(op)
    assert H.J >= 1
    A1 = sum(m * A for A in H.Aq[H.J - 1])

    def T(n):
        return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])

    nx, ny, nz = grid
    Px, Py, Pz = (mg.prolongation_1d(k) for k in grid)
    hx2, hy2, hz2 = ((k + 1) ** 2 for k in grid)
    M = lambda P: P.T @ P
    G = lambda P, n: P.T @ T(n) @ P
    ref = m * (hx2 * sp.kron(M(Pz), sp.kron(M(Py), G(Px, nx)))
               + hy2 * sp.kron(M(Pz), sp.kron(G(Py, ny), M(Px)))
               + hz2 * sp.kron(G(Pz, nz), sp.kron(M(Py), M(Px))))
    d = (A1 - ref).toarray()
    assert np.max(np.abs(d)) <= 1e-12 * np.max(np.abs(ref.toarray()))


def test_level_rule():
    assert mg.level_grids((64, 64, 64)) == [(4, 4, 4), (8, 8, 8), (16, 16, 16), (32, 32, 32), (64, 64, 64)]
    assert mg.level_grids((4, 4, 4)) == [(4, 4, 4)]
    assert mg.level_grids((9, 7, 5)) == [(4, 3, 2), (9, 7, 5)]
    assert mg.level_grids((24, 20, 18)) == [(3, 2, 2), (6, 5, 4), (12, 10, 9), (24, 20, 18)]
    assert mg.level_grids((130, 9, 3)) == [(65, 4, 1), (130, 9, 3)]  # an axis reached 1 node


def test_vcycle_is_symmetric_positive_definite():
    op = O.assemble((24, 20, 18), (2, 2, 1))
    H = mg.Hierarchy(op)
    lv = H.operators(inputs.log_uniform(3, 1, 4, 0.01, 100.0)[0])
    x, y = inputs.random_field(4, (2, op.n))
    Mx, My = mg.vcycle(lv, x), mg.vcycle(lv, y)
    assert abs(x @ My - y @ Mx) <= 1e-12 * abs(x @ My)
    assert x @ Mx > 0 and y @ My > 0


def test_smoother_first_step_and_one_level_cycle():
    op = O.assemble((4, 4, 3), (2, 1, 1))
    mu = np.array([0.3, 4.0])
    H = mg.Hierarchy(op)
    assert H.J == 0
    lv = H.operators(mu)
    b = inputs.random_field(5, op.n)
    A = op.dense(mu)
    assert np.allclose(mg.smooth(lv.A[0], lv.dinv[0], b, None, 1), mg.OMEGA * b / np.diag(A), rtol=1e-15)
    # one level: MG is the exact solve, so MGCG converges in one iteration
    assert np.allclose(mg.vcycle(lv, b), np.linalg.solve(A, b), rtol=1e-11, atol=0)
    r = mg.mgcg(op, mu, tol=1e-12)
    assert r.iters == 1 and r.status == 0


@pytest.mark.parametrize("grid,blocks", [((24, 20, 18), (2, 2, 1)), ((16, 16, 16), (2, 1, 1))])
def test_mgcg_matches_direct_solve(grid, blocks):
    op = O.assemble(grid, blocks)
    mu = inputs.log_uniform(6, 1, op.Q, 0.01, 100.0)[0]
    r = mg.mgcg(op, mu, tol=1e-13)
    u = np.linalg.solve(op.dense(mu), np.ones(op.n))
    assert r.status == 0
    assert np.linalg.norm(r.u - u) <= 1e-10 * np.linalg.norm(u)
    assert r.iters < 25
    # error propagation of one V-cycle contracts: ||I - M A|| estimated by power iteration
    lv = mg.Hierarchy(op).operators(mu)
    e = inputs.random_field(7, op.n)
    for _ in range(15):
        e = e - mg.vcycle(lv, op.matvec(mu, e))
        e /= np.linalg.norm(e)
    e2 = e - mg.vcycle(lv, op.matvec(mu, e))
    assert np.linalg.norm(e2) < 0.5


def test_mgcg_iterations_do_not_grow_with_the_grid():
    # constant coefficient, p = 1: the V-cycle preconditioner is mesh-independent
    its = []
    for n in (15, 31):
        op = O.assemble((n, n, n), (1, 1, 1))
        its.append(mg.mgcg(op, [1.0], tol=1e-10).iters)
    assert its[1] <= its[0] + 3, its
    jac = O.pcg(O.assemble((31, 31, 31), (1, 1, 1)), [1.0], tol=1e-10).iters
    assert its[1] * 4 < jac


def test_batch_reference_solutions_match_direct_solves():
    """oracle.batch spreads MGCG solves over spawned workers on the directly assembled A(mu);
    each must equal a solve with the affine operator, and its own error summary is zero."""
    import oracle as O
    from oracle import batch
    grid, blocks = (12, 10, 8), (2, 2, 1)
    mus = inputs.log_uniform(91, 3, 4, 0.1, 10.0)
    U, its, rel, st, _, procs = batch.reference_solutions(grid, mus, blocks=blocks, tol=1e-12, processes=2)
    assert procs == 2 and np.all(st == 0) and np.all(rel < 1e-12)
    op = O.assemble(grid, blocks)
    for b in range(3):
        r = mg.mgcg(op, mus[b], tol=1e-12)
        assert np.linalg.norm(U[b] - r.u) <= 1e-11 * np.linalg.norm(r.u)
    s = batch.error_summary(grid, mus, U, U, blocks=blocks)
    assert s["relL2_max"] == 0.0 and s["true_relres_max"] < 1e-12
