"""Pins of the oracle's PCG (Algorithm 1, with Algorithm 4's true-residual check)."""
import numpy as np
import pytest

import oracle as O
from paper_2311_13862_gb300 import inputs


def sine_mode(n, a, b, c):
    h = 1.0 / (n + 1)
    i = np.arange(1, n + 1)
    return np.einsum("k,j,i->kji", np.sin(c * np.pi * i * h), np.sin(b * np.pi * i * h),
                     np.sin(a * np.pi * i * h)).ravel()


def closed_form_unit_source(n, m):
    """u for f = 1 and kappa = m, from the discrete sine expansion of the constant vector:
    1 = sum_{a odd} (2/(n+1)) cot(a pi h / 2) sin(a pi i h) per axis."""
    h = 1.0 / (n + 1)
    i = np.arange(1, n + 1)
    odd = np.arange(1, n + 1, 2)
    s = 2.0 / (n + 1) / np.tan(odd * np.pi * h / 2)
    S = np.sin(np.outer(odd, i) * np.pi * h)              # [mode][node]
    e = 4.0 / h**2 * np.sin(odd * np.pi * h / 2) ** 2     # 1-D eigenvalues
    lam = m * (e[:, None, None] + e[None, :, None] + e[None, None, :])  # [c][b][a]
    coef = s[:, None, None] * s[None, :, None] * s[None, None, :] / lam
    return np.einsum("cba,ck,bj,ai->kji", coef, S, S, S).ravel()


@pytest.mark.parametrize("grid,blocks", [((4, 4, 4), (2, 1, 1)), ((6, 5, 7), (2, 2, 2)),
                                         ((8, 8, 8), (3, 3, 3))])
@pytest.mark.parametrize("precond", [O.PREC_NONE, O.PREC_JACOBI])
def test_matches_dense_direct_solve(grid, blocks, precond):
    op = O.assemble(grid, blocks)
    mu = inputs.log_uniform(21, 1, op.Q, 0.01, 100)[0]
    f = inputs.random_field(22, op.n)
    x = np.linalg.solve(op.dense(mu), f)
    r = O.pcg(op, mu, f=f, precond=precond, tol=1e-14)
    assert r.status == O.CONVERGED
    assert np.linalg.norm(r.u - x) <= 1e-12 * np.linalg.norm(x) * 10  # cond(A) <~ 1e3 here


def test_one_iteration_for_an_eigenvector():
    n, m = 8, 3.0
    v = sine_mode(n, 2, 1, 3)
    op = O.assemble((n, n, n), (2, 1, 1))
    r = O.pcg(op, [m, m], f=v, precond=O.PREC_NONE, tol=1e-13)
    h = 1.0 / (n + 1)
    lam = 4 * m / h**2 * sum(np.sin(k * np.pi * h / 2) ** 2 for k in (2, 1, 3))
    assert r.iters == 1
    assert np.linalg.norm(r.u - v / lam) <= 1e-14 * np.linalg.norm(v / lam)
    # Jacobi with constant kappa scales the residual uniformly: still one iteration
    rj = O.pcg(op, [m, m], f=v, precond=O.PREC_JACOBI, tol=1e-13)
    assert rj.iters == 1
    # the residual history: ||f|| / ||f|| = 1 from u0 = 0, then the exact solve
    assert r.hist[0] == 1.0 and r.hist[1] < 1e-14 and len(r.hist) == 2


def test_residual_history_entries():
    # entry 0 is the initial residual of the given u0 (recomputed here with the CSR operator),
    # the last one the reported residual, one entry per application of A
    op = O.assemble((10, 9, 8), (2, 2, 1))
    mu = inputs.log_uniform(91, 1, 4, 0.1, 10.0)[0]
    u0 = inputs.random_field(92, op.n)
    r = O.pcg(op, mu, u0=u0, precond=O.PREC_NONE, tol=1e-12)
    f = np.ones(op.n)
    assert r.hist[0] == pytest.approx(np.linalg.norm(f - op.matvec(mu, u0)) / np.linalg.norm(f), rel=1e-14)
    assert r.hist[-1] == pytest.approx(r.relres, rel=1e-6) and len(r.hist) == r.iters + 1
    assert np.all(r.hist > 0) and r.hist[-1] < 1e-12


def test_closed_form_solution_unit_source():
    n, m = 16, 1.7
    op = O.assemble((n, n, n), (2, 1, 1))
    r = O.pcg(op, [m, m], precond=O.PREC_NONE, tol=1e-14)
    u = closed_form_unit_source(n, m)
    assert np.linalg.norm(r.u - u) <= 1e-11 * np.linalg.norm(u)


def test_mu_homogeneity_bitwise():
    # u(t mu) = u(mu)/t; with t = 2 every CG quantity scales by an exact power of two
    op = O.assemble((16, 16, 16), (2, 1, 1))
    mu = np.array([0.37, 4.1])
    a = O.pcg(op, mu, precond=O.PREC_NONE, tol=1e-12)
    b = O.pcg(op, 2 * mu, precond=O.PREC_NONE, tol=1e-12)
    assert a.iters == b.iters
    assert np.array_equal(a.u, 2 * b.u)
    assert np.array_equal(a.hist, b.hist)


def test_mirror_symmetry_half_cubes():
    # kappa = (a, b) on x < 1/2, x > 1/2  <=>  (b, a) mirrored in x; also y <-> z and y -> 1-y.
    # n even so that n+1 is odd and no node sits on the interface x = 1/2.
    n = 12
    op = O.assemble((n, n, n), (2, 1, 1))
    ua = O.pcg(op, [0.3, 5.0], tol=1e-14).u.reshape(n, n, n)
    ub = O.pcg(op, [5.0, 0.3], tol=1e-14).u.reshape(n, n, n)
    s = np.linalg.norm(ua)
    assert np.linalg.norm(ua - ub[:, :, ::-1]) <= 1e-12 * s
    assert np.linalg.norm(ua - ua.transpose(1, 0, 2)) <= 1e-12 * s  # swap (z, y)
    assert np.linalg.norm(ua - ua[:, ::-1, :]) <= 1e-12 * s


def test_cg_a_norm_error_monotone():
    op = O.assemble((6, 5, 4), (2, 2, 1))
    mu = np.array([0.2, 7.0, 1.5, 0.6])
    A = op.dense(mu)
    x = np.linalg.solve(A, np.ones(op.n))
    errs = []
    for k in range(1, 25):
        r = O.pcg(op, mu, precond=O.PREC_JACOBI, tol=0.0, max_iters=k, max_restarts=0)
        e = r.u - x
        errs.append(e @ A @ e)
        if errs[-1] < 1e-24 * (x @ A @ x):
            break
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) for i in range(len(errs) - 1))


def test_warm_start_at_solution_takes_zero_iterations():
    op = O.assemble((5, 5, 5), (2, 1, 1))
    x = np.linalg.solve(op.dense([1.0, 2.0]), np.ones(op.n))
    r = O.pcg(op, [1.0, 2.0], u0=x, tol=1e-10)
    assert r.iters == 0 and r.status == O.CONVERGED


def test_breakdown_and_max_iters_status():
    op = O.assemble((6, 6, 6), (2, 1, 1))
    r = O.pcg(op, [1.0, 2.0], tol=1e-14, max_iters=3, max_restarts=0)
    assert r.status == O.MAX_ITERS and r.iters == 3
