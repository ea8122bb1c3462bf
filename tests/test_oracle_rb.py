"""Pins of the oracle's reduced basis parts: the Galerkin RB system (Sec. 2.3), the greedy
(Algorithm 5 skeleton), the warm start (Algorithm 4) and the MSRB preconditioner (Algorithm 3)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2311_13862_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def c1_small():
    w = inputs.small(grid=(10, 9, 8), blocks=(2, 2, 1), n_max=8, n_train=24, n_test=6)
    op = O.assemble(w.grid, w.blocks)
    basis = O.greedy(op, inputs.train_mu(w), w.n_max, snapshot_tol=1e-13)
    return w, op, basis


def test_orthonormal_basis(c1_small):
    _, _, b = c1_small
    assert b.N == 8
    assert np.max(np.abs(b.W @ b.W.T - np.eye(b.N))) <= 1e-13


def test_reduced_operators_are_projections(c1_small):
    _, op, b = c1_small
    for q in range(op.Q):
        e = np.eye(op.Q)[q]
        AW = np.stack([op.matvec(e, w) for w in b.W])
        assert np.max(np.abs(b.ANq[q] - b.W @ AW.T)) <= 1e-12 * np.max(np.abs(b.ANq[q]))
    assert np.allclose(b.fN, b.W @ np.ones(op.n), rtol=1e-13, atol=0)


def test_galerkin_orthogonality_and_reduced_solve(c1_small):
    w, op, b = c1_small
    for mu in inputs.test_mu(w):
        c = O.rb_solve(b.ANq, b.fN, mu)
        AN = np.tensordot(mu, b.ANq, axes=1)
        assert np.linalg.norm(c - np.linalg.solve(AN, b.fN)) <= 1e-12 * np.linalg.norm(c)
        res = np.ones(op.n) - op.matvec(mu, b.W.T @ c)
        assert np.max(np.abs(b.W @ res)) <= 1e-12 * np.linalg.norm(np.ones(op.n))


def test_snapshot_reproduction(c1_small):
    w, op, b = c1_small
    mus = inputs.train_mu(w)
    for k, idx in enumerate(b.selected):
        mu = mus[idx]
        snap = O.pcg(op, mu, tol=1e-13).u
        c = O.rb_solve(b.ANq, b.fN, mu)
        assert np.linalg.norm(b.W.T @ c - snap) <= 1e-8 * np.linalg.norm(snap)


def test_a_norm_error_non_increasing_in_N(c1_small):
    w, op, b = c1_small
    for mu in inputs.test_mu(w)[:3]:
        A = op.dense(mu) if op.n <= 1000 else None
        x = np.linalg.solve(A, np.ones(op.n))
        errs = []
        for N in range(1, b.N + 1):
            c = O.rb_solve(b.ANq[:, :N, :N], b.fN[:N], mu)
            e = b.W[:N].T @ c - x
            errs.append(e @ A @ e)
        assert all(errs[i + 1] <= errs[i] * (1 + 1e-8) + 1e-28 for i in range(len(errs) - 1))


def test_indicator_is_relative_residual_and_argmax(c1_small):
    w, op, b = c1_small
    mus = inputs.train_mu(w)
    # the history's last value is the max over unselected points of the residual indicator
    etas = [O.rb_indicator(op, b, mus[t]) if t not in set(b.selected) else -1 for t in range(len(mus))]
    assert b.eta_hist[-1] == pytest.approx(max(etas), rel=1e-12)


def test_one_subdomain_is_exact_with_one_vector():
    # p = 1: u(mu) = u(1)/mu, so N = 1 is exact and the greedy stops at breakdown
    op = O.assemble((7, 6, 5), (1, 1, 1))
    mus = np.array([[0.5], [3.0], [7.0], [0.2]])
    b = O.greedy(op, mus, 4, snapshot_tol=1e-13)
    assert b.N == 1
    assert np.all(b.eta_hist[0] < 1e-11)
    r = O.solve_batch(op, [[2.2], [0.15]], warm=O.WARM_GALERKIN, basis=b, tol=1e-10)
    assert np.all(r.iters == 0)


def test_warm_start_initial_residual_equals_indicator_and_saves_iterations(c1_small):
    w, op, b = c1_small
    mus = inputs.test_mu(w)
    z = O.solve_batch(op, mus, warm=O.WARM_ZERO, tol=1e-12, n_threads=2)
    g = O.solve_batch(op, mus, warm=O.WARM_GALERKIN, basis=b, tol=1e-12, n_threads=2)
    for i, mu in enumerate(mus):
        assert g.relres0[i] == pytest.approx(O.rb_indicator(op, b, mu), rel=1e-9)
    assert np.all(z.relres0 == pytest.approx(1.0))
    assert np.all(g.iters <= z.iters)
    assert np.all(g.status == O.CONVERGED) and np.all(z.status == O.CONVERGED)
    # both reach the same solution
    assert np.max(np.linalg.norm(g.u - z.u, axis=1) / np.linalg.norm(z.u, axis=1)) <= 1e-9


def test_paper_trend_warm_start_fewer_iterations_as_N_grows():
    """Table 2 (Example 1, delta = 1e-16) prints 20 iterations from zero and 13/9/5 from RB
    starts with N = 10/15/20: fewer iterations for a larger basis.  Same trend here."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_table2_example1.txt"))
            if l.strip() and not l.startswith("#")]
    paper = {r[0] + ":" + r[1]: int(r[2]) for r in rows}
    assert paper["MGCG:-"] > paper["RBI-MGCG:10"] > paper["RBI-MGCG:15"] > paper["RBI-MGCG:20"]
    w = inputs.small(grid=(12, 12, 12), blocks=(2, 1, 1), n_max=10, n_train=32)
    op = O.assemble(w.grid, w.blocks)
    b = O.greedy(op, inputs.train_mu(w), w.n_max, snapshot_tol=1e-13)
    mus = inputs.test_mu(w, 6)
    it = [O.solve_batch(op, mus, warm=O.WARM_ZERO, tol=1e-12, n_threads=2).iters.mean()]
    for N in (5, 10):
        bN = O.Basis(b.W[:N], b.ANq[:, :N, :N], b.fN[:N], b.selected[:N], b.eta_hist[:N], N)
        it.append(O.solve_batch(op, mus, warm=O.WARM_GALERKIN, basis=bN, tol=1e-12,
                                n_threads=2).iters.mean())
    assert it[0] > it[1] > it[2]


def test_msrb_with_complete_basis_is_an_exact_solver():
    """Algorithm 3 with W spanning R^n: s = D^-1 b + A^-1 (b - A D^-1 b) = A^-1 b, so PCG
    with this preconditioner converges in one iteration."""
    op = O.assemble((3, 2, 2), (2, 1, 1))
    mu = np.array([0.7, 3.0])
    A = op.dense(mu)
    W = np.eye(op.n)
    L = O.cholesky(W @ A @ W.T)
    f = inputs.random_field(3, op.n)
    r = O.pcg(op, mu, f=f, precond=O.PREC_MSRB, msrb=(W, L), tol=1e-13)
    assert r.iters == 1
    assert np.linalg.norm(r.u - np.linalg.solve(A, f)) <= 1e-13 * np.linalg.norm(r.u)


def test_msrb_with_empty_correction_is_jacobi():
    """Algorithm 3 with a basis orthogonal to everything the residual touches reduces to one
    Jacobi sweep; a basis vector supported on a single node far from f's support changes
    nothing when f vanishes near it... use instead W = 0 (a zero vector, A_N = [1])."""
    op = O.assemble((5, 4, 3), (2, 1, 1))
    mu = np.array([0.7, 3.0])
    W = np.zeros((1, op.n))
    L = np.ones((1, 1))
    f = inputs.random_field(4, op.n)
    a = O.pcg(op, mu, f=f, precond=O.PREC_MSRB, msrb=(W, L), tol=1e-12)
    b = O.pcg(op, mu, f=f, precond=O.PREC_JACOBI, tol=1e-12)
    assert a.iters == b.iters
    assert np.array_equal(a.u, b.u)


def test_l1_indicator_is_coefficient_norm_in_the_snapshot_basis():
    """Sec. 3.1's indicator: the L1 norm of the RB solution's coefficients with respect to the
    unorthogonalised snapshots.  Recomputed here from the snapshots themselves (least squares
    of W c on U), independently of the Gram-Schmidt factor the oracle keeps."""
    w = inputs.small(grid=(10, 9, 8), blocks=(2, 2, 1), n_max=5, n_train=20)
    op = O.assemble(w.grid, w.blocks)
    mus = inputs.train_mu(w)
    b = O.greedy(op, mus, w.n_max, snapshot_tol=1e-13, indicator=1)
    assert b.N == 5
    U = np.stack([O.pcg(op, mus[i], tol=1e-13).u for i in b.selected]).T  # [n][N]
    vals = []
    for t in range(len(mus)):
        if t in set(b.selected):
            continue
        c = O.rb_solve(b.ANq, b.fN, mus[t])
        x, *_ = np.linalg.lstsq(U, b.W.T @ c, rcond=None)
        vals.append(np.abs(x).sum())
    assert b.eta_hist[-1] == pytest.approx(max(vals), rel=1e-6)
    # the first pick is index 0 whatever the indicator, later picks maximise the L1 norm
    assert b.selected[0] == 0


def test_rb_residual_of_a_subspace_is_the_dense_galerkin_residual(c1_small):
    """The r_N view (residual of the Galerkin RB solution with the first n vectors): the oracle's
    leading-block reduced solve equals a dense projection onto span(W[:n]) formed from scratch."""
    w, op, b = c1_small
    f = np.ones(op.n)
    for mu in inputs.test_mu(w)[:3]:
        A = op.dense(mu)
        for n in (1, 3, b.N):
            Wn = b.W[:n]
            c = np.linalg.solve(Wn @ A @ Wn.T, Wn @ f)
            ref = np.linalg.norm(f - A @ (Wn.T @ c)) / np.linalg.norm(f)
            assert O.rb_indicator(op, b, mu, n_use=n) == pytest.approx(ref, rel=1e-9)
    with pytest.raises(ValueError):
        O.rb_indicator(op, b, inputs.test_mu(w)[0], n_use=b.N + 1)


def test_rb_residual_vanishes_at_the_selected_parameters(c1_small):
    """Exact reproduction: with all N vectors, the RB solution at a selected training parameter is
    its snapshot, so the residual is at the snapshot tolerance's level."""
    w, op, b = c1_small
    mus = inputs.train_mu(w)
    for t in b.selected:
        assert O.rb_indicator(op, b, mus[t]) < 1e-9
