"""Pins of the oracle's L1ROC (Sec. 3.1, Algorithm 5): the DEIM structure of the basis, the
snapshot factorisation U = W T, exact reproduction of the selected snapshots by the
over-collocation solve, the value of the L1 indicator there, and the one-subdomain case."""
import numpy as np
import pytest

import oracle as O
from oracle import l1roc
from paper_2311_13862_gb300 import inputs


@pytest.fixture(scope="module")
def built():
    w = inputs.small(grid=(14, 12, 10), blocks=(2, 2, 1), n_max=6, n_train=24)
    op = O.assemble(w.grid, w.blocks)
    mus = inputs.train_mu(w)
    return op, mus, l1roc.offline(op, mus, w.n_max)


def test_deim_vectors_are_unit_lower_triangular_at_their_points(built):
    op, mus, b = built
    assert b.N == 6 and len(set(b.pts_s.tolist())) == b.N
    M = b.W[:, b.pts_s].T           # M[i][j] = w_j at point i
    assert np.allclose(np.diag(M), 1.0, rtol=0, atol=1e-15)
    assert np.max(np.abs(np.triu(M, 1))) <= 1e-12   # w_j vanishes at the earlier points


def test_snapshots_factor_through_the_basis(built):
    op, mus, b = built
    for k, t in enumerate(b.selected):
        u = O.pcg(op, mus[t], tol=1e-12).u    # re-solved independently
        assert np.linalg.norm(b.W.T @ b.T[:, k] - u) <= 1e-9 * np.linalg.norm(u)
    assert np.allclose(np.tril(b.T, -1), 0.0)


def test_collocation_points_and_reproduction_at_selected_parameters(built):
    op, mus, b = built
    assert len(b.pts) == len(set(b.pts.tolist())) <= 2 * b.N - 1
    assert set(b.pts_s.tolist()) | set(b.pts_r.tolist()) == set(b.pts.tolist())
    for k, t in enumerate(b.selected):
        c = l1roc.colloc_solve(op, b.W, b.pts, mus[t])
        u = b.W.T @ c
        ref = O.pcg(op, mus[t], tol=1e-12).u
        assert np.linalg.norm(u - ref) <= 1e-7 * np.linalg.norm(ref)
        # the coefficients in the snapshot basis are the k-th unit vector
        assert l1roc.l1_indicator(b.T, c) == pytest.approx(1.0, abs=1e-6)


def test_collocation_residual_vanishes_at_the_points_when_square():
    # with as many points as vectors the over-collocation problem is interpolation
    op = O.assemble((10, 9, 8), (2, 1, 1))
    mus = inputs.log_uniform(31, 8, 2, 0.1, 10.0)
    b = l1roc.offline(op, mus, 3)
    W, pts = b.W, b.pts_s[:3]
    c = l1roc.colloc_solve(op, W, pts, mus[5])
    r = np.ones(op.n) - op.matvec(mus[5], W.T @ c)
    assert np.max(np.abs(r[pts])) <= 1e-10


def test_one_subdomain_is_exact_with_one_vector():
    # p = 1: u(mu) = u(1)/mu, so one snapshot spans every solution
    op = O.assemble((12, 10, 9), (1, 1, 1))
    b = l1roc.offline(op, np.array([[1.0], [3.0], [0.2]]), 3, snapshot_tol=1e-13)
    assert b.N == 1
    for m in (0.5, 7.0):
        c = l1roc.colloc_solve(op, b.W, b.pts, [m])
        ref = O.pcg(op, [m], tol=1e-13).u
        assert np.linalg.norm(b.W.T @ c - ref) <= 1e-10 * np.linalg.norm(ref)
