"""Pins of the oracle's per-instance right-hand sides: the Gaussian source (closed-form values
and symmetries) and the greedy with a right-hand side per training parameter (it reduces to the
fixed-f greedy when every right-hand side is f = 1; snapshot reproduction; Galerkin
orthogonality)."""
import numpy as np
import pytest

import oracle as O
from oracle import rhs as R
from paper_2311_13862_gb300 import inputs


def test_gaussian_source_values_and_symmetry():
    grid = (9, 7, 5)
    h = [1.0 / (n + 1) for n in grid]
    # a centre on node (i, j, k) = (4, 3, 2): value 1 there, exp(-1/2) one width away along x
    c = (5 * h[0], 4 * h[1], 3 * h[2])
    sg = h[0]
    f = R.gaussian_source(grid, [[c[0], c[1], c[2], sg]])[0].reshape(grid[2], grid[1], grid[0])
    assert f[2, 3, 4] == pytest.approx(1.0, rel=1e-15)
    assert f[2, 3, 5] == pytest.approx(np.exp(-0.5), rel=1e-14)
    assert f.max() == f[2, 3, 4]
    # mirroring the centre in x mirrors the field
    g = R.gaussian_source(grid, [[1 - 0.3, 0.4, 0.5, 0.2], [0.3, 0.4, 0.5, 0.2]]).reshape(2, 5, 7, 9)
    assert np.allclose(g[0], g[1][:, :, ::-1], rtol=1e-14, atol=0)


@pytest.fixture(scope="module")
def small():
    w = inputs.small(grid=(10, 9, 8), blocks=(2, 2, 1), n_max=5, n_train=12, n_test=3)
    return w, O.assemble(w.grid, w.blocks)


def test_greedy_rhs_with_constant_sources_is_the_fixed_f_greedy(small):
    w, op = small
    mus = inputs.train_mu(w)
    ref = O.greedy(op, mus, w.n_max, snapshot_tol=1e-13)
    got = R.greedy_rhs(op, mus, np.ones((len(mus), op.n)), w.n_max, snapshot_tol=1e-13)
    assert got.N == ref.N
    assert np.array_equal(got.selected, ref.selected)
    assert np.allclose(got.eta_hist, ref.eta_hist, rtol=1e-8, equal_nan=True)
    assert np.max(np.abs(got.W.T @ (got.W @ ref.W.T) - ref.W.T)) <= 1e-9   # same span


def test_greedy_rhs_reproduces_its_snapshots(small):
    w, op = small
    mus = inputs.train_mu(w)
    rng = np.random.default_rng(7)
    prm = np.column_stack([rng.uniform(0.3, 0.7, (len(mus), 3)), np.full(len(mus), 0.15)])
    F = R.gaussian_source(w.grid, prm)
    b = R.greedy_rhs(op, mus, F, w.n_max, snapshot_tol=1e-13)
    assert np.max(np.abs(b.W @ b.W.T - np.eye(b.N))) <= 1e-12
    for t in b.selected:
        u = O.pcg(op, mus[t], f=F[t], tol=1e-13).u
        urb = R.rb_start(b, mus[t], F[t])
        assert np.linalg.norm(urb - u) <= 1e-8 * np.linalg.norm(u)
    # Galerkin orthogonality at an unselected parameter
    t = next(t for t in range(len(mus)) if t not in set(b.selected))
    urb = R.rb_start(b, mus[t], F[t])
    assert np.max(np.abs(b.W @ (F[t] - op.matvec(mus[t], urb)))) <= 1e-10 * np.linalg.norm(F[t])
