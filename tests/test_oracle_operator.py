"""Pins of the oracle's operator (Eq. 1 with the Sec. 4 diffusion model, 7-point FD).

Each test checks the explicit CSR assembly against something other than itself:
a textbook construction, a closed form, or an invariant of the PDE."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_2311_13862_gb300 import inputs


def laplacian_1d(n):
    h = 1.0 / (n + 1)
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h**2


def laplacian_3d(nx, ny, nz):
    """Textbook Kronecker-sum 7-point Laplacian, x fastest."""
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    return (sp.kron(sp.kron(Iz, Iy), laplacian_1d(nx)) + sp.kron(sp.kron(Iz, laplacian_1d(ny)), Ix)
            + sp.kron(sp.kron(laplacian_1d(nz), Iy), Ix)).tocsr()


@pytest.mark.parametrize("grid,blocks", [((4, 4, 4), (2, 1, 1)), ((5, 3, 4), (2, 2, 1)),
                                         ((6, 5, 7), (2, 2, 2)), ((7, 7, 7), (3, 3, 3))])
def test_sum_of_terms_is_constant_coefficient_laplacian(grid, blocks):
    op = O.assemble(grid, blocks)
    A = op.dense(np.ones(op.Q))
    L = laplacian_3d(*grid).toarray()
    assert np.max(np.abs(A - L)) <= 1e-12 * np.max(np.abs(L))


@pytest.mark.parametrize("grid,blocks", [((4, 4, 4), (2, 1, 1)), ((6, 5, 7), (2, 2, 2)),
                                         ((8, 8, 8), (3, 3, 3))])
def test_symmetric_positive_definite(grid, blocks):
    op = O.assemble(grid, blocks)
    mu = inputs.log_uniform(5, 1, op.Q, 0.01, 100.0)[0]
    A = op.dense(mu)
    assert np.array_equal(A, A.T)  # bitwise: one coefficient per face
    assert np.all(np.diag(A) > 0)
    off = np.abs(A).sum(1) - np.abs(np.diag(A))
    assert np.all(np.diag(A) >= off * (1 - 1e-14))
    L_np = np.linalg.cholesky(A)
    L_or = O.cholesky(A)
    assert np.max(np.abs(L_np - L_or)) <= 1e-13 * np.max(np.abs(L_np))


def test_affine_in_mu():
    op = O.assemble((6, 5, 4), (2, 2, 1))
    mu = inputs.log_uniform(7, 1, 4, 0.1, 10)[0]
    x = inputs.random_field(8, op.n)
    y = op.matvec(mu, x)
    ys = sum(mu[q] * op.matvec(np.eye(4)[q], x) for q in range(4))
    assert np.linalg.norm(y - ys) <= 1e-14 * np.linalg.norm(y)


def test_block_map_rule():
    # 16 interior nodes, 2 blocks: nodes 1..8 -> block 0, 9..16 -> block 1 (split at x = 0.5)
    m = O.block_map((16, 1, 1), (2, 1, 1))
    assert list(m) == [0] * 8 + [1] * 8
    # 128 nodes with 3 blocks: node i -> floor(3 i / 129): node 43 is exactly on x = 1/3 and
    # goes to the upper block
    m = O.block_map((128, 1, 1), (3, 1, 1))
    assert m[41] == 0 and m[42] == 1 and m[85] == 2 and m[84] == 1


@pytest.mark.parametrize("n,m", [(8, 1.0), (9, 2.5)])
def test_closed_form_eigenpairs(n, m):
    op = O.assemble((n, n, n), (2, 1, 1))
    h = 1.0 / (n + 1)
    i = np.arange(1, n + 1)
    for (a, b, c) in [(1, 1, 1), (2, 3, 1), (n, 1, n - 1)]:
        v = np.einsum("k,j,i->kji", np.sin(c * np.pi * i * h), np.sin(b * np.pi * i * h),
                      np.sin(a * np.pi * i * h)).ravel()
        lam = 4 * m / h**2 * (np.sin(a * np.pi * h / 2) ** 2 + np.sin(b * np.pi * h / 2) ** 2
                              + np.sin(c * np.pi * h / 2) ** 2)
        Av = op.matvec([m, m], v)
        assert np.linalg.norm(Av - lam * v) <= 1e-13 * np.linalg.norm(lam * v)


def test_face_coefficient_is_arithmetic_mean():
    # two nodes on either side of the x interface: the coupling is -(k0+k1)/2/h^2
    op = O.assemble((4, 1, 1), (2, 1, 1))
    A = op.dense([2.0, 6.0])
    h2 = (1 / 5) ** 2
    assert A[1, 2] == pytest.approx(-4.0 / h2, rel=1e-15)
    # node 0: two x faces with kappa 2 (one to the boundary) + four y/z faces to the boundary
    assert A[0, 0] == pytest.approx((2 * 2.0 / h2) + 4 * 2.0 / (1 / 2) ** 2, rel=1e-15)


@pytest.mark.parametrize("grid,blocks", [((4, 4, 4), (2, 1, 1)), ((6, 5, 7), (2, 2, 2)),
                                         ((7, 7, 7), (3, 3, 3)), ((9, 4, 6), (3, 1, 2))])
def test_direct_assembly_equals_the_affine_sum(grid, blocks):
    """orc_assemble_mu writes Eq. (1) for one mu directly; it must equal sum_q mu_q A_q of the
    affine terms (same pattern, values to rounding) and, at mu = 1, the textbook Laplacian."""
    op = O.assemble(grid, blocks)
    for seed in (11, 12):
        mu = inputs.log_uniform(seed, 1, op.Q, 0.01, 100.0)[0]
        one = O.assemble_mu(grid, mu, blocks=blocks)
        assert np.array_equal(one.row_ptr, op.row_ptr) and np.array_equal(one.col, op.col)
        ref = op.values(mu)
        assert np.max(np.abs(one.vals_q[0] - ref)) <= 4e-16 * np.max(np.abs(ref))
        A = sp.csr_matrix((one.vals_q[0], one.col, one.row_ptr)).toarray()
        assert np.array_equal(A, A.T)
    lap = O.assemble_mu(grid, np.ones(op.Q), blocks=blocks)
    A1 = sp.csr_matrix((lap.vals_q[0], lap.col, lap.row_ptr)).toarray()
    L = laplacian_3d(*grid).toarray()
    assert np.max(np.abs(A1 - L)) <= 1e-12 * np.max(np.abs(L))


def test_direct_assembly_with_an_explicit_map():
    grid = (6, 5, 4)
    m = inputs.random_field(13, 6 * 5 * 4)
    submap = (np.abs(m) * 7).astype(np.uint8) % 3
    op = O.assemble(grid, submap=submap, Q=3)
    mu = np.array([0.5, 3.0, 40.0])
    one = O.assemble_mu(grid, mu, submap=submap, Q=3)
    x = inputs.random_field(14, op.n)
    y_ref = op.matvec(mu, x)
    assert np.linalg.norm(one.matvec([1.0], x) - y_ref) <= 1e-14 * np.linalg.norm(y_ref)
