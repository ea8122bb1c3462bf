"""Pins of the oracle's operator with a face-sampled coefficient and of its Dirichlet lift (the
paper's Example 1, Sec. 4: kappa = 1 + mu_1 g(x), f = 3 pi^2 sin sin sin, affine Dirichlet
data): agreement with the block assembly where the two describe the same operator, exact
reproduction of linear solutions, second-order convergence to the closed-form solution,
linearity and symmetry."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from oracle import mg
from oracle import rhs as R
from paper_2311_13862_gb300 import inputs


def csr(op, theta):
    return sp.csr_matrix((op.values(theta), op.col, op.row_ptr), shape=(op.n, op.n))


def ones_faces(grid, Q=1, c=1.0):
    nx, ny, nz = grid
    return (np.full((Q, nz, ny, nx + 1), c), np.full((Q, nz, ny + 1, nx), c), np.full((Q, nz + 1, ny, nx), c))


def nodes(grid):
    nx, ny, nz = grid
    Z, Y, X = np.meshgrid(*(np.arange(1, m + 1) / (m + 1) for m in (nz, ny, nx)), indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


@pytest.mark.parametrize("grid", [(5, 4, 3), (8, 8, 8), (7, 6, 9)])
def test_constant_coefficient_is_the_block_laplacian(grid):
    op = O.assemble_field(grid, *ones_faces(grid))
    ref = O.assemble(grid, (1, 1, 1))
    assert np.array_equal(op.row_ptr, ref.row_ptr) and np.array_equal(op.col, ref.col)
    scale = np.abs(ref.vals_q[0]).max()
    assert np.max(np.abs(op.vals_q[0] - ref.vals_q[0])) <= 1e-14 * scale


@pytest.mark.parametrize("grid,blocks", [((9, 7, 5), (2, 2, 1)), ((8, 10, 6), (2, 1, 3))])
def test_faces_from_a_block_map_give_the_block_terms(grid, blocks):
    """Face values built from the block indicator with the mean rule (and a boundary face
    taking its node's value) describe the block operator: every term matches orc_assemble_affine."""
    nx, ny, nz = grid
    Q = blocks[0] * blocks[1] * blocks[2]
    m = O.block_map(grid, blocks).reshape(nz, ny, nx)
    ind = np.stack([(m == q).astype(float) for q in range(Q)])  # [Q][nz][ny][nx]
    kfx = np.zeros((Q, nz, ny, nx + 1))
    kfx[..., 1:nx] = 0.5 * (ind[..., :-1] + ind[..., 1:])
    kfx[..., 0], kfx[..., nx] = ind[..., 0], ind[..., -1]
    kfy = np.zeros((Q, nz, ny + 1, nx))
    kfy[:, :, 1:ny, :] = 0.5 * (ind[:, :, :-1, :] + ind[:, :, 1:, :])
    kfy[:, :, 0, :], kfy[:, :, ny, :] = ind[:, :, 0, :], ind[:, :, -1, :]
    kfz = np.zeros((Q, nz + 1, ny, nx))
    kfz[:, 1:nz] = 0.5 * (ind[:, :-1] + ind[:, 1:])
    kfz[:, 0], kfz[:, nz] = ind[:, 0], ind[:, -1]
    op = O.assemble_field(grid, kfx, kfy, kfz)
    ref = O.assemble(grid, blocks)
    scale = np.abs(ref.vals_q).max()
    assert np.max(np.abs(op.vals_q - ref.vals_q)) <= 1e-14 * scale


@pytest.mark.parametrize("grid", [(6, 5, 4), (4, 7, 5)])
def test_linear_boundary_data_is_reproduced_exactly(grid):
    """kappa = 1 (and any constant): the 7-point operator annihilates linear functions, so with
    f = 0 and g_D = a + b x + c y + d z the discrete solution is g_D at the nodes.  Every
    boundary plane and every axis's lift enters."""
    a, b, c, d = 0.3, -1.7, 2.2, 0.9
    for kap in (1.0, 3.5):
        faces = ones_faces(grid, 1, kap)
        op = O.assemble_field(grid, *faces)
        X, Y, Z = inputs.boundary_points(grid)
        lift = O.dirichlet_lift(grid, *faces, a + b * X + c * Y + d * Z)[0]
        u = spla.spsolve(csr(op, [1.0]).tocsc(), lift)
        x, y, z = nodes(grid)
        assert np.max(np.abs(u - (a + b * x + c * y + d * z))) <= 1e-12


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_coefficient_varying_along_one_axis_keeps_linear_data_across_it(axis):
    """kappa varying along one axis only (random positive face values): a linear function of
    another coordinate has zero flux divergence there, node by node, so it is reproduced
    exactly; data linear along the varying axis is not (the check is not vacuous)."""
    grid = (6, 5, 7)
    nx, ny, nz = grid
    rng = np.random.default_rng(40 + axis)
    faces = list(ones_faces(grid))
    # faces of the varying axis take kappa at that axis's face coordinate, the others kappa at
    # the node coordinate: both from one random profile along the axis, per face and node
    n_ax = grid[axis]
    prof_f = rng.uniform(0.5, 3.0, n_ax + 1)
    prof_n = rng.uniform(0.5, 3.0, n_ax)
    for a in range(3):
        shape = faces[a].shape[1:]  # (z, y, x) extents of this face array
        idx = np.indices(shape)[2 - axis]  # index along `axis` in [z][y][x] order
        faces[a][0] = (prof_f if a == axis else prof_n)[idx]
    op = O.assemble_field(grid, *faces)
    A = csr(op, [1.0]).tocsc()
    X, Y, Z = inputs.boundary_points(grid)
    x, y, z = nodes(grid)
    coords_b, coords_n = (X, Y, Z), (x, y, z)
    other = (axis + 1) % 3
    u = spla.spsolve(A, O.dirichlet_lift(grid, *faces, 1.0 + 2.0 * coords_b[other])[0])
    assert np.max(np.abs(u - (1.0 + 2.0 * coords_n[other]))) <= 1e-12
    u2 = spla.spsolve(A, O.dirichlet_lift(grid, *faces, 1.0 + 2.0 * coords_b[axis])[0])
    assert np.max(np.abs(u2 - (1.0 + 2.0 * coords_n[axis]))) > 1e-3


def test_example1_at_mu1_zero_converges_to_the_closed_form_at_second_order():
    """mu_1 = 0 and zero boundary data: -Laplace u = 3 pi^2 sin sin sin has the solution
    u = sin(pi x) sin(pi y) sin(pi z); the 7-point error falls by about 4 per halving of h."""
    errs = []
    for n in (7, 15, 31):
        grid = (n, n, n)
        op = O.assemble_field(grid, *inputs.example1_faces(grid))
        F = inputs.example1_source(grid)
        u = spla.spsolve(csr(op, [1.0, 0.0]).tocsc(), F)
        x, y, z = nodes(grid)
        errs.append(np.max(np.abs(u - np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2, errs
    assert errs[-1] < 2e-3


def test_lift_is_linear_and_the_example1_rhs_is_its_affine_expansion():
    """dirichlet_lift is linear in the data and in each term; example1_rhs equals the source
    plus the lift of g_D(mu) through the single-term operator with kappa = 1 + mu_1 g."""
    grid = (9, 8, 7)
    faces = inputs.example1_faces(grid)
    G1, G2 = inputs.example1_boundary(grid)
    L1 = O.dirichlet_lift(grid, *faces, G1)
    L2 = O.dirichlet_lift(grid, *faces, G2)
    L12 = O.dirichlet_lift(grid, *faces, 0.25 * G1 - 2.0 * G2)
    assert np.allclose(L12, 0.25 * L1 - 2.0 * L2, rtol=0, atol=1e-12 * np.abs(L1).max())
    F = inputs.example1_source(grid)
    mu = inputs.example1_mu(41, 3)
    b = R.example1_rhs(F, L1, L2, mu)
    for k, (m1, m2) in enumerate(mu):
        one = tuple(f[:1] + m1 * f[1:2] for f in faces)  # kappa = 1 + mu_1 g as one term
        ref = F + O.dirichlet_lift(grid, *one, (1.0 - m2) * G1 + m2 * G2)[0]
        assert np.max(np.abs(b[k] - ref)) <= 1e-12 * np.abs(ref).max()
        # and the combined operator is the affine combination of the two terms
        op1 = O.assemble_field(grid, *one)
        opq = O.assemble_field(grid, *faces)
        assert np.max(np.abs(op1.vals_q[0] - opq.values(R.example1_affine(mu)[k]))) <= \
            1e-13 * np.abs(op1.vals_q[0]).max()


def test_example1_operator_is_symmetric_positive_definite():
    grid = (6, 5, 4)
    op = O.assemble_field(grid, *inputs.example1_faces(grid))
    for m1 in (0.0, 1.0, 2.0):
        A = csr(op, [1.0, m1]).toarray()
        assert np.array_equal(A, A.T)
        assert np.linalg.eigvalsh(A).min() > 0.0


def test_boundary_layout_faces_the_right_nodes():
    """A boundary value placed on one plane reaches only the nodes next to that plane, with the
    face coefficient of that face: a unit value on each plane in turn."""
    grid = (5, 4, 3)
    nx, ny, nz = grid
    faces = inputs.example1_faces(grid)
    sizes = [nz * ny, nz * ny, nz * nx, nz * nx, ny * nx, ny * nx]
    off = np.concatenate([[0], np.cumsum(sizes)])
    h2 = [(nx + 1) ** 2, (ny + 1) ** 2, (nz + 1) ** 2]
    for p in range(6):
        gb = np.zeros(O.boundary_size(grid))
        gb[off[p]:off[p + 1]] = 1.0
        lift = O.dirichlet_lift(grid, *faces, gb)[1].reshape(nz, ny, nx)
        a, hi = p // 2, p % 2
        kf = faces[a][1]
        if a == 0:
            expect_face = kf[:, :, nx] if hi else kf[:, :, 0]
            got = lift[:, :, nx - 1] if hi else lift[:, :, 0]
            rest = np.delete(lift, nx - 1 if hi else 0, axis=2)
        elif a == 1:
            expect_face = kf[:, ny, :] if hi else kf[:, 0, :]
            got = lift[:, ny - 1, :] if hi else lift[:, 0, :]
            rest = np.delete(lift, ny - 1 if hi else 0, axis=1)
        else:
            expect_face = kf[nz] if hi else kf[0]
            got = lift[nz - 1] if hi else lift[0]
            rest = np.delete(lift, nz - 1 if hi else 0, axis=0)
        assert np.allclose(got, expect_face * h2[a], rtol=1e-15, atol=0)
        assert np.all(rest == 0.0)


def test_mgcg_solves_example1_at_the_largest_contrast():
    """The oracle's MGCG (Galerkin coarse operators of the face-field terms) reaches 1e-10 on
    Example 1 with mu_1 = 2 in a modest number of iterations."""
    grid = (15, 15, 15)
    op = O.assemble_field(grid, *inputs.example1_faces(grid))
    G1, G2 = inputs.example1_boundary(grid)
    L1, L2 = (O.dirichlet_lift(grid, *inputs.example1_faces(grid), G) for G in (G1, G2))
    mu = np.array([[2.0, 0.5]])
    b = R.example1_rhs(inputs.example1_source(grid), L1, L2, mu)[0]
    r = mg.mgcg(op, R.example1_affine(mu)[0], f=b, tol=1e-10)
    assert r.status == 0 and r.iters <= 30
    assert np.linalg.norm(b - op.matvec(R.example1_affine(mu)[0], r.u)) <= 1e-10 * np.linalg.norm(b)
