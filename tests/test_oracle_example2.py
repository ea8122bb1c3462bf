"""Pins of the oracle's mixed boundary value operator (the shape of the paper's Example 2,
Sec. 4): an anisotropic diffusion tensor diag(kx, ky, kz) times kappa and a homogeneous
Neumann face at coordinate 1 of an axis, node-centred finite volumes with a half control
volume on the Neumann face.  Each test checks orc_assemble_ex against something other than
itself: closed-form eigenpairs of the generalised problem A v = lambda W v, symmetry and
definiteness, hand-computed rows, the source formula, and a direct sparse solve."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from oracle import mg
from oracle import rhs as R
from paper_2311_13862_gb300 import inputs


def test_node_weights_halve_on_neumann_faces():
    w = O.node_weights((3, 4, 2), (1, 1, 0)).reshape(2, 4, 3)
    assert w[0, 0, 0] == 1.0 and w[1, 1, 2] == 0.5 and w[0, 3, 1] == 0.5 and w[1, 3, 2] == 0.25
    assert np.all(O.node_weights((3, 4, 2)) == 1.0)


@pytest.mark.parametrize("grid,kscale,neumann", [((8, 6, 5), (1.0, 1.0, 1e-2), (1, 0, 0)),
                                                 ((6, 7, 4), (2.0, 0.5, 1.0), (1, 1, 0)),
                                                 ((5, 5, 6), (1.0, 1.0, 1.0), (0, 0, 1))])
def test_generalised_eigenpairs_in_closed_form(grid, kscale, neumann):
    """Constant kappa: with the half-cell rows A = W L, L the ghost-node operator, so the
    products of sin((a - 1/2) pi x) (Neumann axis, nodes i/n) and sin(b pi y) (Dirichlet axis,
    nodes j/(n+1)) satisfy A v = lambda W v, lambda = sum over axes of k * 4 sin^2(theta/2) / h^2."""
    op = O.assemble(grid, (1, 1, 1), kscale=kscale, neumann=neumann)
    W = O.node_weights(grid, neumann)
    for modes in [(1, 1, 1), (2, 3, 1), (grid[0], 1, grid[2] - 1)]:
        vecs, lam = [], 0.0
        for n, nm, k, m in zip(grid, neumann, kscale, modes):
            i = np.arange(1, n + 1)
            if nm:
                th = (m - 0.5) * np.pi / n
                h = 1.0 / n
            else:
                th = m * np.pi / (n + 1)
                h = 1.0 / (n + 1)
            vecs.append(np.sin(th * i))
            lam += k * 4.0 * np.sin(th / 2) ** 2 / h ** 2
        v = np.einsum("k,j,i->kji", vecs[2], vecs[1], vecs[0]).ravel()
        Av = op.matvec([1.0], v)
        assert np.linalg.norm(Av - lam * W * v) <= 1e-12 * np.linalg.norm(lam * W * v)


def test_symmetric_positive_definite_with_anisotropy_and_a_neumann_face():
    grid = (6, 5, 4)
    op = O.assemble(grid, (1, 2, 2), kscale=(1.0, 1.0, 1e-2), neumann=(1, 0, 0))
    mu = inputs.log_uniform(31, 1, 4, 0.1, 1.0)[0]
    A = op.dense(mu)
    assert np.array_equal(A, A.T)
    assert np.all(np.linalg.eigvalsh(A) > 0)


def test_a_neumann_face_row_by_hand():
    # 4 nodes in x with the Neumann face at x = 1 (h = 1/4), 1 node in y and z (h = 1/2),
    # kappa = 3, tensor diag(1, 1, 0.01): the last node has half a control volume
    op = O.assemble((4, 1, 1), (1, 1, 1), kscale=(1.0, 1.0, 0.01), neumann=(1, 0, 0))
    A = op.dense([3.0])
    hx2, hy2 = (1 / 4) ** 2, (1 / 2) ** 2
    assert A[3, 2] == pytest.approx(-3.0 / hx2, rel=1e-15)
    # west face whole; y faces (two, to the boundary) and z faces at half area
    assert A[3, 3] == pytest.approx(3.0 / hx2 + 0.5 * 2 * 3.0 / hy2 + 0.5 * 2 * 0.03 / hy2, rel=1e-15)
    # an interior node: two x faces, full y and z faces
    assert A[1, 1] == pytest.approx(2 * 3.0 / hx2 + 2 * 3.0 / hy2 + 2 * 0.03 / hy2, rel=1e-15)


def test_block_map_by_coordinate_on_a_neumann_axis():
    # 8 nodes on a Neumann axis sit at i/8: two blocks split at 0.5 put nodes 1..3 below and
    # 4..8 (node 4 at exactly 0.5) above
    m = O.block_map((8, 1, 1), (2, 1, 1), neumann=(1, 0, 0))
    assert list(m) == [0, 0, 0, 1, 1, 1, 1, 1]
    # the four subregions of Example 2 by y and z halves
    m = O.block_map((2, 4, 4), (1, 2, 2), neumann=(1, 0, 0)).reshape(4, 4, 2)
    assert m[0, 0, 0] == 0 and m[0, 3, 1] == 1 and m[3, 0, 0] == 2 and m[3, 3, 1] == 3


def test_example2_source_formula():
    grid = (4, 3, 3)
    f = R.example2_source(grid, [[1.0, 0.5, 0.5, 0.25]], neumann=(1, 0, 0))[0].reshape(3, 3, 4)
    # node (x, y, z) = (1, 1/2, 1/2) is the centre, on the Neumann face: half of 0.25 + 1/0.25
    assert f[1, 1, 3] == pytest.approx(0.5 * (0.25 + 4.0), rel=1e-15)
    # node (1/4, 1/4, 1/4): d^2 = 9/16 + 1/16 + 1/16
    assert f[0, 0, 0] == pytest.approx(0.25 + np.exp(-(11 / 16) / 0.25) / 0.25, rel=1e-15)


def test_mgcg_on_the_mixed_problem_matches_a_direct_solve():
    grid = (16, 15, 14)
    op = O.assemble(grid, (1, 2, 2), kscale=(1.0, 1.0, 1e-2), neumann=(1, 0, 0))
    mu = np.array([0.3, 0.7, 0.15, 1.0])
    f = R.example2_source(grid, [[0.45, 0.55, 0.5, 0.3]])[0]
    r = mg.mgcg(op, mu, f=f, tol=1e-12)
    assert r.status == 0
    A = sp.csr_matrix((op.values(mu), op.col, op.row_ptr))
    u = spla.spsolve(A.tocsc(), f)
    assert np.linalg.norm(r.u - u) <= 1e-10 * np.linalg.norm(u)
