"""The paper's Example 1 (Sec. 4) on the GPU, against the oracle: a coefficient that varies from
node to node, kappa = 1 + mu_1 g(x), given at the cell faces as two affine terms (kappa_0 = 1,
kappa_1 = g), Dirichlet data g_D(mu) = (1 - mu_2) G1 + mu_2 G2 eliminated into the right-hand
side (the lift), and the source 3 pi^2 sin sin sin.  Operator, lift, affine right-hand sides,
V-cycle, FP64 PCG, the greedy with a right-hand side per training parameter, the mixed-precision
MGCG of every instance from zero and Galerkin starts, and the checkpoint."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import batch as OB
from oracle import mg
from oracle import rhs as R
from paper_2311_13862_gb300 import inputs, rbws

pytestmark = pytest.mark.gpu

GRIDS = [(16, 12, 10), (33, 20, 17), (40, 36, 32)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2311_13862_gb300 import build
    build.build()


def theta_f(mu):
    """Coefficients of the right-hand side's affine terms (F, L1_0, L1_1, L2_0, L2_1)."""
    m1, m2 = mu[:, 0], mu[:, 1]
    return np.column_stack([np.ones(len(mu)), 1.0 - m2, m1 * (1.0 - m2), m2, m1 * m2])


class Ex1:
    """The GPU problem and its affine right-hand side terms on the device."""

    def __init__(self, grid):
        self.grid = grid
        self.faces = inputs.example1_faces(grid)
        self.P = rbws.Problem.field(grid, *self.faces)
        n = self.P.n
        G1, G2 = inputs.example1_boundary(grid)
        L = torch.empty((2, 2, n), dtype=torch.float64, device="cuda")
        rbws.rbws_dirichlet_lift(self.P.h, G1, L[0])
        rbws.rbws_dirichlet_lift(self.P.h, G2, L[1])
        self.L = L
        F = torch.from_numpy(inputs.example1_source(grid)).cuda()
        self.Fk = torch.stack([F, L[0, 0], L[0, 1], L[1, 0], L[1, 1]]).contiguous()

    def rhs(self, mu):
        f = torch.empty((len(mu), self.P.n), dtype=torch.float64, device="cuda")
        rbws.rbws_affine_sources(self.P.h, self.Fk, theta_f(mu), f)
        return f

    def close(self):
        self.P.close()


def oracle_rhs(grid, mu):
    faces = inputs.example1_faces(grid)
    G1, G2 = inputs.example1_boundary(grid)
    L1, L2 = (O.dirichlet_lift(grid, *faces, G) for G in (G1, G2))
    return R.example1_rhs(inputs.example1_source(grid), L1, L2, mu)


@pytest.mark.parametrize("grid", GRIDS)
def test_operator_lift_and_sources_match_the_oracle(grid):
    op = O.assemble_field(grid, *inputs.example1_faces(grid))
    mu = inputs.example1_mu(301, 3)
    th = R.example1_affine(mu)
    x = inputs.random_field(302, (3, op.n))
    ref = np.stack([op.matvec(th[b], x[b]) for b in range(3)])
    E = Ex1(grid)
    try:
        xd = torch.from_numpy(x).cuda()
        y = torch.empty_like(xd)
        rbws.rbws_apply_operator(E.P.h, th, xd, y, rbws.FP64)
        y32 = torch.empty_like(xd.float())
        rbws.rbws_apply_operator(E.P.h, th, xd.float(), y32, rbws.FP32_IR)
        Lg = E.L.cpu().numpy()
        fg = E.rhs(mu).cpu().numpy()
    finally:
        E.close()
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.max(np.abs(y.cpu().numpy() - ref) / scale) <= 1e-14
    ref32 = np.stack([op.matvec(th[b], x[b].astype(np.float32).astype(np.float64)) for b in range(3)])
    assert np.max(np.abs(y32.cpu().numpy() - ref32) / scale) <= 1e-5
    faces = inputs.example1_faces(grid)
    for k, G in enumerate(inputs.example1_boundary(grid)):
        Lo = O.dirichlet_lift(grid, *faces, G)
        assert np.max(np.abs(Lg[k] - Lo)) <= 1e-15 * np.abs(Lo).max()
    fo = oracle_rhs(grid, mu)
    assert np.max(np.abs(fg - fo)) <= 1e-14 * np.abs(fo).max()


@pytest.mark.parametrize("grid", GRIDS[:2])
def test_vcycle_matches_the_oracle(grid):
    op = O.assemble_field(grid, *inputs.example1_faces(grid))
    H = mg.Hierarchy(op)
    th = R.example1_affine(inputs.example1_mu(303, 2))
    x = inputs.random_field(304, (2, op.n))
    ref = np.stack([mg.vcycle(H.operators(th[b]), x[b]) for b in range(2)])
    E = Ex1(grid)
    try:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        rbws.rbws_apply_preconditioner(E.P.h, th, xd, yd, rbws.PREC_MG)
        y = yd.cpu().numpy()
    finally:
        E.close()
    err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= 1e-11), err


def test_fp64_pcg_matches_the_oracle():
    grid = (16, 12, 10)
    op = O.assemble_field(grid, *inputs.example1_faces(grid))
    mu = inputs.example1_mu(305, 4)
    th = R.example1_affine(mu)
    F = oracle_rhs(grid, mu)
    E = Ex1(grid)
    try:
        f = E.rhs(mu)
        u = torch.empty_like(f)
        rc, it, rel, st = rbws.rbws_solve_batch_rhs(E.P.h, th, f, 1e-12, rbws.WARM_ZERO, u,
                                                    rbws.rbws_options_default())
        uh = u.cpu().numpy()
    finally:
        E.close()
    assert rc == 0 and np.all(st == 0)
    for b in range(4):
        ref = O.pcg(op, th[b], f=F[b], tol=1e-12)
        assert abs(int(it[b]) - ref.iters) <= 2
        assert np.linalg.norm(uh[b] - ref.u) <= 1e-10 * np.linalg.norm(ref.u)


def test_greedy_and_mixed_precision_mgcg_of_every_instance_against_the_oracle():
    """The greedy over training parameters, each with its own right-hand side, selects what the
    oracle's greedy selects; then every test instance's FP32-IR MGCG solution, from zero and from
    the Galerkin start, is compared with the oracle's FP64 MGCG solution."""
    grid = (40, 36, 32)
    op = O.assemble_field(grid, *inputs.example1_faces(grid))
    mu_t = inputs.example1_mu(306, 16)
    th_t = R.example1_affine(mu_t)
    Ft = oracle_rhs(grid, mu_t)
    gref = R.greedy_rhs(op, th_t, Ft, 6, snapshot_tol=1e-12)
    mu = inputs.example1_mu(307, 8)
    th = R.example1_affine(mu)
    F = oracle_rhs(grid, mu)
    U_ref = OB.reference_solutions(grid, th, f=F, tol=1e-13, processes=4, fields=inputs.example1_faces(grid))[0]
    E = Ex1(grid)
    try:
        N, sel, eta = rbws.rbws_offline_greedy_rhs(E.P.h, th_t, E.rhs(mu_t), 6, 0.0, 1e-12)
        assert N == gref.N and np.array_equal(sel, gref.selected), (sel, gref.selected)
        assert np.allclose(eta, gref.eta_hist, rtol=1e-6, equal_nan=True)
        f = E.rhs(mu)
        its = {}
        for warm in (rbws.WARM_ZERO, rbws.WARM_GALERKIN):
            u = torch.empty_like(f)
            rc, it, rel, st = rbws.rbws_solve_batch_rhs(
                E.P.h, th, f, 1e-10, warm, u,
                rbws.rbws_options_default(precision=rbws.FP32_IR, precond=rbws.PREC_MG))
            assert rc == 0 and np.all(st == 0)
            es = OB.error_summary(grid, th, u.cpu().numpy(), U_ref, f=F, fields=inputs.example1_faces(grid))
            print("Example 1 MGCG FP32-IR warm %d: iterations %s; rel-L2 vs oracle max %.2e; true rel-res max %.2e"
                  % (warm, it.tolist(), es["relL2_max"], es["true_relres_max"]))
            assert es["true_relres_max"] < 1e-10
            assert es["relL2_max"] <= 1e-8
            its[warm] = it.copy()
        assert its[rbws.WARM_GALERKIN].mean() <= its[rbws.WARM_ZERO].mean()
    finally:
        E.close()


def test_checkpoint_and_the_static_apply(tmp_path):
    grid = (16, 12, 10)
    th = R.example1_affine(inputs.example1_mu(308, 2))
    x = torch.from_numpy(inputs.random_field(309, (2, grid[0] * grid[1] * grid[2]))).cuda()
    E = Ex1(grid)
    try:
        y0 = torch.empty_like(x)
        rbws.rbws_apply_operator(E.P.h, th, x, y0, rbws.FP64)
        with pytest.raises(rbws.RbwsError) as ei:
            rbws.rbws_apply_operator_static(E.P.h, th, x, torch.empty_like(x))
        assert ei.value.status == rbws.ERR_UNSUPPORTED
        path = tmp_path / "ex1.ckpt"
        rbws.rbws_save(E.P.h, path)
    finally:
        E.close()
    Q = rbws.Problem.load(path)
    try:
        y1 = torch.empty_like(x)
        rbws.rbws_apply_operator(Q.h, th, x, y1, rbws.FP64)
        assert torch.equal(y0, y1)  # the face fields came back
    finally:
        Q.close()
    with rbws.Problem(grid, (2, 1, 1)) as P:  # the lift belongs to face-field problems only
        with pytest.raises(rbws.RbwsError) as ei:
            rbws.rbws_dirichlet_lift(P.h, np.zeros(O.boundary_size(grid)),
                                     torch.empty((2, P.n), dtype=torch.float64, device="cuda"))
        assert ei.value.status == rbws.ERR_UNSUPPORTED
