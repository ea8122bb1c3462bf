"""Parity of the CUDA multigrid V-cycle (Algorithm 2) and MGCG with the oracle's
(oracle.mg: scipy Galerkin products, dense Cholesky on the coarsest level)."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import mg
from paper_2311_13862_gb300 import inputs, rbws

pytestmark = pytest.mark.gpu

GRIDS = [((16, 16, 16), (2, 1, 1)),     # 3 levels
         ((24, 20, 18), (2, 2, 1)),     # 4 levels, odd and even axes
         ((33, 17, 20), (2, 2, 2)),     # ragged
         ((40, 36, 32), (3, 3, 3)),     # 27 subdomains, node on no interface
         ((4, 4, 3), (2, 1, 1)),        # one level: the exact solve
         ((130, 9, 3), (3, 1, 1))]      # an axis reaches one node: coarsest level of 260


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2311_13862_gb300 import build
    build.build()


@pytest.mark.parametrize("grid,blocks", GRIDS)
def test_vcycle_matches_oracle(grid, blocks):
    op = O.assemble(grid, blocks)
    H = mg.Hierarchy(op)
    B = 3
    mu = inputs.log_uniform(101, B, op.Q, 0.01, 100.0)
    x = inputs.random_field(102, (B, op.n))
    ref = np.stack([mg.vcycle(H.operators(mu[b]), x[b]) for b in range(B)])
    with rbws.Problem(grid, blocks) as P:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        rbws.rbws_apply_preconditioner(P.h, mu, xd, yd, rbws.PREC_MG)
        y = yd.cpu().numpy()
        assert torch.equal(xd.cpu(), torch.from_numpy(x))  # the input is left alone
    err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= 1e-11), err


def test_jacobi_preconditioner_is_the_inverse_diagonal():
    grid, blocks = (33, 17, 20), (2, 2, 2)
    op = O.assemble(grid, blocks)
    mu = inputs.log_uniform(103, 2, op.Q, 0.01, 100.0)
    x = inputs.random_field(104, (2, op.n))
    with rbws.Problem(grid, blocks) as P:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        rbws.rbws_apply_preconditioner(P.h, mu, xd, yd, rbws.PREC_JACOBI)
        y = yd.cpu().numpy()
    for b in range(2):
        d = O.mg.Hierarchy(op).operators(mu[b]).A[mg.Hierarchy(op).J].diagonal()
        assert np.allclose(y[b], x[b] / d, rtol=1e-14, atol=0)


@pytest.mark.parametrize("grid,blocks", GRIDS[:4])
def test_mgcg_matches_oracle(grid, blocks):
    op = O.assemble(grid, blocks)
    H = mg.Hierarchy(op)
    mu = inputs.log_uniform(105, 4, op.Q, 0.01, 100.0)
    with rbws.Problem(grid, blocks) as P:
        u = torch.empty((len(mu), P.n), dtype=torch.float64, device="cuda")
        rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, 1e-12, rbws.WARM_ZERO, u,
                                                rbws.rbws_options_default(precond=rbws.PREC_MG))
        u = u.cpu().numpy()
    assert rc == 0 and np.all(st == 0)
    for b in range(len(mu)):
        ref = mg.mgcg(op, mu[b], tol=1e-12, hier=H)
        assert abs(it[b] - ref.iters) <= 2, (it[b], ref.iters)
        assert np.linalg.norm(u[b] - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
        assert it[b] < 40


def test_rb_warm_started_mgcg_matches_oracle():
    """RBI-MGCG: the Galerkin RB initial value (Algorithm 4) with the MG preconditioner."""
    w = inputs.small(grid=(24, 20, 18), blocks=(2, 2, 1), n_max=8, n_train=24, n_test=4)
    op = O.assemble(w.grid, w.blocks)
    H = mg.Hierarchy(op)
    basis = O.greedy(op, inputs.train_mu(w), w.n_max)
    mu = inputs.test_mu(w)
    with rbws.Problem(w.grid, w.blocks) as P:
        rbws.rbws_set_basis(P.h, basis.W, basis.ANq, basis.fN)
        u = torch.empty((len(mu), P.n), dtype=torch.float64, device="cuda")
        opt = rbws.rbws_options_default(precond=rbws.PREC_MG)
        rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, 1e-12, rbws.WARM_GALERKIN, u, opt)
        u0 = torch.empty_like(u)
        _, it0, _, _ = rbws.rbws_solve_batch(P.h, mu, 1e-12, rbws.WARM_ZERO, u0, opt)
        u = u.cpu().numpy()
    assert rc == 0 and np.all(st == 0)
    for b in range(len(mu)):
        c = O.rb_solve(basis.ANq, basis.fN, mu[b])
        ref = mg.mgcg(op, mu[b], u0=basis.W.T @ c, tol=1e-12, hier=H)
        assert abs(it[b] - ref.iters) <= 2, (it[b], ref.iters)
        assert np.linalg.norm(u[b] - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
    assert it.mean() < it0.mean()


@pytest.mark.parametrize("grid,blocks", [((40, 36, 32), (2, 2, 2)),   # 4-node FP32 kernels
                                         ((33, 17, 20), (2, 2, 2)),   # nx % 4 != 0: one-node kernels
                                         ((64, 48, 40), (2, 2, 1)),
                                         ((64, 48, 34), (2, 2, 1))])  # odd z-chunk: unfused restriction
@pytest.mark.parametrize("warm", [rbws.WARM_ZERO, rbws.WARM_GALERKIN])
def test_fp32_mgcg_with_reliable_updates_reaches_the_fp64_residual(grid, blocks, warm):
    op = O.assemble(grid, blocks)
    H = mg.Hierarchy(op)
    mu = inputs.log_uniform(107, 4, op.Q, 0.01, 100.0)
    with rbws.Problem(grid, blocks) as P:
        if warm == rbws.WARM_GALERKIN:
            rbws.rbws_offline_greedy(P.h, inputs.log_uniform(108, 16, op.Q, 0.01, 100.0), 6, 0.0, 1e-12)
        u = torch.empty((len(mu), P.n), dtype=torch.float64, device="cuda")
        rc, it, rel, st = rbws.rbws_solve_batch(
            P.h, mu, 1e-10, warm, u, rbws.rbws_options_default(precond=rbws.PREC_MG, precision=rbws.FP32_IR))
        u = u.cpu().numpy()
    assert rc == 0 and np.all(st == 0)
    for b in range(len(mu)):
        true_rel = np.linalg.norm(np.ones(op.n) - op.matvec(mu[b], u[b])) / np.sqrt(op.n)
        assert true_rel < 1e-10
        assert rel[b] == pytest.approx(true_rel, rel=1e-6)
        ref = mg.mgcg(op, mu[b], tol=1e-13, hier=H)
        assert np.linalg.norm(u[b] - ref.u) <= 1e-7 * np.linalg.norm(ref.u)
        # FP32 inner iterations track the FP64 MGCG count closely
        assert it[b] <= 2 * mg.mgcg(op, mu[b], tol=1e-10, hier=H).iters + 4


def test_msrb_rejects_mixed_precision():
    with rbws.Problem((16, 16, 16), (2, 1, 1)) as P:
        u = torch.empty((1, P.n), dtype=torch.float64, device="cuda")
        with pytest.raises(rbws.RbwsError, match="UNSUPPORTED"):
            rbws.rbws_solve_batch(P.h, np.array([[1.0, 2.0]]), 1e-10, rbws.WARM_ZERO, u,
                                  rbws.rbws_options_default(precond=rbws.PREC_MSRB, precision=rbws.FP32_IR))


@pytest.mark.parametrize("warm", [rbws.WARM_ZERO, rbws.WARM_GALERKIN])
def test_fp32_mgcg_tracks_the_oracle_mgcg_on_the_64cube_workload(warm):
    """Every instance of a 64-parameter slice of the 64^3 workload: the FP32 iteration with
    reliable updates needs at most 3 iterations more than the oracle's FP64 MGCG from the same
    kind of start (zero, or the oracle's own Galerkin RB start from its own greedy over the same
    training parameters), and reaches the oracle's solution."""
    from oracle import batch as OB
    w = inputs.WORKLOADS["c2"]
    mu = inputs.test_mu(w)[:64]
    mtrain = inputs.train_mu(w)[:32]
    u0 = None
    if warm == rbws.WARM_GALERKIN:
        op = O.assemble(w.grid, w.blocks)
        basis = O.greedy(op, mtrain, w.n_max)
        u0 = np.stack([basis.W.T @ O.rb_solve(basis.ANq, basis.fN, m) for m in mu])
    _, it_ref, _, st_ref, _, _ = OB.reference_solutions(w.grid, mu, blocks=w.blocks, tol=1e-10, u0=u0)
    U_ref = OB.reference_solutions(w.grid, mu, blocks=w.blocks, tol=1e-13)[0]
    assert np.all(st_ref == 0)
    with rbws.Problem(w.grid, w.blocks) as P:
        rbws.rbws_offline_greedy(P.h, mtrain, w.n_max, 0.0, 1e-12)
        u = torch.empty((len(mu), P.n), dtype=torch.float64, device="cuda")
        _, it32, rel, st32 = rbws.rbws_solve_batch(
            P.h, mu, 1e-10, warm, u, rbws.rbws_options_default(precond=rbws.PREC_MG, precision=rbws.FP32_IR))
        uh = u.cpu().numpy()
    assert np.all(st32 == 0)
    assert np.all(it32 <= it_ref + 3), (it32 - it_ref).max()
    err = np.linalg.norm(uh - U_ref, axis=1) / np.linalg.norm(U_ref, axis=1)
    assert np.all(err <= 1e-8), err.max()


@pytest.mark.parametrize("grid,blocks", [((40, 36, 32), (2, 2, 2)),   # TMA-fed finest level, ragged tiles
                                         ((64, 48, 34), (2, 2, 1)),   # odd z-chunks: unfused restriction
                                         ((24, 20, 18), (2, 2, 1)),   # 4 levels
                                         ((36, 28, 24), (2, 2, 1)),   # nx % 8 == 4: 4-node prolongation
                                         ((33, 17, 20), (2, 2, 2))])  # nx % 4 != 0: one-node kernels
def test_fp32_vcycle_as_the_iteration_applies_it_matches_oracle(grid, blocks):
    """One FP32 V-cycle through the mixed-precision iteration's kernels (TMA-fed smoothing
    steps, the residual + restriction pass, the 32^3-style coarse steps and the tail) against
    the oracle's FP64 V-cycle, at FP32 accuracy."""
    op = O.assemble(grid, blocks)
    H = mg.Hierarchy(op)
    B = 3
    mu = inputs.log_uniform(111, B, op.Q, 0.01, 100.0)
    x = inputs.random_field(112, (B, op.n))
    ref = np.stack([mg.vcycle(H.operators(mu[b]), x[b]) for b in range(B)])
    with rbws.Problem(grid, blocks) as P:
        xd = torch.from_numpy(x).float().cuda()
        yd = torch.empty_like(xd)
        rbws.rbws_apply_mg32(P.h, mu, xd, yd)
        y = yd.double().cpu().numpy()
    err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= 2e-5), err
