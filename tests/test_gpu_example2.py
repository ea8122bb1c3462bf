"""The mixed boundary value problem of the paper's Example 2 (Sec. 4) on the GPU, against the
oracle: anisotropic tensor diag(1, 1, 1e-2) on four subregions (kappa = mu_1..mu_3 and 1), a
homogeneous Neumann face at x = 1 with half control volumes, and the Example 2 source
mu7 + exp(-|x - (mu4, mu5, mu6)|^2 / mu7) / mu7.  Operator, source, V-cycle, FP64 PCG and the
mixed-precision MGCG of every instance, the greedy with a source per training parameter, and
the checkpoint of the axes."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import batch as OB
from oracle import mg
from oracle import rhs as R
from paper_2311_13862_gb300 import inputs, rbws

pytestmark = pytest.mark.gpu

KS = (1.0, 1.0, 1e-2)
NM = (1, 0, 0)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2311_13862_gb300 import build
    build.build()


def ex2_mu(seed, n):
    """(mu1..mu3) in [0.1, 1]^3 as the kappas of the subregions in block order (y-lower/z-lower,
    y-upper/z-lower, y-lower/z-upper, y-upper/z-upper = 1), and the source parameters
    (mu4, mu5, mu6) in [0.4, 0.6]^3, mu7 in [0.25, 0.5]."""
    rng = np.random.default_rng(seed)
    m = np.column_stack([rng.uniform(0.1, 1.0, (n, 3)), rng.uniform(0.4, 0.6, (n, 3)), rng.uniform(0.25, 0.5, n)])
    kap = np.column_stack([m[:, 0], m[:, 2], m[:, 1], np.ones(n)])  # block id = (kz*2 + ky)
    src = np.column_stack([m[:, 3:6], m[:, 6], 1.0 / m[:, 6], m[:, 6]])
    return m, kap, src


GRIDS = [(24, 20, 18), (25, 16, 12), (32, 32, 32)]


@pytest.mark.parametrize("grid", GRIDS)
def test_operator_and_source_match_the_oracle(grid):
    op = O.assemble(grid, (1, 2, 2), kscale=KS, neumann=NM)
    m, kap, src = ex2_mu(201, 3)
    x = inputs.random_field(202, (3, op.n))
    ref = np.stack([op.matvec(kap[b], x[b]) for b in range(3)])
    with rbws.Problem(grid, (1, 2, 2), kappa_scale=KS, neumann=NM) as P:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        rbws.rbws_apply_operator(P.h, kap, xd, yd, rbws.FP64)
        y = yd.cpu().numpy()
        y32 = torch.empty_like(xd.float())
        rbws.rbws_apply_operator(P.h, kap, xd.float(), y32, rbws.FP32_IR)
        f = torch.empty_like(xd)
        rbws.rbws_gaussian_source_ex(P.h, src, f)
        fg = f.cpu().numpy()
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.max(np.abs(y - ref) / scale) <= 1e-14
    ref32 = np.stack([op.matvec(kap[b], x[b].astype(np.float32).astype(np.float64)) for b in range(3)])
    assert np.max(np.abs(y32.cpu().numpy() - ref32) / scale) <= 1e-5
    assert np.allclose(fg, R.example2_source(grid, m[:, 3:], NM), rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("grid", GRIDS[:2])
def test_vcycle_matches_the_oracle(grid):
    op = O.assemble(grid, (1, 2, 2), kscale=KS, neumann=NM)
    H = mg.Hierarchy(op)
    _, kap, _ = ex2_mu(203, 2)
    x = inputs.random_field(204, (2, op.n))
    ref = np.stack([mg.vcycle(H.operators(kap[b]), x[b]) for b in range(2)])
    with rbws.Problem(grid, (1, 2, 2), kappa_scale=KS, neumann=NM) as P:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        rbws.rbws_apply_preconditioner(P.h, kap, xd, yd, rbws.PREC_MG)
        y = yd.cpu().numpy()
    err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= 1e-11), err


def test_fp64_pcg_matches_the_oracle():
    grid = (24, 20, 18)
    op = O.assemble(grid, (1, 2, 2), kscale=KS, neumann=NM)
    m, kap, src = ex2_mu(205, 4)
    F = R.example2_source(grid, m[:, 3:], NM)
    with rbws.Problem(grid, (1, 2, 2), kappa_scale=KS, neumann=NM) as P:
        f = torch.from_numpy(F).cuda()
        u = torch.empty_like(f)
        rc, it, rel, st = rbws.rbws_solve_batch_rhs(P.h, kap, f, 1e-12, rbws.WARM_ZERO, u,
                                                    rbws.rbws_options_default())
        uh = u.cpu().numpy()
    assert np.all(st == 0)
    for b in range(4):
        ref = O.pcg(op, kap[b], f=F[b], tol=1e-12)
        assert abs(int(it[b]) - ref.iters) <= 2
        assert np.linalg.norm(uh[b] - ref.u) <= 1e-10 * np.linalg.norm(ref.u)


def test_mixed_precision_mgcg_every_instance_against_the_oracle():
    grid = (48, 40, 36)
    m, kap, src = ex2_mu(206, 8)
    F = R.example2_source(grid, m[:, 3:], NM)
    U_ref = OB.reference_solutions(grid, kap, blocks=(1, 2, 2), f=F, tol=1e-13, processes=4, kscale=KS,
                                   neumann=NM)[0]
    with rbws.Problem(grid, (1, 2, 2), kappa_scale=KS, neumann=NM) as P:
        f = torch.empty((8, P.n), dtype=torch.float64, device="cuda")
        rbws.rbws_gaussian_source_ex(P.h, src, f)
        u = torch.empty_like(f)
        rc, it, rel, st = rbws.rbws_solve_batch_rhs(
            P.h, kap, f, 1e-10, rbws.WARM_ZERO, u,
            rbws.rbws_options_default(precision=rbws.FP32_IR, precond=rbws.PREC_MG))
        assert rc == 0 and np.all(st == 0)
        es = OB.error_summary(grid, kap, u.cpu().numpy(), U_ref, blocks=(1, 2, 2), f=F, kscale=KS, neumann=NM)
    print("Example 2 MGCG FP32-IR: iterations %s; rel-L2 vs oracle max %.2e; true rel-res max %.2e"
          % (it.tolist(), es["relL2_max"], es["true_relres_max"]))
    assert es["true_relres_max"] < 1e-10
    assert es["relL2_max"] <= 1e-8


def test_greedy_with_example2_sources_and_the_checkpoint(tmp_path):
    grid = (24, 20, 16)
    op = O.assemble(grid, (1, 2, 2), kscale=KS, neumann=NM)
    m, kap, src = ex2_mu(207, 20)
    Ft = R.example2_source(grid, m[:, 3:], NM)
    ref = R.greedy_rhs(op, kap, Ft, 6, snapshot_tol=1e-12)
    with rbws.Problem(grid, (1, 2, 2), kappa_scale=KS, neumann=NM) as P:
        N, sel, eta = rbws.rbws_offline_greedy_rhs(P.h, kap, torch.from_numpy(Ft).cuda(), 6, 0.0, 1e-12)
        assert N == ref.N and np.array_equal(sel, ref.selected), (sel, ref.selected)
        assert np.allclose(eta, ref.eta_hist, rtol=1e-6, equal_nan=True)
        x = torch.from_numpy(inputs.random_field(208, (2, op.n))).cuda()
        y0 = torch.empty_like(x)
        rbws.rbws_apply_operator(P.h, kap[:2], x, y0, rbws.FP64)
        path = tmp_path / "ex2.ckpt"
        rbws.rbws_save(P.h, path)
    Q = rbws.Problem.load(path)
    try:
        y1 = torch.empty_like(x)
        rbws.rbws_apply_operator(Q.h, kap[:2], x, y1, rbws.FP64)
        assert torch.equal(y0, y1)  # the axes (anisotropy, Neumann face) came back
    finally:
        Q.close()
