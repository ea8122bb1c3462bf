"""Per-instance right-hand sides on the GPU (a non-affine Gaussian source, the shape of the
paper's Example 2): the source kernel, the PCG solve and the greedy with a right-hand side per
training parameter, against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import rhs as R
from paper_2311_13862_gb300 import inputs, rbws

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2311_13862_gb300 import build
    build.build()


def gauss_params(seed, n, lo=0.3, hi=0.7, sigma=0.15):
    rng = np.random.default_rng(seed)
    return np.column_stack([rng.uniform(lo, hi, (n, 3)), np.full(n, sigma)])


def test_gaussian_source_matches_oracle():
    grid = (24, 20, 18)
    prm = gauss_params(11, 5)
    with rbws.Problem(grid, (2, 2, 1)) as P:
        f = torch.empty((5, P.n), dtype=torch.float64, device="cuda")
        rbws.rbws_gaussian_source(P.h, prm, f)
        got = f.cpu().numpy()
        with pytest.raises(rbws.RbwsError, match="INVALID_ARG"):
            bad = prm.copy()
            bad[0, 3] = 0.0
            rbws.rbws_gaussian_source(P.h, bad, f)
    # exp of arguments up to about 60: a last-bit difference in the argument is ~1e-14 relative
    assert np.allclose(got, R.gaussian_source(grid, prm), rtol=1e-12, atol=1e-300)


def test_solve_with_per_instance_sources_matches_oracle():
    grid, blocks = (24, 20, 18), (2, 2, 1)
    op = O.assemble(grid, blocks)
    mu = inputs.log_uniform(12, 4, op.Q, 0.1, 10.0)
    prm = gauss_params(13, 4)
    F = R.gaussian_source(grid, prm)
    with rbws.Problem(grid, blocks) as P:
        f = torch.from_numpy(F).cuda()
        u = torch.empty_like(f)
        rc, it, rel, st = rbws.rbws_solve_batch_rhs(P.h, mu, f, 1e-12, rbws.WARM_ZERO, u,
                                                    rbws.rbws_options_default())
        u = u.cpu().numpy()
    assert np.all(st == 0)
    for b in range(4):
        ref = O.pcg(op, mu[b], f=F[b], tol=1e-12)
        assert abs(int(it[b]) - ref.iters) <= 2
        assert np.linalg.norm(u[b] - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
        true_rel = np.linalg.norm(F[b] - op.matvec(mu[b], u[b])) / np.linalg.norm(F[b])
        assert true_rel < 1e-12 and rel[b] == pytest.approx(true_rel, rel=1e-6)


def test_greedy_with_per_training_sources_matches_oracle_and_warm_starts():
    grid, blocks = (24, 20, 18), (2, 2, 1)
    w = inputs.small(grid=grid, blocks=blocks, n_max=6, n_train=24, n_test=6)
    op = O.assemble(grid, blocks)
    mus = inputs.train_mu(w)
    Ft = R.gaussian_source(grid, gauss_params(14, len(mus)))
    ref = R.greedy_rhs(op, mus, Ft, w.n_max, snapshot_tol=1e-12)
    mtest = inputs.test_mu(w)
    Fs = R.gaussian_source(grid, gauss_params(15, len(mtest)))
    with rbws.Problem(grid, blocks) as P:
        N, sel, eta = rbws.rbws_offline_greedy_rhs(P.h, mus, torch.from_numpy(Ft).cuda(), w.n_max, 0.0, 1e-12)
        W, _, _ = rbws.rbws_get_basis(P.h)
        assert N == ref.N
        assert np.array_equal(sel, ref.selected), (sel, ref.selected)
        assert np.allclose(eta, ref.eta_hist, rtol=1e-6, equal_nan=True)
        assert np.max(np.abs(W.T @ (W @ ref.W.T) - ref.W.T)) <= 1e-8
        f = torch.from_numpy(Fs).cuda()
        u = torch.empty_like(f)
        # the Galerkin start with per-instance reduced right-hand sides: its residual is the oracle's
        rbws.rbws_solve_batch_rhs(P.h, mtest, f, 1e-12, rbws.WARM_GALERKIN, u, rbws.rbws_options_default(max_iters=0))
        u0 = u.cpu().numpy()
        for b in range(len(mtest)):
            exp = R.rb_start(ref, mtest[b], Fs[b])
            assert np.linalg.norm(u0[b] - exp) <= 1e-8 * np.linalg.norm(exp)
        # the mixed-precision start forms W^T f_b from the FP32 copy of W (FP32 products, FP64
        # sums): the same start to FP32 rounding
        rbws.rbws_solve_batch_rhs(P.h, mtest, f, 1e-12, rbws.WARM_GALERKIN, u,
                                  rbws.rbws_options_default(max_iters=0, precision=rbws.FP32_IR))
        u0 = u.cpu().numpy()
        for b in range(len(mtest)):
            exp = R.rb_start(ref, mtest[b], Fs[b])
            assert np.linalg.norm(u0[b] - exp) <= 1e-5 * np.linalg.norm(exp)
        # and the MG-preconditioned FP32 solve from it reaches the FP64 residual
        rc, it, rel, st = rbws.rbws_solve_batch_rhs(
            P.h, mtest, f, 1e-10, rbws.WARM_GALERKIN, u,
            rbws.rbws_options_default(precond=rbws.PREC_MG, precision=rbws.FP32_IR))
        uu = u.cpu().numpy()
    assert np.all(st == 0)
    for b in range(len(mtest)):
        true_rel = np.linalg.norm(Fs[b] - op.matvec(mtest[b], uu[b])) / np.linalg.norm(Fs[b])
        assert true_rel < 1e-10


# 17 and 45: the tensor-core projection (N <= 48; 2 and 3 row tiles); 100: the CUDA-core kernel
@pytest.mark.parametrize("N", [17, 45, 100])
def test_mixed_precision_start_projection_matches_oracle(N):
    """W^T f_b for the mixed-precision start (one pass over the sources, FP32 products) with an
    installed orthonormal basis of N vectors: the start equals the oracle's Galerkin RB solution
    to FP32 rounding, and the FP64 start to FP64 rounding."""
    grid, blocks = (24, 20, 18), (2, 2, 1)
    op = O.assemble(grid, blocks)
    rng = np.random.default_rng(100 + N)
    W = np.linalg.qr(rng.standard_normal((op.n, N)))[0].T.copy()      # [N][n], orthonormal rows
    ANq = np.stack([W @ np.stack([op.matvec(np.eye(op.Q)[q], W[j]) for j in range(N)]).T
                    for q in range(op.Q)])
    fN = W @ np.ones(op.n)
    basis = O.Basis(W, ANq, fN, np.zeros(0, np.int32), np.zeros(0), N)
    B = 37  # two instance groups of the projection, the second ragged
    mu = inputs.log_uniform(16, B, op.Q, 0.1, 10.0)
    Fs = R.gaussian_source(grid, gauss_params(17, B))
    exp = np.stack([R.rb_start(basis, mu[b], Fs[b]) for b in range(B)])
    with rbws.Problem(grid, blocks) as P:
        rbws.rbws_set_basis(P.h, W, ANq, fN)
        f = torch.from_numpy(Fs).cuda()
        u = torch.empty_like(f)
        got = {}
        for name, prec in (("fp32ir", rbws.FP32_IR), ("fp64", rbws.FP64)):
            rbws.rbws_solve_batch_rhs(P.h, mu, f, 1e-12, rbws.WARM_GALERKIN, u,
                                      rbws.rbws_options_default(max_iters=0, precision=prec))
            got[name] = u.cpu().numpy()
    rel = lambda x: np.linalg.norm(x - exp, axis=1) / np.linalg.norm(exp, axis=1)
    assert np.all(rel(got["fp32ir"]) <= 1e-5), rel(got["fp32ir"]).max()
    assert np.all(rel(got["fp64"]) <= 1e-10), rel(got["fp64"]).max()


def test_unsupported_starts_are_refused():
    with rbws.Problem((16, 16, 16), (2, 1, 1)) as P:
        f = torch.ones((1, P.n), dtype=torch.float64, device="cuda")
        u = torch.empty_like(f)
        with pytest.raises(rbws.RbwsError, match="UNSUPPORTED"):
            rbws.rbws_solve_batch_rhs(P.h, np.array([[1.0, 2.0]]), f, 1e-10, rbws.WARM_LEARNED, u)
        with pytest.raises(rbws.RbwsError, match="INVALID_ARG"):
            rbws.rbws_solve_batch_rhs(P.h, np.array([[1.0, 2.0]]), torch.zeros_like(f), 1e-10, rbws.WARM_ZERO, u)
