"""Learned warm start: the GPU network (BF16 tensor-core operands, FP32 accumulation) against
the oracle's FP64 network on the same weights, and what training buys over a zero start."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2311_13862_gb300 import inputs, rbws

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2311_13862_gb300 import build
    build.build()


def bf16_round(a):
    """Round float64 values to bfloat16 (round to nearest even), back to float64."""
    t = torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.to(torch.float64).numpy()


def normalised(mu, lo, hi):
    return 2.0 * (np.log(mu) - np.log(lo)) / (np.log(hi) - np.log(lo)) - 1.0


@pytest.fixture(scope="module")
def small_problem():
    w = inputs.small(grid=(16, 16, 12), blocks=(2, 2, 1), n_max=6, n_train=24, n_test=6)
    op = O.assemble(w.grid, w.blocks)
    basis = O.greedy(op, inputs.train_mu(w), w.n_max)
    return w, op, basis


@pytest.mark.parametrize("H", [32, 256])
def test_forward_matches_oracle(small_problem, H):
    w, op, basis = small_problem
    p, N = op.Q, basis.N
    rng = np.random.default_rng(5)
    params = bf16_round(rng.standard_normal(O.mlp_param_count(p, H, N)) / np.sqrt(H))
    scale = np.linspace(0.5, 2.0, N)
    mu = inputs.log_uniform(6, 40, p, 0.1, 10.0)
    with rbws.Problem(w.grid, w.blocks) as P:
        rbws.rbws_set_basis(P.h, basis.W, basis.ANq, basis.fN)
        rbws.rbws_surrogate_set_params(P.h, H, params, scale, 0.1, 10.0)
        c = rbws.rbws_surrogate_forward(P.h, mu)
    ref = O.mlp_forward(p, H, N, params, normalised(mu, 0.1, 10.0)) * scale
    assert np.max(np.abs(c - ref)) <= 1e-2 * np.max(np.abs(ref))


def test_gradients_match_oracle(small_problem):
    w, op, basis = small_problem
    p, N, H = op.Q, basis.N, 64
    rng = np.random.default_rng(7)
    params = bf16_round(rng.standard_normal(O.mlp_param_count(p, H, N)) / np.sqrt(H))
    x = rng.uniform(-1, 1, (48, p))
    t = rng.standard_normal((48, N))
    with rbws.Problem(w.grid, w.blocks) as P:
        rbws.rbws_set_basis(P.h, basis.W, basis.ANq, basis.fN)
        rbws.rbws_surrogate_set_params(P.h, H, params)
        loss, g = rbws.rbws_surrogate_loss_grad(P.h, x, t)
    loss_ref, g_ref = O.mlp_loss_grad(p, H, N, params, x, t)
    assert loss == pytest.approx(loss_ref, rel=1e-2)
    # per tensor (W1 b1 W2 b2 W3 b3 W4 b4): relative L2 error
    sizes = [H * p, H, H * H, H, H * H, H, N * H, N]
    off = 0
    for k, sz in enumerate(sizes):
        a, b = g[off:off + sz].astype(np.float64), g_ref[off:off + sz]
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b), k
        off += sz


def test_initial_parameters_and_first_adam_step_match_oracle(small_problem):
    """epochs = 0 installs the starting parameters: bitwise the oracle's draw (splitmix64 as
    the header states it).  One epoch of one minibatch is one Adam step from them: the scales
    and the loss at the start match the oracle's FP64 network, and every parameter moves as
    the oracle's Adam step on the oracle's FP64 gradient (about lr against the gradient's
    sign), except where the BF16 operands' rounding decides a sign."""
    from oracle import mlp_train as T
    w, op, basis = small_problem
    p, N, H, seed, lr = op.Q, basis.N, 32, 11, 1e-3
    mu = inputs.surrogate_mu(w, 64)
    kw = dict(hidden=H, batch=64, lr=lr, mu_lo=w.mu_lo, mu_hi=w.mu_hi, seed=seed)
    with rbws.Problem(w.grid, w.blocks) as P:
        rbws.rbws_set_basis(P.h, basis.W, basis.ANq, basis.fN)
        rbws.rbws_train_surrogate(P.h, mu, epochs=0, **kw)
        H0, theta0, scale0 = rbws.rbws_surrogate_get_params(P.h)
        loss1 = rbws.rbws_train_surrogate(P.h, mu, epochs=1, **kw)
        _, theta1, scale1 = rbws.rbws_surrogate_get_params(P.h)
    assert H0 == H
    assert np.array_equal(theta0, T.init_params(p, H, N, seed))
    C = np.stack([O.rb_solve(basis.ANq, basis.fN, m) for m in mu])
    np.testing.assert_allclose(scale0, T.rms_scale(C), rtol=1e-6)
    assert np.array_equal(scale1, scale0)
    x = T.normalise(mu, w.mu_lo, w.mu_hi)
    loss_ref, g = O.mlp_loss_grad(p, H, N, theta0.astype(np.float64), x, C / scale0.astype(np.float64))
    assert loss1 == pytest.approx(loss_ref, rel=3e-2)
    step = theta1.astype(np.float64) - theta0.astype(np.float64)
    ref_step = T.adam(theta0, 0.0, 0.0, g, 1, lr)[0] - theta0.astype(np.float64)
    assert np.all(np.abs(step) <= lr * (1 + 1e-4))
    for name, a, e, _ in T.layer_segments(p, H, N):
        ga = g[a:e]
        clear = np.abs(ga) > 0.1 * np.sqrt(np.mean(ga * ga))
        off = np.abs(step[a:e] - ref_step[a:e]) > 1e-2 * lr
        assert np.count_nonzero(off & clear) <= max(1, int(0.01 * np.count_nonzero(clear))), name


@pytest.fixture(scope="module")
def halves_problem():
    """16^3, two half-cubes: the RB warm start pays off here (N = 10)."""
    w = inputs.WORKLOADS["c1"]
    op = O.assemble(w.grid, w.blocks)
    basis = O.greedy(op, inputs.train_mu(w), w.n_max)
    return w, op, basis


def test_trained_network_gains_over_zero_start(halves_problem):
    """The network is trained on the GPU on Galerkin coefficients; its warm start must be
    closer to the solution than a zero start and save iterations.  (The residual 2-norm of a
    reduced start can exceed that of u0 = 0 on these block-coefficient problems: it is
    dominated by interface rows, so the error is compared instead.  By Galerkin optimality no
    learned c beats the Galerkin start in the A-norm.)"""
    w, op, basis = halves_problem
    mu_train = inputs.surrogate_mu(w, 1024)
    mu = inputs.test_mu(w)
    with rbws.Problem(w.grid, w.blocks) as P:
        rbws.rbws_set_basis(P.h, basis.W, basis.ANq, basis.fN)
        loss = rbws.rbws_train_surrogate(P.h, mu_train, hidden=64, epochs=1500, batch=128, lr=1e-3,
                                         mu_lo=w.mu_lo, mu_hi=w.mu_hi, seed=1)
        assert loss < 1e-2
        c_net = rbws.rbws_surrogate_forward(P.h, mu)
        c_gal = rbws.rbws_reduced_solve(P.h, mu)
        rel_c = np.linalg.norm(c_net - c_gal, axis=1) / np.linalg.norm(c_gal, axis=1)
        assert np.median(rel_c) < 0.1
        res = {}
        for name, warm in [("zero", rbws.WARM_ZERO), ("learned", rbws.WARM_LEARNED),
                           ("corrected", rbws.WARM_LEARNED_CORRECTED), ("galerkin", rbws.WARM_GALERKIN)]:
            u = torch.empty((len(mu), P.n), dtype=torch.float64, device="cuda")
            rc, it, rel, st = rbws.rbws_solve_batch(P.h, mu, 1e-10, warm, u)
            assert rc == 0 and np.all(st == 0)
            res[name] = it
        # the oracle's own solves give the same picture on the learned coefficients
        lw = O.solve_batch(op, mu, warm=O.WARM_GIVEN, basis=basis, c_given=c_net, tol=1e-10)
        z = O.solve_batch(op, mu, warm=O.WARM_ZERO, tol=1e-12)
    u_star = z.u
    err_l = np.linalg.norm(c_net @ basis.W - u_star, axis=1) / np.linalg.norm(u_star, axis=1)
    err_g = np.linalg.norm(c_gal @ basis.W - u_star, axis=1) / np.linalg.norm(u_star, axis=1)
    print("iterations", {k: float(v.mean()) for k, v in res.items()}, "oracle learned", lw.iters.mean(),
          "rel err learned %.3g galerkin %.3g" % (err_l.mean(), err_g.mean()),
          "relres0 learned", np.round(lw.relres0, 3))
    assert err_l.mean() < 0.05 and np.all(err_l < 0.3)  # a zero start has relative error 1
    assert res["learned"].mean() < res["zero"].mean()
    assert res["corrected"].mean() <= res["learned"].mean() + 2
