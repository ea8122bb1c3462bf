"""Pins of the oracle's training set-up for the learned warm start (oracle/mlp_train.py): the
generator against its check values, the parameter draw against the layout and the uniform
law it states, Adam against torch's implementation of the same algorithm."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import mlp_train as T


def test_splitmix64_check_values_from_state_zero():
    # the first outputs of splitmix64 from state 0, the values the generator is usually
    # checked against
    assert T.splitmix64(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


@pytest.mark.parametrize("seed", [0, 11, 3004, (1 << 64) - 5])
def test_direct_outputs_equal_the_sequential_generator(seed):
    seq = T.splitmix64(seed, 50)
    direct = T._splitmix64_at(seed, np.arange(50))
    assert [int(v) for v in direct] == seq


@pytest.mark.parametrize("p,H,N", [(4, 32, 6), (2, 256, 20), (8, 64, 40)])
def test_layout_matches_the_oracle_network(p, H, N):
    segs = T.layer_segments(p, H, N)
    assert segs[0][1] == 0
    assert all(segs[k][2] == segs[k + 1][1] for k in range(len(segs) - 1))
    assert segs[-1][2] == O.mlp_param_count(p, H, N)
    assert [s[3] for s in segs] == [p, p, H, H, H, H, H, H]


def test_initial_parameters_follow_the_stated_draw():
    p, H, N, seed = 4, 256, 20, 3004
    w = T.init_params(p, H, N, seed)
    assert w.dtype == np.float32 and w.shape == (O.mlp_param_count(p, H, N),)
    # parameter 0 by hand from the sequential generator
    z = T.splitmix64(seed, 1)[0]
    u = (z >> 11) / 2.0 ** 53
    assert w[0] == np.float32((2.0 * u - 1.0) * float(np.float32(1.0 / np.sqrt(p))))
    for name, a, e, fan_in in T.layer_segments(p, H, N):
        b = float(np.float32(1.0 / np.sqrt(fan_in)))
        x = w[a:e].astype(np.float64)
        assert np.all(np.abs(x) <= b), name
        if e - a >= 4096:  # uniform on [-b, b]: mean 0, variance b^2 / 3
            assert abs(x.mean()) < 4 * b / np.sqrt(3 * (e - a)), name
            assert x.var() == pytest.approx(b * b / 3, rel=0.05), name
    assert not np.array_equal(w, T.init_params(p, H, N, seed + 1))
    assert np.array_equal(w, T.init_params(p, H, N, seed))


def test_adam_equals_torch_adam():
    rng = np.random.default_rng(3)
    theta0 = rng.standard_normal(200)
    grads = [rng.standard_normal(200) * s for s in (1.0, 1e-3, 5.0, 1e-9)]
    th = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([th], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    theta, m, v = theta0.copy(), np.zeros(200), np.zeros(200)
    for t, g in enumerate(grads, start=1):
        opt.zero_grad()
        th.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        theta, m, v = T.adam(theta, m, v, g, t, 1e-3)
        np.testing.assert_allclose(theta, th.detach().numpy(), rtol=0, atol=1e-15)


def test_first_adam_step_moves_every_parameter_by_about_lr():
    g = np.array([3.0, -2e-4, 1e-8, 0.0, -7.5])
    theta, _, _ = T.adam(np.zeros(5), np.zeros(5), np.zeros(5), g, 1, 1e-3)
    np.testing.assert_allclose(theta, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_scales_and_inputs():
    C = np.array([[3.0, 0.0, 1.0], [-3.0, 0.0, 2.0], [3.0, 0.0, 2.0]])
    s = T.rms_scale(C)
    assert s.dtype == np.float32
    np.testing.assert_allclose(s, [3.0, 1.0, np.sqrt(3.0)], rtol=1e-7)
    np.testing.assert_allclose(np.sqrt(np.mean((C[:, [0, 2]] / s[[0, 2]]) ** 2, axis=0)), 1.0, rtol=1e-7)
    x = T.normalise(np.array([[0.1, 10.0, 1.0]]), 0.1, 10.0)
    np.testing.assert_allclose(x, [[-1.0, 1.0, 0.0]], atol=1e-15)
