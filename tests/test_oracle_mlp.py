"""Pins of the oracle's warm-start network (p -> H -> H -> H -> N, GELU with erf)."""
import numpy as np
import torch

import oracle as O


def torch_reference(p, H, N, params, x):
    """Same network from torch.nn layers in float64 (an independent implementation)."""
    layers, off = [], 0
    for (i, o) in [(p, H), (H, H), (H, H), (H, N)]:
        lin = torch.nn.Linear(i, o).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(params[off:off + i * o].reshape(o, i)))
            off += i * o
            lin.bias.copy_(torch.from_numpy(params[off:off + o]))
            off += o
        layers += [lin, torch.nn.GELU(approximate="none")]
    net = torch.nn.Sequential(*layers[:-1])
    return net(torch.from_numpy(x)).detach().numpy()


def test_param_count():
    assert O.mlp_param_count(8, 256, 40) == 8 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 40 + 40


def test_forward_matches_torch_layers():
    p, H, N = 4, 16, 5
    rng = np.random.default_rng(0)
    params = rng.standard_normal(O.mlp_param_count(p, H, N)) * 0.5
    x = rng.uniform(-1, 1, (7, p))
    y = O.mlp_forward(p, H, N, params, x)
    assert np.max(np.abs(y - torch_reference(p, H, N, params, x))) <= 1e-13 * np.max(np.abs(y))


def test_gradient_central_differences():
    p, H, N = 4, 8, 3
    rng = np.random.default_rng(1)
    params = rng.standard_normal(O.mlp_param_count(p, H, N)) * 0.7
    x = rng.uniform(-1, 1, (5, p))
    t = rng.standard_normal((5, N))
    loss, g = O.mlp_loss_grad(p, H, N, params, x, t)
    y = O.mlp_forward(p, H, N, params, x)
    assert abs(loss - np.mean((y - t) ** 2)) <= 1e-14 * loss
    eps = 1e-6
    fd = np.empty_like(params)
    for k in range(params.size):
        e = np.zeros_like(params)
        e[k] = eps
        fd[k] = (O.mlp_loss_grad(p, H, N, params + e, x, t)[0]
                 - O.mlp_loss_grad(p, H, N, params - e, x, t)[0]) / (2 * eps)
    assert np.max(np.abs(fd - g)) <= 1e-6 * max(1.0, np.max(np.abs(g)))


def test_gradient_matches_torch_autograd():
    p, H, N = 3, 12, 4
    rng = np.random.default_rng(2)
    params = rng.standard_normal(O.mlp_param_count(p, H, N)) * 0.4
    x = rng.uniform(-1, 1, (9, p))
    t = rng.standard_normal((9, N))
    _, g = O.mlp_loss_grad(p, H, N, params, x, t)
    pt = torch.tensor(params, requires_grad=True)
    off, h = 0, torch.from_numpy(x)
    for li, (i, o) in enumerate([(p, H), (H, H), (H, H), (H, N)]):
        Wl = pt[off:off + i * o].reshape(o, i)
        off += i * o
        bl = pt[off:off + o]
        off += o
        h = h @ Wl.T + bl
        if li < 3:
            h = torch.nn.functional.gelu(h)
    loss = ((h - torch.from_numpy(t)) ** 2).mean()
    loss.backward()
    assert np.max(np.abs(pt.grad.numpy() - g)) <= 1e-13 * np.max(np.abs(g))
