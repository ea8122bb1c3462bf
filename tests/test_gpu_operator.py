"""Parity of the matrix-free CUDA stencil (Eq. 1, 7-point diffusion operator) with the
oracle's explicit CSR matvec, element by element, on ragged multi-tile grids."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2311_13862_gb300 import inputs, rbws

pytestmark = pytest.mark.gpu

CASES = [((9, 7, 5), (2, 1, 1)), ((16, 16, 16), (2, 1, 1)), ((33, 17, 20), (2, 2, 2)),
         ((64, 64, 64), (2, 2, 1)), ((37, 41, 29), (3, 3, 3)), ((2, 2, 2), (1, 1, 1)),
         ((130, 9, 11), (3, 1, 2))]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2311_13862_gb300 import build
    build.build()


@pytest.mark.parametrize("grid,blocks", CASES)
def test_apply_fp64_matches_csr(grid, blocks):
    op = O.assemble(grid, blocks)
    B = 3
    mu = inputs.log_uniform(41, B, op.Q, 0.01, 100.0)
    x = inputs.random_field(42, (B, op.n))
    ref = np.stack([op.matvec(mu[b], x[b]) for b in range(B)])
    with rbws.Problem(grid, blocks) as P:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        rbws.rbws_apply_operator(P.h, mu, xd, yd, rbws.FP64)
        y = yd.cpu().numpy()
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.max(np.abs(y - ref) / scale) <= 1e-14


@pytest.mark.parametrize("grid,blocks", CASES[:5])
def test_apply_fp32_matches_csr(grid, blocks):
    op = O.assemble(grid, blocks)
    B = 2
    mu = inputs.log_uniform(43, B, op.Q, 0.1, 10.0)
    x = inputs.random_field(44, (B, op.n)).astype(np.float32)
    ref = np.stack([op.matvec(mu[b], x[b].astype(np.float64)) for b in range(B)])
    with rbws.Problem(grid, blocks) as P:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        rbws.rbws_apply_operator(P.h, mu, xd, yd, rbws.FP32_IR)
        y = yd.cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    # 7 terms with coefficients up to ~1e2/h^2: FP32 rounding of each product
    assert np.max(np.abs(y - ref) / scale) <= 1e-5


def test_apply_many_instances_and_full_size_sample():
    """Full-size 64^3 grid with 256 instances, as the online workload launches it; sampled
    rows checked against the CSR operator."""
    w = inputs.WORKLOADS["c2"]
    op = O.assemble(w.grid, w.blocks)
    B = 256
    mu = inputs.test_mu(w)
    x = torch.from_numpy(inputs.random_field(45, (B, op.n))).cuda()
    y = torch.empty_like(x)
    with rbws.Problem(w.grid, w.blocks) as P:
        rbws.rbws_apply_operator(P.h, mu, x, y, rbws.FP64)
    for b in (0, 17, 255):
        ref = op.matvec(mu[b], x[b].cpu().numpy())
        got = y[b].cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-14 * np.abs(ref).max()
