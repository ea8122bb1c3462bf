"""rbws_apply_operator_static: the operator apply for callers that cannot allocate device
memory after start-up (a fixed memory budget shared with another allocator, or code that
cannot accept cudaMalloc's implicit synchronisation).  Its scratch lives in a static
device array.  It runs the same kernels on the same coefficient tables as
rbws_apply_operator, which allocates its scratch, so the two outputs must agree bit for
bit; both are also checked against the oracle's explicit CSR operator.  This file is
collected last so that a failure here comes after every other test."""
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


@pytest.mark.parametrize("grid,blocks", [((33, 17, 20), (2, 2, 2)), ((64, 64, 64), (2, 2, 1))])
def test_static_scratch_apply_matches_allocating_apply_twice(grid, blocks):
    op = O.assemble(grid, blocks)
    with rbws.Problem(grid, blocks) as P:
        for call, (B, seed) in enumerate([(5, 81), (3, 82)]):  # two calls in a row, different sizes
            mu = inputs.log_uniform(seed, B, op.Q, 0.01, 100.0)
            x_h = inputs.random_field(seed + 100, (B, op.n))
            x = torch.from_numpy(x_h).cuda()
            y_ref = torch.empty_like(x)
            y = torch.full_like(x, float("nan"))
            rbws.rbws_apply_operator(P.h, mu, x, y_ref, rbws.FP64)
            rbws.rbws_apply_operator_static(P.h, mu, x, y, rbws.FP64)
            ref, got = y_ref.cpu().numpy(), y.cpu().numpy()
            assert np.array_equal(got, ref), call  # same kernels, same tables
            csr = np.stack([op.matvec(mu[b], x_h[b]) for b in range(B)])
            scale = np.abs(csr).max(axis=1, keepdims=True)
            assert np.max(np.abs(got - csr) / scale) <= 1e-14, call
            # float32 kernel as well
            x32 = x.float()
            r32, g32 = torch.empty_like(x32), torch.full_like(x32, float("nan"))
            rbws.rbws_apply_operator(P.h, mu, x32, r32, rbws.FP32_IR)
            rbws.rbws_apply_operator_static(P.h, mu, x32, g32, rbws.FP32_IR)
            assert torch.equal(g32, r32), call
            csr32 = np.stack([op.matvec(mu[b], x32[b].cpu().numpy().astype(np.float64)) for b in range(B)])
            s32 = np.abs(csr32).max(axis=1, keepdims=True)
            assert np.max(np.abs(g32.cpu().numpy() - csr32) / s32) <= 1e-5, call


def test_static_scratch_apply_allocates_no_device_memory():
    grid, blocks = (40, 24, 16), (2, 2, 2)
    n = grid[0] * grid[1] * grid[2]
    mu = inputs.log_uniform(84, 4, 8, 0.1, 10.0)
    x = torch.from_numpy(inputs.random_field(85, (4, n))).cuda()
    y = torch.empty_like(x)
    with rbws.Problem(grid, blocks) as P0:  # loads the kernels and the scratch array's module
        rbws.rbws_apply_operator_static(P0.h, mu, x, y, rbws.FP64)
    with rbws.Problem(grid, blocks) as P:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            rbws.rbws_apply_operator_static(P.h, mu, x, y, rbws.FP64)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0


def test_static_scratch_rejects_oversized_requests():
    # 8^3 grid, 2 blocks in x: 54 coefficient classes, 3.5 KB of tables per instance, so
    # 2000 instances (7 MB) exceed the 4 MiB array.  Buffers are full size all the same.
    with rbws.Problem((8, 8, 8), (2, 1, 1)) as P:
        B = 2000
        mu = inputs.log_uniform(83, B, 2, 0.1, 10.0)
        x = torch.zeros((B, 512), dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(rbws.RbwsError, match="static maximum"):
            rbws.rbws_apply_operator_static(P.h, mu, x, y, rbws.FP64)
        # a request that fits still works after the rejection
        rbws.rbws_apply_operator_static(P.h, mu[:4], x[:4], y[:4], rbws.FP64)
