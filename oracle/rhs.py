"""Per-instance right-hand sides for the oracle: the Gaussian source (a non-affine f(mu), the
shape of the paper's Example 2, Sec. 4) and the greedy RB of Algorithm 5 with one right-hand
side per training parameter, written plainly with numpy on top of the oracle's C operator and
PCG.

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product.  Shares no code with
the CUDA library.

Readings where the paper leaves a choice open (the same as the oracle's fixed-f greedy):
  * first parameter: index 0 of the training set;
  * Gram-Schmidt twice against the current basis; a snapshot whose orthogonal part is below
    1e-10 of its norm ends the greedy (no new direction);
  * indicator: ||f_t - A(mu_t) W c_t|| / ||f_t|| with the Galerkin coefficients
    A_N(mu_t) c_t = W^T f_t; the largest over the training points not yet selected, ties to
    the smallest index.
"""
from __future__ import annotations

import numpy as np

from . import Basis, assemble, pcg  # noqa: F401  (assemble re-exported for callers)


def gaussian_source(grid, params) -> np.ndarray:
    """f[b] = exp(-|x - c_b|^2 / (2 s_b^2)) at the interior nodes x = ((i+1)/(nx+1), ...), in
    [z][y][x] order; params [B][4] = (c_x, c_y, c_z, s_b)."""
    nx, ny, nz = grid
    x = np.arange(1, nx + 1) / (nx + 1)
    y = np.arange(1, ny + 1) / (ny + 1)
    z = np.arange(1, nz + 1) / (nz + 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    out = []
    for cx, cy, cz, sg in np.atleast_2d(params):
        d2 = (X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2
        out.append(np.exp(-d2 / (2.0 * sg * sg)).ravel())
    return np.array(out)


def node_coordinates(grid, neumann=(0, 0, 0)):
    """Coordinates of the nodes along each axis: i/(n+1), or i/n on an axis with a Neumann face
    at coordinate 1 (i = 1..n)."""
    return [np.arange(1, n + 1) / (n if nm else n + 1) for n, nm in zip(grid, neumann)]


def example2_source(grid, params, neumann=(1, 0, 0)) -> np.ndarray:
    """The source of the paper's Example 2 (Sec. 4), f = mu7 + exp(-|x - (mu4, mu5, mu6)|^2 / mu7) / mu7,
    at the nodes, times each node's relative control volume (the right-hand side of the
    finite-volume system of orc_assemble_ex); params [B][4] = (mu4, mu5, mu6, mu7)."""
    from . import node_weights
    x, y, z = node_coordinates(grid, neumann)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    w = node_weights(grid, neumann)
    out = []
    for c4, c5, c6, m7 in np.atleast_2d(params):
        d2 = (X - c4) ** 2 + (Y - c5) ** 2 + (Z - c6) ** 2
        out.append((m7 + np.exp(-d2 / m7) / m7).ravel() * w)
    return np.array(out)


def greedy_rhs(op, mu_train, F_train, n_max, snapshot_tol=1e-12) -> Basis:
    """Algorithm 5's loop (Galerkin RB, residual indicator) with right-hand side F_train[t] for
    training parameter t."""
    mu_train = np.asarray(mu_train, dtype=np.float64)
    F = np.asarray(F_train, dtype=np.float64)
    n_train = mu_train.shape[0]
    W = []
    sel, eta_hist = [], []
    taken = np.zeros(n_train, dtype=bool)
    nxt = 0
    while len(W) < n_max:
        u = pcg(op, mu_train[nxt], f=F[nxt], tol=snapshot_tol, max_iters=100000).u
        w = u.copy()
        for _ in range(2):
            for v in W:
                w -= (v @ w) * v
        if not np.linalg.norm(w) >= 1e-10 * np.linalg.norm(u):
            break
        W.append(w / np.linalg.norm(w))
        sel.append(nxt)
        taken[nxt] = True
        Wa = np.array(W)
        eta = np.full(n_train, -1.0)
        for t in range(n_train):
            if taken[t]:
                continue
            AW = np.array([op.matvec(mu_train[t], v) for v in Wa])   # rows A(mu_t) w_j
            c = np.linalg.solve(Wa @ AW.T, Wa @ F[t])
            eta[t] = np.linalg.norm(F[t] - c @ AW) / np.linalg.norm(F[t])
        if taken.all():
            eta_hist.append(np.nan)
            break
        nxt = int(np.argmax(eta))
        eta_hist.append(float(eta[nxt]))
    Wa = np.array(W)
    Q = op.Q
    ANq = np.zeros((Q, len(W), len(W)))
    for q in range(Q):
        e = np.eye(Q)[q]
        ANq[q] = Wa @ np.array([op.matvec(e, v) for v in Wa]).T
    fN = Wa @ np.ones(op.n)
    return Basis(Wa, ANq, fN, np.array(sel, dtype=np.int32), np.array(eta_hist), len(W))


def rb_start(basis: Basis, mu, f) -> np.ndarray:
    """The Galerkin RB solution W^T c with A_N(mu) c = W^T f (reduced system from the affine terms)."""
    A = np.tensordot(np.asarray(mu, dtype=np.float64), basis.ANq, axes=1)
    c = np.linalg.solve(A, basis.W @ np.asarray(f, dtype=np.float64))
    return basis.W.T @ c


def example1_rhs(F, L1, L2, mu) -> np.ndarray:
    """Right-hand sides of the paper's Example 1 (Sec. 4) for parameters mu [B][2]: the source
    F [n] plus the Dirichlet lift of g_D(mu) = (1 - mu_2) G1 + mu_2 G2 through
    A(mu) = A_0 + mu_1 A_1, with L1 = dirichlet_lift(G1), L2 = dirichlet_lift(G2) ([2][n] each):
    b = F + (1 - mu_2) (L1_0 + mu_1 L1_1) + mu_2 (L2_0 + mu_1 L2_1)."""
    out = []
    for m1, m2 in np.atleast_2d(mu):
        out.append(F + (1.0 - m2) * (L1[0] + m1 * L1[1]) + m2 * (L2[0] + m1 * L2[1]))
    return np.array(out)


def example1_affine(mu) -> np.ndarray:
    """theta_A [B][2] = (1, mu_1): the coefficients of A(mu) = A_0 + mu_1 A_1 in Example 1."""
    mu = np.atleast_2d(mu)
    return np.column_stack([np.ones(mu.shape[0]), mu[:, 0]])
