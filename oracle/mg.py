"""Multigrid V-cycle preconditioner (Algorithm 2, Sec. 2.2) and the MGCG method built on it
(Algorithm 1 with s = MG(r)), written plainly with scipy.sparse for the oracle.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the benchmark's
CPU-baseline leg, never by the product.  Shares no code with the CUDA library.

Notation follows Sec. 2.2: levels i = 0..J with J the finest (A^J = A(mu)); P_i prolongs
from level i to level i+1; the coarse operators are Galerkin products
A^i = P_i^T A^{i+1} P_i; S(u, A, b, nu) is nu smoothing steps.

Readings where the paper leaves a choice open:
  * grid hierarchy: along an axis with n nodes the coarse grid has m = n // 2 nodes, at the
    fine nodes 2, 4, ..., 2m (1-based); P is linear interpolation along each axis (tensor
    product), with the Dirichlet boundary contributing zero;
  * depth: coarsen while the level has more than MAX_COARSE = 64 unknowns and every axis has
    at least 2 nodes (64^3 gives 5 levels, J = 4, down to 4^3; the paper's experiments used
    J = 3 on their meshes);
  * smoother: damped Jacobi u <- u + omega D^-1 (b - A u), omega = 2/3, nu = 2 pre- and
    post-smoothing steps, the pre-smoothing starting from zero;
  * coarsest level: exact solve by dense Cholesky;
  * each A^i(mu) is formed as sum_q mu_q A_q^i with A_q^i = P_i^T A_q^{i+1} P_i, which equals
    the Galerkin product of A^{i+1}(mu) since P does not depend on mu.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

MAX_COARSE = 64
OMEGA = 2.0 / 3.0
NU = 2


def prolongation_1d(n: int) -> sp.csr_matrix:
    """Linear interpolation from the m = n // 2 coarse nodes (fine nodes 2J) to the n fine
    nodes: fine 2J takes coarse J, fine 2J +- 1 take half of it."""
    m = n // 2
    rows, cols, vals = [], [], []
    for J in range(1, m + 1):
        for i, w in ((2 * J - 1, 0.5), (2 * J, 1.0), (2 * J + 1, 0.5)):
            if 1 <= i <= n:
                rows.append(i - 1)
                cols.append(J - 1)
                vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, m))


def prolongation(grid) -> sp.csr_matrix:
    """3D prolongation for [z][y][x] ordering (x fastest): P = Pz (x) Py (x) Px."""
    nx, ny, nz = grid
    return sp.kron(prolongation_1d(nz), sp.kron(prolongation_1d(ny), prolongation_1d(nx))).tocsr()


def level_grids(grid) -> list:
    """Grids of levels 0..J (coarsest first)."""
    dims = [tuple(grid)]
    while True:
        nx, ny, nz = dims[-1]
        if nx * ny * nz <= MAX_COARSE or min(nx, ny, nz) < 2:
            break
        dims.append((nx // 2, ny // 2, nz // 2))
    return dims[::-1]


class Hierarchy:
    """The mu-independent part: P_i and the Galerkin coarse terms A_q^i of every level."""

    def __init__(self, op):
        self.grids = level_grids(op.grid)
        self.J = len(self.grids) - 1
        self.Q = op.Q
        fine = [sp.csr_matrix((op.vals_q[q], op.col, op.row_ptr), shape=(op.n, op.n)) for q in range(op.Q)]
        self.Aq = {self.J: fine}
        self.P = {}
        for i in range(self.J - 1, -1, -1):
            P = prolongation(self.grids[i + 1])
            self.P[i] = P
            self.Aq[i] = [(P.T @ A @ P).tocsr() for A in self.Aq[i + 1]]

    def operators(self, mu) -> "Levels":
        A = {i: sum(float(mu[q]) * self.Aq[i][q] for q in range(self.Q)).tocsr() for i in range(self.J + 1)}
        dinv = {i: 1.0 / A[i].diagonal() for i in range(self.J + 1)}
        chol = sla.cho_factor(A[0].toarray(), lower=True)
        return Levels(self, A, dinv, chol)


@dataclasses.dataclass
class Levels:
    """A^i(mu), D_i^-1 and the coarsest factor for one parameter."""
    h: Hierarchy
    A: dict
    dinv: dict
    chol: tuple


def smooth(A, dinv, b, u, nu):
    """S(u, A, b, nu): nu damped Jacobi steps; u = None is the zero initial value."""
    for _ in range(nu):
        if u is None:
            u = OMEGA * dinv * b
        else:
            u = u + OMEGA * dinv * (b - A @ u)
    return u


def vcycle(lv: Levels, b, i=None):
    """u = MG(b, A^i, i) of Algorithm 2."""
    i = lv.h.J if i is None else i
    if i == 0:
        return sla.cho_solve(lv.chol, b)
    A, dinv, P = lv.A[i], lv.dinv[i], lv.h.P[i - 1]
    u = smooth(A, dinv, b, None, NU)          # pre-smoothing from zero
    r = b - A @ u                              # residual
    rc = P.T @ r                               # restriction
    ec = vcycle(lv, rc, i - 1)                 # coarse correction (exact on level 0)
    u = u + P @ ec                             # prolongation
    return smooth(A, dinv, b, u, NU)           # post-smoothing


@dataclasses.dataclass
class MGCGResult:
    u: np.ndarray
    iters: int
    relres: float
    status: int
    hist: np.ndarray


def mgcg(op, mu, f=None, u0=None, tol=1e-10, max_iters=1000, max_restarts=3, hier=None) -> MGCGResult:
    """Algorithm 1 with the preconditioner s = MG(r), plus the true-residual check and restarts
    of Algorithm 4 (the same loop as the oracle's Jacobi PCG).  Status 0 converged, 1 max
    iterations, 2 breakdown."""
    hier = Hierarchy(op) if hier is None else hier
    lv = hier.operators(mu)
    A = lv.A[hier.J]
    f = np.ones(op.n) if f is None else np.asarray(f, dtype=np.float64)
    u = np.zeros(op.n) if u0 is None else np.array(u0, dtype=np.float64)
    fnorm = np.linalg.norm(f)
    hist = [np.nan] * (max_iters + 1)
    k, status, rel = 0, 0, 0.0
    for attempt in range(max_restarts + 1):
        r = f - A @ u
        rel = np.linalg.norm(r) / fnorm
        if attempt == 0:
            hist[0] = rel
        if rel < tol:
            status = 0
            break
        if k >= max_iters:
            status = 1
            break
        s = vcycle(lv, r)
        p = s.copy()
        rs = r @ s
        status = 1
        while rel >= tol and k < max_iters:
            q = A @ p
            pq = p @ q
            if not pq > 0.0:
                status = 2
                break
            alpha = rs / pq
            u = u + alpha * p
            r = r - alpha * q
            s = vcycle(lv, r)
            rs_new = r @ s
            beta = rs_new / rs
            rs = rs_new
            p = s + beta * p
            k += 1
            rel = np.linalg.norm(r) / fnorm
            hist[k] = rel
        if status == 2:
            break
        if rel >= tol:
            status = 1
            break
        status = 0
        if attempt == max_restarts:
            rel = np.linalg.norm(f - A @ u) / fnorm
            if rel >= tol:
                status = 1
    return MGCGResult(u, k, rel, status, np.array(hist[: k + 1]))
