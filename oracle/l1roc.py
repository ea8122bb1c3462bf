"""L1-based reduced over-collocation (L1ROC, Sec. 3.1): the offline greedy (Algorithm 5 with
DEIM on snapshots and on RB residuals) and the online over-collocation least-squares solve,
written plainly with numpy on top of the oracle's C operator and PCG.

TEST INFRASTRUCTURE ONLY: imported by the tests and the benchmark's CPU-baseline leg, never
by the product.  Shares no code with the CUDA library.

Readings where the paper leaves a choice open:
  * first parameter: index 0 of the training set (the paper draws it at random);
  * DEIM(V, v): with V's interpolation points p, c solves V[p] c = v[p]; the residual
    rho = v - V c vanishes at p; the new point is the smallest node index with
    |rho| >= (1 - 1e-8) max |rho| (near-ties, which mirror symmetries of the grid and the
    blocks make exact in exact arithmetic, resolve to the smaller index whatever the
    rounding) and the new vector is rho / rho[point] (one at its own point, zero at the
    earlier ones);
  * the online problem minimises ||P (b - A W c)||_2 (the paper's "argmax" read as argmin)
    over the points X^m = X_s u X_r, kept in the order they were added; a point found by
    both DEIM processes is kept once;
  * the L1 indicator is ||c_U||_1 with u_rb = W c = U c_U, U the snapshots: U = W T with T
    upper triangular, column k = (DEIM coefficients of snapshot k, rho_k[point_k]);
  * the greedy picks the largest indicator among the training points not yet selected and
    stops at N, or when a snapshot adds nothing new: max |rho| <= 1e-10 max |u| (the same
    breakdown rule as the Galerkin greedy's Gram-Schmidt, in the max norm); a residual
    that small adds no residual point.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from . import pcg as _pcg


@dataclasses.dataclass
class L1ROCBasis:
    W: np.ndarray          # [N][n] DEIM basis (u_k = W^T T[:, k])
    T: np.ndarray          # [N][N] upper triangular
    pts: np.ndarray        # collocation nodes X^m, in the order they were added
    pts_s: np.ndarray      # DEIM points of the snapshots (N)
    pts_r: np.ndarray      # DEIM points of the RB residuals (N - 1)
    R: np.ndarray          # [N-1][n] DEIM basis of the residuals
    selected: np.ndarray
    eta_hist: np.ndarray   # eta_hist[k]: largest L1 indicator over the unselected points, k+1 vectors
    N: int


def deim_step(V, pts, v):
    """One DEIM step on v against the vectors V (rows) with interpolation points pts.
    Returns (new vector, new point, coefficients c, rho[point])."""
    v = np.asarray(v, dtype=np.float64)
    k = len(pts)
    if k:
        Vm = np.asarray(V, dtype=np.float64)[:k]
        c = np.linalg.solve(Vm[:, pts].T, v[pts])
        rho = v - Vm.T @ c
    else:
        c = np.zeros(0)
        rho = v.copy()
    a = np.abs(rho)
    x = int(np.flatnonzero(a >= (1.0 - 1e-8) * a.max())[0])  # first of the (near-)largest
    return rho / rho[x], x, c, float(rho[x])


def colloc_solve(op, W, pts, mu, f=None, n=None):
    """c = argmin ||P (f - A(mu) W^T c)||_2 over the nodes pts (numpy least squares)."""
    n = W.shape[0] if n is None else n
    f = np.ones(op.n) if f is None else np.asarray(f, dtype=np.float64)
    G = np.stack([op.matvec(mu, W[j])[pts] for j in range(n)], axis=1)
    c, *_ = np.linalg.lstsq(G, f[pts], rcond=None)
    return c


def l1_indicator(T, c):
    """||c_U||_1 with W c = U c_U and U = W T (T upper triangular)."""
    n = len(c)
    return float(np.abs(sla.solve_triangular(T[:n, :n], c, lower=False)).sum())


def offline(op, mu_train, N, f=None, snapshot_tol=1e-12) -> L1ROCBasis:
    """Algorithm 5 (offline L1ROC)."""
    mu_train = np.asarray(mu_train, dtype=np.float64)
    f = np.ones(op.n) if f is None else np.asarray(f, dtype=np.float64)
    n_train = mu_train.shape[0]
    W, R, pts_s, pts_r, pts = [], [], [], [], []
    T = np.zeros((N, N))
    selected, eta_hist = [], np.full(N, np.nan)
    taken = np.zeros(n_train, dtype=bool)
    nxt = 0
    while len(W) < N:
        u = _pcg(op, mu_train[nxt], f=f, tol=snapshot_tol, max_iters=100000).u
        w, x, c, s = deim_step(W, pts_s, u)
        if not abs(s) > 1e-10 * np.max(np.abs(u)):
            break
        k = len(W)
        new_pts = [x]
        if k:
            # the RB residual of the new parameter with the current space, then its DEIM point
            crb = colloc_solve(op, np.array(W), pts, mu_train[nxt], f)
            r = f - op.matvec(mu_train[nxt], np.array(W).T @ crb)
            rw, xr, _, sr = deim_step(R, pts_r, r)
            if abs(sr) > 1e-10 * np.max(np.abs(f)):
                R.append(rw)
                pts_r.append(xr)
                new_pts.append(xr)
        T[:k, k] = c
        T[k, k] = s
        W.append(w)
        pts_s.append(x)
        # X^m = X_s u X_r in the order of addition (snapshot point first)
        for q in new_pts:
            if q not in pts:
                pts.append(q)
        selected.append(nxt)
        taken[nxt] = True
        Wa = np.array(W)
        eta = np.full(n_train, -1.0)
        for t in range(n_train):
            if not taken[t]:
                eta[t] = l1_indicator(T, colloc_solve(op, Wa, pts, mu_train[t], f))
        if taken.all():
            break
        nxt = int(np.argmax(eta))
        eta_hist[len(W) - 1] = eta[nxt]
    Nb = len(W)
    return L1ROCBasis(np.array(W), T[:Nb, :Nb].copy(), np.array(pts, dtype=np.int64),
                      np.array(pts_s, dtype=np.int64), np.array(pts_r, dtype=np.int64),
                      np.array(R).reshape(len(R), op.n), np.array(selected, dtype=np.int64),
                      eta_hist[:Nb].copy(), Nb)
