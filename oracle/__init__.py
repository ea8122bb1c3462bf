"""CPU FP64 oracle of the reduced basis warm-start method (arXiv 2311.13862).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this package; the product path never
does.  It shares nothing with the CUDA library: the arithmetic lives in
rbws_oracle.c (plain C, FP64, explicit CSR), and this module only marshals
numpy arrays through ctypes.

Function map (paper passage -> function):
  Eq. (1), Sec. 4 model problem        assemble(), Operator.matvec(); assemble_mu() (one mu)
  Algorithm 1 (PCG), Algorithm 4       pcg()
  Sec. 2.3 RB system (Galerkin)        rb_solve(), cholesky()
  Algorithm 3 (MSRB preconditioner)    pcg(precond=MSRB), solve_batch(precond=MSRB)
  Algorithm 5 skeleton (greedy)        greedy()
  Algorithm 4 over a batch             solve_batch()
  Algorithm 2 (MG V-cycle), MGCG       oracle.mg: Hierarchy, vcycle(), mgcg() (numpy/scipy)
  Sec. 3.1 L1ROC (Algorithm 5, DEIM,   oracle.l1roc: offline(), colloc_solve(), l1_indicator()
    over-collocation)                    (numpy)
  learned warm start network           mlp_forward(), mlp_loss_grad()
  its training set-up (starting draw,  oracle.mlp_train: init_params(), rms_scale(),
    target scales, Adam step)            normalise(), adam() (numpy)
Parity status: every function is pinned by CPU tests.  Training is compared with the GPU
through its starting parameters and its first Adam step; longer runs of the GPU training
are judged by what the network buys (its warm start against a zero start).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

PREC_NONE, PREC_JACOBI, PREC_MSRB = 0, 1, 2
WARM_ZERO, WARM_GALERKIN, WARM_GIVEN = 0, 1, 2
CONVERGED, MAX_ITERS, BREAKDOWN = 0, 1, 2

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        i64, i32, d = C.c_int64, C.c_int, C.c_double
        L.orc_block_map.argtypes = [i32] * 6 + [P]
        L.orc_csr_nnz.argtypes = [i32] * 3
        L.orc_csr_nnz.restype = i64
        L.orc_assemble_affine.argtypes = [i32, i32, i32, P, i32, P, P, P]
        L.orc_assemble_ex.argtypes = [i32, i32, i32, P, i32, P, P, P, P, P]
        L.orc_node_weights.argtypes = [i32, i32, i32, P, P]
        L.orc_assemble_field.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P]
        L.orc_dirichlet_lift.argtypes = [i32, i32, i32, i32, P, P, P, P, P]
        L.orc_block_map_ex.argtypes = [i32] * 6 + [P, P]
        L.orc_assemble_mu.argtypes = [i32, i32, i32, P, i32, P, P, P, P]
        L.orc_csr_combine.argtypes = [i64, i32, P, P, P]
        L.orc_csr_matvec.argtypes = [i64, P, P, P, P, P]
        L.orc_cholesky.argtypes = [i32, P]
        L.orc_cholesky_solve.argtypes = [i32, P, P]
        L.orc_rb_solve.argtypes = [i32, i32, i32, P, P, P, P]
        L.orc_pcg.argtypes = [i64, P, P, P, P, P, i32, P, d, i32, i32, P, P, P]
        L.orc_greedy.argtypes = [i64, P, P, P, i32, i64, P, P, i32, i32, d, d, i32, P, P, P, P, P, P]
        L.orc_rb_indicator.argtypes = [i64, P, P, P, i32, i64, P, P, i32, i32, P, P, P]
        L.orc_rb_indicator.restype = d
        L.orc_solve_batch.argtypes = ([i64, P, P, P, i32, i64, P, P, i32, i32, P, i32, i32, P, P, P,
                                       i32, d, i32, i32, P, P, P, P, P, i32])
        L.orc_mlp_param_count.argtypes = [i32, i32, i32]
        L.orc_mlp_param_count.restype = i64
        L.orc_mlp_forward.argtypes = [i32, i32, i32, P, i32, P, P]
        L.orc_mlp_loss_grad.argtypes = [i32, i32, i32, P, i32, P, P, P]
        L.orc_mlp_loss_grad.restype = d
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _MSRB(C.Structure):
    _fields_ = [("N", C.c_int), ("n", C.c_int64), ("W", C.c_void_p), ("chol_AN", C.c_void_p)]


def block_map(grid, blocks, neumann=(0, 0, 0)) -> np.ndarray:
    nx, ny, nz = grid
    m = np.zeros(nx * ny * nz, dtype=np.uint8)
    if any(neumann):
        nm = np.ascontiguousarray(neumann, dtype=np.int32)
        lib().orc_block_map_ex(nx, ny, nz, blocks[0], blocks[1], blocks[2], _p(nm), _p(m))
    else:
        lib().orc_block_map(nx, ny, nz, blocks[0], blocks[1], blocks[2], _p(m))
    return m


def node_weights(grid, neumann=(0, 0, 0)) -> np.ndarray:
    """Relative control volume of each node (the source weight in the right-hand side)."""
    nx, ny, nz = grid
    w = np.zeros(nx * ny * nz)
    nm = np.ascontiguousarray(neumann, dtype=np.int32)
    lib().orc_node_weights(nx, ny, nz, _p(nm), _p(w))
    return w


@dataclasses.dataclass
class Operator:
    """Explicit CSR of the Q affine terms A_q on one grid (shared pattern)."""
    grid: tuple
    Q: int
    row_ptr: np.ndarray
    col: np.ndarray
    vals_q: np.ndarray  # [Q][nnz]

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def values(self, mu) -> np.ndarray:
        """CSR values of A(mu) = sum_q mu_q A_q."""
        mu = _f64(mu)
        out = np.empty(self.nnz)
        lib().orc_csr_combine(self.nnz, self.Q, _p(self.vals_q), _p(mu), _p(out))
        return out

    def matvec(self, mu, x) -> np.ndarray:
        x = _f64(x)
        val = self.values(mu)
        y = np.empty(self.n)
        lib().orc_csr_matvec(self.n, _p(self.row_ptr), _p(self.col), _p(val), _p(x), _p(y))
        return y

    def matvec_values(self, val, x) -> np.ndarray:
        x = _f64(x)
        y = np.empty(self.n)
        lib().orc_csr_matvec(self.n, _p(self.row_ptr), _p(self.col), _p(_f64(val)), _p(x), _p(y))
        return y

    def dense(self, mu) -> np.ndarray:
        """Dense A(mu) (small grids only)."""
        A = np.zeros((self.n, self.n))
        val = self.values(mu)
        for r in range(self.n):
            for e in range(self.row_ptr[r], self.row_ptr[r + 1]):
                A[r, self.col[e]] = val[e]
        return A


def assemble(grid, blocks=None, submap=None, Q=None, kscale=(1.0, 1.0, 1.0), neumann=(0, 0, 0)) -> Operator:
    """Affine terms A_q; kscale: diffusion tensor diagonal; neumann: per axis, 1 for a homogeneous
    Neumann face at coordinate 1 (orc_assemble_ex)."""
    nx, ny, nz = grid
    if submap is None:
        submap = block_map(grid, blocks, neumann)
        Q = blocks[0] * blocks[1] * blocks[2]
    submap = np.ascontiguousarray(submap, dtype=np.uint8)
    L = lib()
    nnz = L.orc_csr_nnz(nx, ny, nz)
    n = nx * ny * nz
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    vals = np.zeros((Q, nnz))
    if tuple(kscale) == (1.0, 1.0, 1.0) and not any(neumann):
        rc = L.orc_assemble_affine(nx, ny, nz, _p(submap), Q, _p(row_ptr), _p(col), _p(vals))
    else:
        ks = np.ascontiguousarray(kscale, dtype=np.float64)
        nm = np.ascontiguousarray(neumann, dtype=np.int32)
        rc = L.orc_assemble_ex(nx, ny, nz, _p(submap), Q, _p(ks), _p(nm), _p(row_ptr), _p(col), _p(vals))
    if rc != 0:
        raise ValueError("orc_assemble_affine failed: %d" % rc)
    return Operator(tuple(grid), Q, row_ptr, col, vals)


def _faces(grid, kfx, kfy, kfz):
    nx, ny, nz = grid
    kfx = np.ascontiguousarray(kfx, dtype=np.float64)
    Q = kfx.shape[0]
    kfx = kfx.reshape(Q, nz, ny, nx + 1)
    kfy = np.ascontiguousarray(kfy, dtype=np.float64).reshape(Q, nz, ny + 1, nx)
    kfz = np.ascontiguousarray(kfz, dtype=np.float64).reshape(Q, nz + 1, ny, nx)
    return Q, kfx, kfy, kfz


def assemble_field(grid, kfx, kfy, kfz) -> Operator:
    """Affine terms A_q of an operator whose coefficient kappa_q is given at the cell faces
    (orc_assemble_field): kfx [Q][nz][ny][nx+1], kfy [Q][nz][ny+1][nx], kfz [Q][nz+1][ny][nx];
    Dirichlet data on the whole boundary.  The paper's Example 1 (Sec. 4) has Q = 2: kappa_0 = 1
    and kappa_1 = g(x), A(mu) = A_0 + mu_1 A_1."""
    nx, ny, nz = grid
    Q, kfx, kfy, kfz = _faces(grid, kfx, kfy, kfz)
    L = lib()
    nnz = L.orc_csr_nnz(nx, ny, nz)
    n = nx * ny * nz
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    vals = np.zeros((Q, nnz))
    rc = L.orc_assemble_field(nx, ny, nz, Q, _p(kfx), _p(kfy), _p(kfz), _p(row_ptr), _p(col), _p(vals))
    if rc != 0:
        raise ValueError("orc_assemble_field failed: %d" % rc)
    return Operator(tuple(grid), Q, row_ptr, col, vals)


def boundary_size(grid) -> int:
    """Values of Dirichlet data on the six boundary planes (the layout of orc_dirichlet_lift)."""
    nx, ny, nz = grid
    return 2 * (nz * ny + nz * nx + ny * nx)


def dirichlet_lift(grid, kfx, kfy, kfz, gb) -> np.ndarray:
    """lift [Q][n]: what Dirichlet data gb (six boundary planes, orc_dirichlet_lift's layout)
    adds to the right-hand side through each term A_q."""
    nx, ny, nz = grid
    Q, kfx, kfy, kfz = _faces(grid, kfx, kfy, kfz)
    gb = np.ascontiguousarray(gb, dtype=np.float64)
    if gb.shape != (boundary_size(grid),):
        raise ValueError("gb must have %d values" % boundary_size(grid))
    out = np.zeros((Q, nx * ny * nz))
    lib().orc_dirichlet_lift(nx, ny, nz, Q, _p(kfx), _p(kfy), _p(kfz), _p(gb), _p(out))
    return out


def assemble_mu(grid, mu, blocks=None, submap=None, Q=None, kscale=(1.0, 1.0, 1.0), neumann=(0, 0, 0)) -> Operator:
    """A(mu) for one parameter, assembled directly (orc_assemble_mu), as a one-term operator:
    its matvec and mg.Hierarchy take the coefficient [1.0].  Holds one value array instead of
    Q, for grids where Q arrays of the affine terms do not fit in memory.  With an anisotropy
    or a Neumann face: the affine terms of assemble(), combined."""
    if tuple(kscale) != (1.0, 1.0, 1.0) or any(neumann):
        op = assemble(grid, blocks=blocks, submap=submap, Q=Q, kscale=kscale, neumann=neumann)
        return Operator(tuple(grid), 1, op.row_ptr, op.col, op.values(mu)[None, :])
    nx, ny, nz = grid
    if submap is None:
        submap = block_map(grid, blocks)
        Q = blocks[0] * blocks[1] * blocks[2]
    submap = np.ascontiguousarray(submap, dtype=np.uint8)
    mu = _f64(mu)
    if mu.shape != (Q,):
        raise ValueError("mu must have Q = %d entries" % Q)
    L = lib()
    nnz = L.orc_csr_nnz(nx, ny, nz)
    n = nx * ny * nz
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    vals = np.zeros((1, nnz))
    rc = L.orc_assemble_mu(nx, ny, nz, _p(submap), Q, _p(mu), _p(row_ptr), _p(col), _p(vals))
    if rc != 0:
        raise ValueError("orc_assemble_mu failed: %d" % rc)
    return Operator(tuple(grid), 1, row_ptr, col, vals)


def cholesky(a) -> np.ndarray:
    a = np.array(a, dtype=np.float64, order="C")
    if lib().orc_cholesky(a.shape[0], _p(a)) != 0:
        raise np.linalg.LinAlgError("not positive definite")
    return a


def cholesky_solve(l, b) -> np.ndarray:
    b = np.array(b, dtype=np.float64)
    lib().orc_cholesky_solve(l.shape[0], _p(_f64(l)), _p(b))
    return b


def rb_solve(ANq, fN, mu, N=None) -> np.ndarray:
    ANq = _f64(ANq)
    Q, Nmax, _ = ANq.shape
    N = Nmax if N is None else N
    c = np.empty(N)
    rc = lib().orc_rb_solve(N, Nmax, Q, _p(ANq), _p(_f64(fN)), _p(_f64(mu)), _p(c))
    if rc != 0:
        raise np.linalg.LinAlgError("reduced matrix not positive definite")
    return c


@dataclasses.dataclass
class PCGResult:
    u: np.ndarray
    iters: int
    relres: float
    status: int
    hist: np.ndarray


def pcg(op: Operator, mu, f=None, u0=None, precond=PREC_JACOBI, tol=1e-10, max_iters=10000,
        max_restarts=3, msrb=None) -> PCGResult:
    """Algorithm 1 (with the true-residual restart of Algorithm 4).

    msrb: (W [N][n], chol(A_N(mu)) [N][N]) for the MSRB preconditioner."""
    n = op.n
    f = np.ones(n) if f is None else _f64(f)
    u = np.zeros(n) if u0 is None else np.array(u0, dtype=np.float64)
    val = op.values(mu)
    it, rel = C.c_int(0), C.c_double(0)
    hist = np.full(max_iters + 1, np.nan)
    ms = None
    keep = None
    if precond == PREC_MSRB:
        W, L = _f64(msrb[0]), _f64(msrb[1])
        keep = (W, L)
        ms = _MSRB(L.shape[0], n, W.ctypes.data, L.ctypes.data)
    st = lib().orc_pcg(n, _p(op.row_ptr), _p(op.col), _p(val), _p(f), _p(u), precond,
                       C.byref(ms) if ms is not None else None, tol, max_iters, max_restarts,
                       C.byref(it), C.byref(rel), _p(hist))
    del keep
    return PCGResult(u, it.value, rel.value, st, hist[: it.value + 1])


@dataclasses.dataclass
class Basis:
    W: np.ndarray        # [N][n]
    ANq: np.ndarray      # [Q][N][N]
    fN: np.ndarray       # [N]
    selected: np.ndarray
    eta_hist: np.ndarray
    N: int


def greedy(op: Operator, mu_train, n_max, f=None, greedy_tol=0.0, snapshot_tol=1e-12, indicator=0) -> Basis:
    """Greedy reduced basis (Algorithm 5 skeleton, Galerkin RB).  indicator 0: FOM residual;
    1: L1 norm of the coefficients w.r.t. the unorthogonalised snapshots (Sec. 3.1)."""
    n = op.n
    f = np.ones(n) if f is None else _f64(f)
    mu_train = _f64(mu_train)
    n_train = mu_train.shape[0]
    W = np.zeros((n_max, n))
    ANq = np.zeros((op.Q, n_max, n_max))
    fN = np.zeros(n_max)
    sel = np.full(n_max, -1, dtype=np.int32)
    eta = np.full(n_max, np.nan)
    nout = C.c_int(0)
    rc = lib().orc_greedy(n, _p(op.row_ptr), _p(op.col), _p(op.vals_q), op.Q, op.nnz, _p(f),
                          _p(mu_train), n_train, n_max, greedy_tol, snapshot_tol, indicator, _p(W), _p(ANq),
                          _p(fN), _p(sel), _p(eta), C.byref(nout))
    if rc != 0:
        raise RuntimeError("orc_greedy failed: %d" % rc)
    N = nout.value
    return Basis(W[:N].copy(), np.ascontiguousarray(ANq[:, :N, :N]), fN[:N].copy(), sel[:N].copy(),
                 eta[:N].copy(), N)


def rb_indicator(op: Operator, basis: Basis, mu, f=None, n_use=None) -> float:
    """||f - A(mu) W_n c_n|| / ||f|| of the Galerkin RB solution (Sec. 2.3) with the first n_use
    basis vectors (default: all); the reduced system is the leading n_use block (nested spaces)."""
    n = op.n
    f = np.ones(n) if f is None else _f64(f)
    k = basis.N if n_use is None else int(n_use)
    if not 1 <= k <= basis.N:
        raise ValueError("n_use must be in 1..N")
    return lib().orc_rb_indicator(n, _p(op.row_ptr), _p(op.col), _p(op.vals_q), op.Q, op.nnz, _p(f),
                                  _p(_f64(basis.W)), k, basis.N, _p(_f64(basis.ANq)),
                                  _p(_f64(basis.fN)), _p(_f64(mu)))


@dataclasses.dataclass
class BatchResult:
    u: np.ndarray        # [B][n]
    iters: np.ndarray
    relres: np.ndarray
    relres0: np.ndarray
    status: np.ndarray
    threads: int


def solve_batch(op: Operator, mu, warm=WARM_ZERO, basis: Basis | None = None, c_given=None,
                precond=PREC_JACOBI, tol=1e-10, max_iters=20000, max_restarts=3, f=None,
                n_threads=0) -> BatchResult:
    """Algorithm 4 for each parameter of a batch (OpenMP over instances)."""
    n = op.n
    f = np.ones(n) if f is None else _f64(f)
    mu = _f64(np.atleast_2d(mu))
    B = mu.shape[0]
    u = np.zeros((B, n))
    it = np.zeros(B, dtype=np.int32)
    rel = np.zeros(B)
    rel0 = np.zeros(B)
    st = np.zeros(B, dtype=np.int32)
    if basis is not None:
        W, ANq, fN, N = _f64(basis.W), _f64(basis.ANq), _f64(basis.fN), basis.N
    else:
        W = ANq = fN = None
        N = 0
    cg = None if c_given is None else _f64(c_given)
    used = lib().orc_solve_batch(n, _p(op.row_ptr), _p(op.col), _p(op.vals_q), op.Q, op.nnz, _p(f),
                                 _p(mu), B, warm, _p(cg), N, N, _p(W), _p(ANq), _p(fN), precond,
                                 tol, max_iters, max_restarts, _p(u), _p(it), _p(rel), _p(rel0),
                                 _p(st), n_threads)
    if used < 0:
        raise RuntimeError("orc_solve_batch failed: %d" % used)
    return BatchResult(u, it, rel, rel0, st, used)


def mlp_param_count(p, H, N) -> int:
    return int(lib().orc_mlp_param_count(p, H, N))


def mlp_forward(p, H, N, params, x) -> np.ndarray:
    x = _f64(np.atleast_2d(x))
    y = np.empty((x.shape[0], N))
    lib().orc_mlp_forward(p, H, N, _p(_f64(params)), x.shape[0], _p(x), _p(y))
    return y


def mlp_loss_grad(p, H, N, params, x, t):
    x = _f64(np.atleast_2d(x))
    g = np.empty(mlp_param_count(p, H, N))
    loss = lib().orc_mlp_loss_grad(p, H, N, _p(_f64(params)), x.shape[0], _p(x), _p(_f64(t)), _p(g))
    return loss, g


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
