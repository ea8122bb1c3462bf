"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle.

This module holds workload descriptions and random parameter draws only; none
of the method's arithmetic lives here.  Parameters are log-uniform,
mu = exp(U(log lo, log hi)), drawn with numpy's default generator from a
fixed seed, shape [n][Q].  Seeds: training set 1000+c, test set 2000+c,
surrogate data 3000+c for workload c (1..5).

Workloads (the diffusion model -div(kappa grad u) = 1 on the unit cube with
zero Dirichlet data, kappa piecewise constant on block subdomains, 7-point
finite differences on an interior grid, h = 1/(n+1)):

  1  16^3,  2 half-cubes split in x,     mu in [0.1, 10]^2,   N <= 10, 64 train, 8 test, tol 1e-12
  2  64^3,  2x2x1 blocks,                mu in [0.1, 10]^4,   N <= 20, 256 train, 256 test, tol 1e-10
  3  128^3, 2x2x2 octants,               mu in [0.01, 100]^8, N <= 40, 256 train, 64 test, tol 1e-10
  4  workload 2 with a learned warm start (4096 surrogate samples)
  5  3x3x3 blocks, mu in [0.1, 10]^27, grids 96^3 / 128^3 / 256^3, N <= 60, 96 requests

The paper's Example 1 (Sec. 4) is problem data here too: its coefficient field, boundary
data and source sampled on the grid (example1_*), with mu uniform on [0, 2] x [0, 1].
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    grid: tuple[int, int, int]      # interior nodes (nx, ny, nz)
    blocks: tuple[int, int, int]    # (bx, by, bz); Q = bx*by*bz
    mu_lo: float
    mu_hi: float
    n_max: int                      # maximum reduced basis dimension
    n_train: int
    n_test: int
    tol: float                      # relative residual target of the online solve
    seed_base: int

    @property
    def Q(self) -> int:
        return self.blocks[0] * self.blocks[1] * self.blocks[2]

    @property
    def n_dof(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2]


WORKLOADS = {
    "c1": Workload("c1-16cube-2halves", (16, 16, 16), (2, 1, 1), 0.1, 10.0, 10, 64, 8, 1e-12, 1),
    "c2": Workload("c2-64cube-2x2x1", (64, 64, 64), (2, 2, 1), 0.1, 10.0, 20, 256, 256, 1e-10, 2),
    "c3": Workload("c3-128cube-octants", (128, 128, 128), (2, 2, 2), 0.01, 100.0, 40, 256, 64, 1e-10, 3),
    "c4": Workload("c4-64cube-2x2x1-learned", (64, 64, 64), (2, 2, 1), 0.1, 10.0, 20, 256, 256, 1e-10, 4),
    "c5-96": Workload("c5-96cube-3x3x3", (96, 96, 96), (3, 3, 3), 0.1, 10.0, 60, 256, 32, 1e-10, 5),
    "c5-128": Workload("c5-128cube-3x3x3", (128, 128, 128), (3, 3, 3), 0.1, 10.0, 60, 256, 32, 1e-10, 5),
    "c5-256": Workload("c5-256cube-3x3x3", (256, 256, 256), (3, 3, 3), 0.1, 10.0, 60, 256, 32, 1e-10, 5),
    # a second workload with a non-affine source: the c2 operator, and per parameter a Gaussian
    # source with its own centre (gauss_params), RB N <= 40 over 256 training parameters
    "c2g": Workload("c2g-64cube-2x2x1-gaussian-source", (64, 64, 64), (2, 2, 1), 0.1, 10.0, 40, 256, 256,
                    1e-10, 6),
}


def log_uniform(seed: int, n: int, Q: int, lo: float, hi: float) -> np.ndarray:
    """n parameter vectors of length Q, log-uniform on [lo, hi]^Q, float64."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=(n, Q)))


def train_mu(w: Workload, n: int | None = None) -> np.ndarray:
    return log_uniform(1000 + w.seed_base, w.n_train if n is None else n, w.Q, w.mu_lo, w.mu_hi)


def test_mu(w: Workload, n: int | None = None) -> np.ndarray:
    return log_uniform(2000 + w.seed_base, w.n_test if n is None else n, w.Q, w.mu_lo, w.mu_hi)


def surrogate_mu(w: Workload, n: int = 4096) -> np.ndarray:
    return log_uniform(3000 + w.seed_base, n, w.Q, w.mu_lo, w.mu_hi)


def gauss_params(seed: int, n: int, lo: float = 0.25, hi: float = 0.75, sigma: float = 0.1) -> np.ndarray:
    """n Gaussian-source parameter rows (c_x, c_y, c_z, sigma): centres uniform in [lo, hi]^3."""
    rng = np.random.default_rng(seed)
    return np.column_stack([rng.uniform(lo, hi, size=(n, 3)), np.full(n, sigma)])


def train_sources(w: Workload, n: int | None = None) -> np.ndarray:
    return gauss_params(4000 + w.seed_base, w.n_train if n is None else n)


def test_sources(w: Workload, n: int | None = None) -> np.ndarray:
    return gauss_params(5000 + w.seed_base, w.n_test if n is None else n)


def random_field(seed: int, shape) -> np.ndarray:
    """Standard-normal float64 array (test vectors for operator checks)."""
    return np.random.default_rng(seed).standard_normal(shape)


def inclusion_map(grid, seed: int) -> np.ndarray:
    """Subdomain map [nz][ny][nx] (uint8, Q = 3) with the structure of a layered medium
    holding one inclusion: two layers split at a seeded z plane (ids 0 and 1) and a
    seeded box (id 2) that crosses the layer interface."""
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    m[int(rng.integers(1, nz)):, :, :] = 1
    lo = [int(rng.integers(0, max(1, n // 2))) for n in (nz, ny, nx)]
    hi = [l + int(rng.integers(1, max(2, n - l))) for l, n in zip(lo, (nz, ny, nx))]
    m[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = 2
    return m


def small(grid=(9, 7, 5), blocks=(2, 1, 1), lo=0.1, hi=10.0, n_max=6, n_train=16, n_test=4,
          tol=1e-12, seed_base=11, name="small") -> Workload:
    """A tiny ragged workload for fast CPU and parity tests."""
    return Workload(name, tuple(grid), tuple(blocks), lo, hi, n_max, n_train, n_test, tol, seed_base)


# ---------------------------------------------------------------------------
# The paper's Example 1 (Sec. 4): -div(kappa grad u) = f on the unit cube with
# kappa = 1 + mu_1 g(x), g = sin^2(20 pi (4 (x-1/2)^2 + (y-1/2)^2 + (z-1/2)^2)),
# f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z), and Dirichlet data
# g_D = (1 - mu_2) cos(10 pi (4 (x-1/2)^2 + (y-1/2)^2 + (z-1/2)^2)) + mu_2 cos(10 pi (x+y+z)),
# mu in [0, 2] x [0, 1].  Sampled on an interior grid with h = 1/(n+1) per axis, node i
# (0-based) at (i+1) h.  Coefficients are taken at the cell faces (face f of an axis at
# (f + 1/2) h, f = 0..n); boundary data at the boundary points across each boundary face.
# ---------------------------------------------------------------------------
def _example1_g(x, y, z):
    return np.sin(20.0 * np.pi * (4.0 * (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)) ** 2


def _axis_nodes(n):
    return np.arange(1, n + 1) / (n + 1)


def _axis_faces(n):
    return (np.arange(0, n + 1) + 0.5) / (n + 1)


def example1_faces(grid):
    """(kfx [2][nz][ny][nx+1], kfy [2][nz][ny+1][nx], kfz [2][nz+1][ny][nx]): the two affine
    terms of Example 1's coefficient at the cell faces, kappa_0 = 1 and kappa_1 = g."""
    nx, ny, nz = grid
    xn, yn, zn = _axis_nodes(nx), _axis_nodes(ny), _axis_nodes(nz)
    xf, yf, zf = _axis_faces(nx), _axis_faces(ny), _axis_faces(nz)
    out = []
    for xs, ys, zs in ((xf, yn, zn), (xn, yf, zn), (xn, yn, zf)):
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        out.append(np.stack([np.ones_like(X), _example1_g(X, Y, Z)]))
    return tuple(out)


def boundary_points(grid):
    """Coordinates (X, Y, Z) of the boundary points facing the interior nodes, in the layout of
    the six boundary planes: x = 0, x = 1 ([nz][ny] each), y = 0, y = 1 ([nz][nx]), z = 0,
    z = 1 ([ny][nx])."""
    nx, ny, nz = grid
    xn, yn, zn = _axis_nodes(nx), _axis_nodes(ny), _axis_nodes(nz)
    pts = []
    for c in (0.0, 1.0):
        Z, Y = np.meshgrid(zn, yn, indexing="ij")
        pts.append((np.full_like(Y, c), Y, Z))
    for c in (0.0, 1.0):
        Z, X = np.meshgrid(zn, xn, indexing="ij")
        pts.append((X, np.full_like(X, c), Z))
    for c in (0.0, 1.0):
        Y, X = np.meshgrid(yn, xn, indexing="ij")
        pts.append((X, Y, np.full_like(X, c)))
    return tuple(np.concatenate([p[a].ravel() for p in pts]) for a in range(3))


def example1_boundary(grid):
    """(G1, G2): the two affine parts of Example 1's Dirichlet data on the boundary planes,
    g_D(mu) = (1 - mu_2) G1 + mu_2 G2."""
    X, Y, Z = boundary_points(grid)
    G1 = np.cos(10.0 * np.pi * (4.0 * (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2))
    G2 = np.cos(10.0 * np.pi * (X + Y + Z))
    return G1, G2


def example1_source(grid):
    """f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) at the interior nodes, [z][y][x] order."""
    nx, ny, nz = grid
    Z, Y, X = np.meshgrid(_axis_nodes(nz), _axis_nodes(ny), _axis_nodes(nx), indexing="ij")
    return (3.0 * np.pi ** 2 * np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)).ravel()


def example1_mu(seed: int, n: int) -> np.ndarray:
    """n parameters (mu_1, mu_2) uniform on [0, 2] x [0, 1]."""
    rng = np.random.default_rng(seed)
    return np.column_stack([rng.uniform(0.0, 2.0, n), rng.uniform(0.0, 1.0, n)])
