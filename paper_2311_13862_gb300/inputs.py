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
