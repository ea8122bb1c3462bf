"""Oracle of the learned warm start's training set-up: the initial parameters, the
coefficient scales, the input map and one Adam step (numpy, FP64 where the library
computes in FP32).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product.

- splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
  OOPSLA 2014): the state advances by the golden-ratio increment 0x9E3779B97F4A7C15, and
  each output is the state passed through the variant-13 mix (shifts 30, 27, 31 and the
  two odd multipliers).
- The draw of the network's starting parameters, the target scales and the input map
  follow the conventions the library's header states for its training entry point.
- Adam: Kingma & Ba, "Adam: A method for stochastic optimization", ICLR 2015,
  Algorithm 1 (bias-corrected first and second moments).
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(state: int, count: int) -> list[int]:
    """The first `count` outputs of splitmix64 started from `state` (Python integers)."""
    out = []
    for _ in range(count):
        state = (state + _GAMMA) & _MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out.append(z ^ (z >> 31))
    return out


def _splitmix64_at(seed: int, index: np.ndarray) -> np.ndarray:
    """Output number index + 1 of splitmix64 from state `seed`, for an array of indices
    (the state after k steps is seed + k * gamma, so each output is formed directly)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + np.uint64(_GAMMA) * (index.astype(np.uint64) + np.uint64(1))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def layer_segments(p: int, H: int, N: int) -> list[tuple[str, int, int, int]]:
    """(name, first index, end index, fan_in) of W1 b1 W2 b2 W3 b3 W4 b4 in the parameter
    vector: W_l row-major [out][in], each followed by its bias."""
    segs, off = [], 0
    for l, (fin, fout) in enumerate([(p, H), (H, H), (H, H), (H, N)], start=1):
        segs.append(("W%d" % l, off, off + fin * fout, fin))
        off += fin * fout
        segs.append(("b%d" % l, off, off + fout, fin))
        off += fout
    return segs


def init_params(p: int, H: int, N: int, seed: int) -> np.ndarray:
    """Starting parameters (FP32): parameter i takes output i + 1 of splitmix64 from `seed`,
    u = (z >> 11) 2^-53 in [0, 1), value (2u - 1) b rounded to FP32, b = 1/sqrt(fan_in)
    rounded to FP32."""
    segs = layer_segments(p, H, N)
    P = segs[-1][2]
    z = _splitmix64_at(seed, np.arange(P, dtype=np.int64))
    u = (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    out = np.empty(P, dtype=np.float32)
    for _, a, e, fan_in in segs:
        b = float(np.float32(1.0 / np.sqrt(float(fan_in))))
        out[a:e] = ((2.0 * u[a:e] - 1.0) * b).astype(np.float32)
    return out


def rms_scale(C: np.ndarray) -> np.ndarray:
    """scale_j = sqrt(mean over the rows of C[:, j]^2), 1 where that is 0, as FP32."""
    C = np.asarray(C, dtype=np.float64)
    r = np.sqrt(np.mean(C * C, axis=0))
    return np.where(r > 0.0, r, 1.0).astype(np.float32)


def normalise(mu: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """The network's inputs: 2 (log mu - log lo) / (log hi - log lo) - 1."""
    return 2.0 * (np.log(mu) - np.log(lo)) / (np.log(hi) - np.log(lo)) - 1.0


def adam(theta, m, v, g, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """Step t (1-based) of Adam on parameters theta with gradient g: returns the new
    (theta, m, v), all FP64."""
    m = b1 * np.asarray(m, dtype=np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, dtype=np.float64) + (1.0 - b2) * g * g
    m_hat = m / (1.0 - b1 ** t)
    v_hat = v / (1.0 - b2 ** t)
    return np.asarray(theta, dtype=np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
