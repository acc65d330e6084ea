"""Counter-based random numbers and the adaptive step-size rule of the HMC sampler.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests use it to replay the
draws and the step-size updates the CUDA library makes on the device.

- Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as
  1, 2, 3", SC 2011): a 128-bit counter and a 64-bit key go through ten rounds, each
  multiplying words 0 and 2 of the counter by two fixed 32-bit constants and mixing the
  high and low halves of the products with words 1 and 3 and the key; the key is bumped
  by two Weyl constants between rounds.
- Uniforms and normals from its output words, as the library defines them: 24-bit
  uniforms u = (w >> 8 + 1/2) 2^-24 in (0, 1) paired by the Box-Muller transform
  (Box and Muller 1958) into normals, and the accept uniform (w + 1/2) 2^-32.
- The step-size rule of App. B (adaptive step size): after a trajectory with acceptance
  probability a = min(1, exp(H0 - H1)), eps <- eps / 1.2 if a < a_min, else
  eps <- min(eps0, 1.2 eps).

Counter layout of the library's draws: (element group i // 4, iteration low word,
iteration high word, stream), key = (seed low word, seed high word); stream 0 gives the
momentum normals, stream 1 the accept uniform (output word 0 of element group 0)."""
from __future__ import annotations

import math

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57          # round multipliers
W0, W1 = 0x9E3779B9, 0xBB67AE85          # key increments (Weyl sequence)
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds on integer arrays: ctr = (c0, c1, c2, c3), key = (k0, k1),
    each an array (or scalar) of uint32 values; returns the four output words (uint64 arrays
    holding 32-bit values)."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK for v in ctr)
    k0, k1 = (np.asarray(v, dtype=np.uint64) & MASK for v in key)
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = c0 * np.uint64(M0)          # < 2^64: exact in uint64
        p1 = c2 * np.uint64(M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _key(seed: int):
    return seed & MASK, (seed >> 32) & MASK


def normals(seed: int, iteration: int, n: int) -> np.ndarray:
    """The momentum draw of one iteration: n standard normals (FP64 here)."""
    g = np.arange((n + 3) // 4, dtype=np.uint64)
    it_lo, it_hi = iteration & MASK, (iteration >> 32) & MASK
    w = philox4x32_10((g, it_lo, it_hi, 0), _key(seed))
    u = [((wk >> np.uint64(8)).astype(np.float64) + 0.5) * 2.0 ** -24 for wk in w]
    out = np.empty((g.size, 4))
    for a, b, j in ((0, 1, 0), (2, 3, 2)):
        r = np.sqrt(-2.0 * np.log(u[a]))
        out[:, j] = r * np.cos(2.0 * math.pi * u[b])
        out[:, j + 1] = r * np.sin(2.0 * math.pi * u[b])
    return out.reshape(-1)[:n]


def uniforms24(seed: int, iteration: int, n: int) -> np.ndarray:
    """The 24-bit uniforms behind normals(), in element order (4 per counter)."""
    g = np.arange((n + 3) // 4, dtype=np.uint64)
    w = philox4x32_10((g, iteration & MASK, (iteration >> 32) & MASK, 0), _key(seed))
    u = np.stack([((wk >> np.uint64(8)).astype(np.float64) + 0.5) * 2.0 ** -24 for wk in w], axis=1)
    return u.reshape(-1)[:n]


def accept_uniform(seed: int, iteration: int) -> float:
    w = philox4x32_10((0, iteration & MASK, (iteration >> 32) & MASK, 1), _key(seed))
    return (float(w[0]) + 0.5) * 2.0 ** -32


def acceptance_probability(h0: float, h1: float) -> float:
    """min(1, exp(H0 - H1)); 0 when either energy is not finite (the trajectory is rejected)."""
    if not (math.isfinite(h0) and math.isfinite(h1)):
        return 0.0
    return 1.0 if h1 <= h0 else math.exp(h0 - h1)


def adapt_step(eps: float, eps0: float, a: float, a_min: float) -> float:
    """Step-size update after one trajectory (App. B): shrink by 1.2 below the threshold,
    otherwise grow by 1.2 up to the initial step."""
    if a < a_min:
        return eps / 1.2
    return min(eps0, 1.2 * eps)
