"""Counter-based probe generator of the oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import anything under ``oracle/``; the product path
never does.

The paper draws i.i.d. Gaussian probe vectors (Lemma thm:trace, Algorithms
1a and 1b) and a uniform {+1,-1} start vector for the power method
(Algorithm alg:power) without naming a generator.  Both sides of the
parity tests therefore implement, each in its own code, SplitMix64 as
published by Steele, Lea and Flood ("Fast splittable pseudorandom number
generators", OOPSLA 2014):

    state_c = seed + (c + 1) * 0x9E3779B97F4A7C15          (mod 2^64)
    z = (state_c ^ (state_c >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    out(seed, c) = z ^ (z >> 31)

so ``out(seed, c)`` is the (c+1)-th output of a SplitMix64 stream started
at ``seed``.  Entry (i, j) of an n x s probe block (row i, probe j) has
the linear counter e = j*n + i:

* Rademacher: +1 if the top bit of out(seed, e) is 0, else -1.
* Gaussian: a = out(seed, 2e), b = out(seed, 2e+1),
  u1 = ((a >> 11) + 1) / 2^53 in (0, 1], u2 = (b >> 11) / 2^53 in [0, 1),
  g = sqrt(-2 ln u1) * cos(2 pi u2)   (Box and Muller, 1958).

The power method's start vectors are Rademacher blocks drawn from the
seed ``seed ^ 0x5851F42D4C957F2D``.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)
POWER_SEED_XOR = 0x5851F42D4C957F2D


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """out(seed, c) for every counter c (uint64 array, wrapping arithmetic)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GAMMA
        z = (state ^ (state >> np.uint64(30))) * MIX1
        z = (z ^ (z >> np.uint64(27))) * MIX2
    return z ^ (z >> np.uint64(31))


def _linear_counters(n: int, s: int) -> np.ndarray:
    i = np.arange(n, dtype=np.uint64)[:, None]
    j = np.arange(s, dtype=np.uint64)[None, :]
    return j * np.uint64(n) + i  # (n, s), e = j*n + i


def rademacher(n: int, s: int, seed: int) -> np.ndarray:
    """n x s block of +-1 (FP64)."""
    top = splitmix64(seed, _linear_counters(n, s)) >> np.uint64(63)
    return np.where(top == 0, 1.0, -1.0)


def gaussian(n: int, s: int, seed: int) -> np.ndarray:
    """n x s block of N(0, 1) draws (FP64), Box-Muller from two 53-bit uniforms."""
    e = _linear_counters(n, s)
    a = splitmix64(seed, np.uint64(2) * e)
    b = splitmix64(seed, np.uint64(2) * e + np.uint64(1))
    u1 = ((a >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (b >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def probes(n: int, s: int, seed: int, kind: str) -> np.ndarray:
    """The probe block G of Algorithms 1a/1b (n x s, FP64)."""
    if kind == "rademacher":
        return rademacher(n, s, seed)
    if kind == "gaussian":
        return gaussian(n, s, seed)
    raise ValueError(f"unknown probe kind {kind!r}")


def power_start(n: int, q: int, seed: int) -> np.ndarray:
    """The q start vectors x_0^j in {+1,-1}^n of Algorithm alg:power (n x q)."""
    return rademacher(n, q, seed ^ POWER_SEED_XOR)
