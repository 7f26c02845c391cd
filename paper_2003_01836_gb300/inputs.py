"""Seeded synthetic particle systems shared by the oracle tests, the GPU tests and the bench.

This module holds no treecode arithmetic: only the counter-based SplitMix64 generator
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) and
the two particle distributions the workloads use.

* Uniform cube: x, y, z, q each ``2u - 1`` with ``u`` in [0, 1), the paper's test systems
  (Sec. IV: particles uniform in [-1, 1]^3, charges uniform in [-1, 1]).
* Truncated Plummer sphere (Aarseth, Henon and Wielen 1974) with scale radius a = 1, cut at
  r = 10: radius by the inverse of the enclosed-mass fraction M(r) = r^3 / (1 + r^2)^(3/2),
  ``r = a / sqrt(U^(-2/3) - 1)`` with ``U = u * M(10)`` (no rejection needed), direction
  uniform on the sphere, charge ``2u - 1``.

Draw k of a stream with seed s is ``mix(s + (k + 1) * 0x9E3779B97F4A7C15)``; particle i of
a system takes draws 4i, 4i+1, 4i+2, 4i+3 in the order stated above.  A double is
``(u64 >> 11) * 2^-53``.  Everything is FP64 on the host.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
SEED_BASE = 20031836
_CHUNK = 1 << 22


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream with ``seed`` (uint64)."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from draws ``start .. start+count-1``: (u64 >> 11) * 2^-53."""
    return (splitmix64(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _draws(seed: int, n: int):
    """Yields (first particle, (m, 4) array of uniforms) chunks for n particles."""
    for p0 in range(0, n, _CHUNK):
        m = min(_CHUNK, n - p0)
        yield p0, uniform01(seed, 4 * p0, 4 * m).reshape(m, 4)


def uniform_cube(n: int, seed: int):
    """Particles uniform in [-1, 1]^3 with charges uniform in [-1, 1] (Sec. IV)."""
    x, y, z, q = (np.empty(n) for _ in range(4))
    for p0, u in _draws(seed, n):
        s = slice(p0, p0 + u.shape[0])
        x[s] = 2.0 * u[:, 0] - 1.0
        y[s] = 2.0 * u[:, 1] - 1.0
        z[s] = 2.0 * u[:, 2] - 1.0
        q[s] = 2.0 * u[:, 3] - 1.0
    return x, y, z, q


PLUMMER_RMAX = 10.0
PLUMMER_MASS_AT_RMAX = PLUMMER_RMAX ** 3 / (1.0 + PLUMMER_RMAX ** 2) ** 1.5


def plummer(n: int, seed: int, a: float = 1.0):
    """Truncated Plummer sphere, scale radius ``a``, cut at r = 10a, charges uniform."""
    x, y, z, q = (np.empty(n) for _ in range(4))
    for p0, u in _draws(seed, n):
        s = slice(p0, p0 + u.shape[0])
        U = u[:, 0] * PLUMMER_MASS_AT_RMAX
        with np.errstate(divide="ignore"):
            inv = np.where(U > 0.0, U ** (-2.0 / 3.0) - 1.0, np.inf)
        r = a / np.sqrt(inv)
        cz = 2.0 * u[:, 1] - 1.0
        sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
        ph = 2.0 * np.pi * u[:, 2]
        x[s] = r * sz * np.cos(ph)
        y[s] = r * sz * np.sin(ph)
        z[s] = r * cz
        q[s] = 2.0 * u[:, 3] - 1.0
    return x, y, z, q


def system(kind: str, n: int, seed: int):
    """``kind`` is "cube" or "plummer"."""
    if kind == "cube":
        return uniform_cube(n, seed)
    if kind == "plummer":
        return plummer(n, seed)
    raise ValueError(f"unknown distribution {kind!r}")
