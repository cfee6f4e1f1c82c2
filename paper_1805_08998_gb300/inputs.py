"""Seeded synthetic point clouds: the only module both the CUDA path and the oracle use.

It holds none of the method's arithmetic. It draws the point sets on which both sides
build their kernel matrices: uniform points in [0,1]^d and uniform points on the unit
sphere S^2 (a stand-in for the paper's Galerkin matrices on the unit sphere, Sec. 6.1).

Generator (stated so any implementation can reproduce it bit for bit):
  * splitmix64 (Steele, Lea, Flood 2014): the c-th output (c = 0, 1, ...) of the stream
    with seed s is mix(s + (c + 1) * 0x9E3779B97F4A7C15 mod 2^64), where
    mix(z) = z ^ (z >> 30) times 0xBF58476D1CE4E5B9, then ^ (>> 27) times
    0x94D049BB133111EB, then ^ (>> 31), all mod 2^64.
  * u = (output >> 11) * 2^-53, a double in [0, 1).
  * cube, dimension d: point i takes draws c = d*i, ..., d*i + d - 1 as its coordinates.
  * sphere: point i takes u1 = draw 2i, u2 = draw 2i+1; z = 2*u1 - 1, phi = 2*pi*u2,
    s = sqrt(1 - z^2), point = (s*cos(phi), s*sin(phi), z).
Point arrays are row-major (n, dim) float64 in the ORIGINAL order.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

PTS_CUBE = 0
PTS_SPHERE = 1


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of the splitmix64 stream with the given seed."""
    c = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + c * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each splitmix64 output."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def points(kind: int, dim: int, n: int, seed: int) -> np.ndarray:
    """n seeded points, shape (n, dim), float64, original order."""
    if n < 0:
        raise ValueError("n must be non-negative")
    if kind == PTS_CUBE:
        if dim not in (1, 2, 3):
            raise ValueError("cube points need dim in {1, 2, 3}")
        return uniform01(seed, n * dim).reshape(n, dim)
    if kind == PTS_SPHERE:
        if dim != 3:
            raise ValueError("sphere points need dim == 3")
        u = uniform01(seed, 2 * n).reshape(n, 2)
        z = 2.0 * u[:, 0] - 1.0
        phi = 2.0 * np.pi * u[:, 1]
        s = np.sqrt(1.0 - z * z)
        return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)
    raise ValueError(f"unknown point distribution {kind}")


def gaussian_ratio_inputs(seed: int, n: int) -> np.ndarray:
    """Uniform draws handed to tests that need extra seeded numbers (e.g. scaling vectors)."""
    return uniform01(seed, n)
