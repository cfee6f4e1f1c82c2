"""Test infrastructure (never imported by the library): the Gaussian test matrices that the
randomized compressors draw, restated on the oracle's side so that an oracle compressor can be
fed the very samples the device drew.

The library draws its samples on the device and cannot take them as inputs, so each side
implements the same counter-based generator from its published parts:
  * splitmix64 (Steele, Lea, Flood 2014): output c of the stream with seed s is
    mix(s + (c + 1) * 0x9E3779B97F4A7C15 mod 2^64);
  * entry (i, c) of the test matrix Omega of target leaf L in sampling round rd uses the counter
    t = ((L * 64 + rd) * 64 + c) * 2^24 + i and the stream outputs z1 = 2t and z2 = 2t + 1;
  * u1 = ((z1 >> 40) + 1) * 2^-24 in (0, 1] and u2 = (z2 >> 40) * 2^-24 in [0, 1);
  * Box-Muller (Box and Muller 1958): g = sqrt(-2 ln u1) cos(2 pi u2), rounded to FP32.
Here g is evaluated in FP64 and rounded once to FP32; the device evaluates it in FP32, so the
two sides can differ in the last bit or two of an entry."""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _stream(seed: int, c: np.ndarray) -> np.ndarray:
    """Outputs c (an array of indices) of the splitmix64 stream with the given seed."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def omega(seed: int, leaf: int, rd: int, n: int, k: int) -> np.ndarray:
    """The n x k Gaussian test matrix of target leaf `leaf` in sampling round `rd`, as float64
    arrays holding FP32 values."""
    if not (0 <= n < (1 << 24) and 0 <= k <= 64 and 0 <= rd < 64 and leaf >= 0):
        raise ValueError("index outside the generator's counter layout")
    i = np.arange(n, dtype=np.uint64)[:, None]
    c = np.arange(k, dtype=np.uint64)[None, :]
    t = (((np.uint64(leaf) * np.uint64(64) + np.uint64(rd)) * np.uint64(64) + c) << np.uint64(24)) + i
    z1 = _stream(seed, np.uint64(2) * t)
    z2 = _stream(seed, np.uint64(2) * t + np.uint64(1))
    u1 = ((z1 >> np.uint64(40)) + np.uint64(1)).astype(np.float64) * 2.0 ** -24
    u2 = (z2 >> np.uint64(40)).astype(np.float64) * 2.0 ** -24
    g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return g.astype(np.float32).astype(np.float64)
