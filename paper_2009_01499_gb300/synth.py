"""Seeded synthetic inputs (no solver arithmetic here).

Both the CUDA path's tests/benchmark and the oracle draw their inputs from
this module, so the two sides see identical random vectors.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): state_k = seed + k * 0x9E3779B97F4A7C15
(mod 2^64), output = mix(state_k) with the published 64-bit finaliser.  A
double in [0, 1) is the top 53 bits times 2^-53.

The paper only says "random vector" for the initial guess (Section 5); the
uniform [-1, 1] distribution and the SplitMix64 stream are this project's
choice.  Seeds: workload index + 20090149.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 20090149


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the SplitMix64 stream of `seed`."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_pm1(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """i.i.d. uniform [-1, 1) doubles."""
    return 2.0 * uniform01(seed, count, offset) - 1.0


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normals by the Box-Muller transform of consecutive uniform pairs."""
    u = uniform01(seed, 2 * count, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def initial_guess(n_total: int, seed: int) -> np.ndarray:
    """Random initial guess u_0 (Section 5: "a random vector")."""
    return uniform_pm1(seed, n_total)


def coefficients(n_total: int, seed: int) -> np.ndarray:
    """Seeded uniform[-1,1] B-spline coefficients of f."""
    return uniform_pm1(seed ^ 0x5DEECE66D, n_total)


def bumps(nb: int, seed: int) -> np.ndarray:
    """nb Gaussian source bumps as rows (a_k, cx_k, cy_k): amplitudes N(0,1), centres
    uniform in [0.1, 0.9]^2 (the width 0.05 keeps each bump inside the domain)."""
    a = normal(seed, nb)
    c = 0.1 + 0.8 * uniform01(seed ^ 0x9E37, 2 * nb)
    return np.stack([a, c[0::2], c[1::2]], axis=1).astype(np.float64)
