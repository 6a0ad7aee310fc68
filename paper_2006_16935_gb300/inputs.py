"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the solver itself: it only draws numbers.
Both sides of every parity test receive the same arrays from here (the CUDA
library also has its own device-side generator of the *same* published
counter-based hash, tested bit-exactly against this one).

Initial wave-function (the paper's INITCONDTYPE 1 draws Gaussian noise; the
synthetic workloads draw i.i.d. uniform values instead): Re and Im of every
site are independent U[-1, 1) values taken from SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) run in
counter mode:

    key  = (seed * 0x9E3779B97F4A7C15  XOR  (2*site + part))  mod 2**64
    z    = splitmix64(key)
    u    = (z >> 11) * 2**-53             in [0, 1)
    value = 2*u - 1                       in [-1, 1)   (exact in binary64)

with site = (x*N + y)*N + z the row-major index and part 0 for Re, 1 for Im.

Gaussian white noise (for the random-field potentials): the same two uniforms
u0, u1 of a site (parts 0 and 1 above, as u in [0, 1)) through the Box-Muller
transform (Box and Muller, Ann. Math. Statist. 29, 1958):
    g = sqrt(-2 ln(1 - u0)) cos(2 pi u1).
"""
from __future__ import annotations

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(key: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to a uint64 counter array."""
    with np.errstate(over="ignore"):
        z = key.astype(np.uint64) + GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, counters: np.ndarray) -> np.ndarray:
    """U[-1, 1) doubles for the given uint64 counters under `seed`."""
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GOLDEN_GAMMA
    z = splitmix64(base ^ counters.astype(np.uint64))
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def uniform_psi(n: int, seed: int, chunk: int = 1 << 24) -> np.ndarray:
    """Seeded complex128 lattice [n, n, n] with Re, Im i.i.d. U[-1, 1)."""
    total = n * n * n
    out = np.empty(total, dtype=np.complex128)
    view = out.view(np.float64)  # interleaved re, im
    for start in range(0, 2 * total, chunk):
        stop = min(2 * total, start + chunk)
        view[start:stop] = uniform_pm1(seed, np.arange(start, stop, dtype=np.uint64))
    return out.reshape(n, n, n)


def plane_wave_mix(n: int, seed: int, modes: int = 4):
    """A few random lattice plane waves: returns (mode indices [m,3], complex amplitudes [m]).

    The lattice function is  psi(x) = sum_j c_j exp(2*pi*i * n_j . x / N); used
    for checks that hold at any lattice size (plane waves are eigenvectors of
    every FFT kinetic term).
    """
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, n, size=(modes, 3))
    idx[0] = [n // 2, n // 2, n // 2]  # always include the Nyquist corner
    amp = rng.uniform(-1, 1, modes) + 1j * rng.uniform(-1, 1, modes)
    return idx.astype(np.int64), amp


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """U[0, 1) doubles (multiples of 2**-53) for the given uint64 counters."""
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GOLDEN_GAMMA
    z = splitmix64(base ^ counters.astype(np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian_noise(n: int, seed: int) -> np.ndarray:
    """Seeded float64 lattice [n, n, n] of i.i.d. N(0, 1) values (Box-Muller on
    the counter-mode uniforms of parts 0 and 1 of every site)."""
    site = np.arange(n * n * n, dtype=np.uint64)
    u0 = uniform01(seed, 2 * site)
    u1 = uniform01(seed, 2 * site + np.uint64(1))
    return (np.sqrt(-2.0 * np.log(1.0 - u0)) * np.cos(2.0 * np.pi * u1)).reshape(n, n, n)
