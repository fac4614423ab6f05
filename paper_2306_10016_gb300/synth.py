"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module draws numbers and nothing else: it holds none of the convolution
arithmetic.  Every generator is a pure function of (seed, shape) built on a
counter-based SplitMix64 stream, so the same call gives the same bits on x86
and on aarch64 (only +, *, shifts and comparisons touch the integer stream;
the transcendental generators below are documented where they use libm).

Workloads (all complex values are stored as interleaved re/im pairs, i.e. the
memory layout of numpy/torch complex128 and complex64):

* ``unit_disk``   -- entries uniform in the closed unit disk of the complex
                     plane, by rejection from the square [-1, 1]^2.
* ``small_ints``  -- real and imaginary parts independent uniform integers in
                     {-8, ..., 8} (the exact-integer workload).
* ``exp_seq``     -- f_j = exp(2 pi i (A j mod P) / P), the input of the
                     exponential closed form; the angle is reduced in integers.
* ``geom_seq``    -- f_j = rho^j exp(2 pi i (A j mod P) / P).
* ``hermitian_normal`` -- seeded N(0,1) complex entries on the half plane of a
                     centered Hermitian-symmetric spectrum (ky >= 0) with the
                     ky = 0 line made conjugate-symmetric: the spectrum of a
                     real field.
* ``log_uniform_lengths`` -- lengths floor(exp(U(ln lo, ln hi))).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 230610016

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Counter-based SplitMix64: element i is the (offset+i+1)-th output of
    the generator started at ``seed`` (Steele, Lea and Flood, 2014)."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles uniform in [0, 1) with 53 random bits each."""
    z = splitmix64(seed, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def unit_disk(seed: int, shape, dtype=np.complex128) -> np.ndarray:
    """Complex entries uniform in the unit disk (rejection sampling)."""
    n = int(np.prod(shape)) if len(tuple(np.atleast_1d(shape))) else 1
    out = np.empty(n, dtype=np.complex128)
    filled = 0
    offset = 0
    while filled < n:
        want = max(64, int((n - filled) * 1.35) + 64)
        u = uniform01(seed, 2 * want, offset)
        offset += 2 * want
        x = 2.0 * u[0::2] - 1.0
        y = 2.0 * u[1::2] - 1.0
        keep = (x * x + y * y) <= 1.0
        x = x[keep]
        y = y[keep]
        take = min(n - filled, x.size)
        out.real[filled:filled + take] = x[:take]
        out.imag[filled:filled + take] = y[:take]
        filled += take
    return out.reshape(shape).astype(dtype)


def small_ints(seed: int, shape, lo: int = -8, hi: int = 8) -> tuple[np.ndarray, np.ndarray]:
    """Integer real and imaginary parts, independent, uniform in {lo..hi}.

    Returned as two int64 arrays; convert with ``ints_to_complex``."""
    n = int(np.prod(shape))
    span = np.uint64(hi - lo + 1)
    z = splitmix64(seed, 2 * n)
    # top 32 bits times span, high half: an unbiased-enough map onto {0..span-1}
    v = (((z >> np.uint64(32)) * span) >> np.uint64(32)).astype(np.int64) + lo
    return v[0::2].reshape(shape).copy(), v[1::2].reshape(shape).copy()


def ints_to_complex(re: np.ndarray, im: np.ndarray, dtype=np.complex128) -> np.ndarray:
    out = np.empty(re.shape, dtype=dtype)
    out.real = re
    out.imag = im
    return out


def exp_seq(A: int, P: int, L: int, dtype=np.complex128) -> np.ndarray:
    """f_j = exp(2 pi i (A j mod P)/P), j < L; the phase index is reduced
    exactly in integers before the (libm) cos/sin."""
    e = (np.int64(A) * np.arange(L, dtype=np.int64)) % np.int64(P)
    ang = (2.0 * np.pi / P) * e.astype(np.float64)
    return (np.cos(ang) + 1j * np.sin(ang)).astype(dtype)


def geom_seq(rho: float, A: int, P: int, L: int, dtype=np.complex128) -> np.ndarray:
    """f_j = rho^j exp(2 pi i (A j mod P)/P), j < L."""
    mag = np.power(float(rho), np.arange(L, dtype=np.float64))
    return (exp_seq(A, P, L, np.complex128) * mag).astype(dtype)


def standard_normal(seed: int, n: int) -> np.ndarray:
    """N(0,1) doubles by Box-Muller on SplitMix64 uniforms (libm log/cos/sin)."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]          # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:n]


def hermitian_normal(seed: int, K: int, dtype=np.complex128) -> np.ndarray:
    """Half plane of a centered Hermitian-symmetric 2-D spectrum.

    Shape (2K-1, K): row index kx + K - 1 for kx in [-(K-1), K-1], column
    ky in [0, K-1].  Entries are N(0,1) in real and imaginary parts; on the
    ky = 0 column f(-kx, 0) = conj(f(kx, 0)) and f(0, 0) is real, so the
    array is the non-redundant half of the spectrum of a real field."""
    nx = 2 * K - 1
    z = standard_normal(seed, 2 * nx * K).reshape(nx, K, 2)
    a = (z[..., 0] + 1j * z[..., 1]).astype(np.complex128)
    c = K - 1
    for kx in range(1, K):
        a[c - kx, 0] = np.conj(a[c + kx, 0])
    a[c, 0] = a[c, 0].real
    return a.astype(dtype)


def log_uniform_lengths(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n lengths floor(exp(U(ln lo, ln hi))), clipped to [lo, hi]."""
    u = uniform01(seed, n)
    L = np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
    return np.clip(L, lo, hi)
