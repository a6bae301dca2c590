"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module only draws random numbers and places points; it holds none of the
method's arithmetic (no kernel entries, trees, factorizations or codecs), so
that both sides of every parity test can take their inputs from it without
sharing any computation.

Workloads (the paper's model problem is a Laplace single-layer BEM on the unit
sphere, Sec. 2.1; a point-kernel stand-in is used here):

* ``sphere_points`` -- jittered Fibonacci points on the unit sphere.
  z_i = 1 - (2i+1)/N + u_i/N,  phi_i = i*pi*(3 - sqrt 5) + v_i*h,
  u_i, v_i ~ U(-1/2, 1/2), h = sqrt(4 pi / N) (the mean spacing).
* ``cube_points`` -- N uniform points in [0,1]^3.
* ``rhs`` -- x ~ U(-1, 1), shape (N, nrhs), column-major in memory.
* ``codec_values`` -- arrays with a prescribed dynamic range, sign mix and
  zero fraction, used as codec test inputs.
"""
from __future__ import annotations

import numpy as np

SEED_POINTS = 20240506
SEED_RHS = 1
SEED_CODEC = 7


def mean_spacing(n: int) -> float:
    """Mean spacing of n equal-area points on the unit sphere: sqrt(4 pi / n)."""
    return float(np.sqrt(4.0 * np.pi / n))


def sphere_points(n: int, seed: int = SEED_POINTS) -> np.ndarray:
    """(n, 3) float64 C-contiguous jittered Fibonacci points on the unit sphere."""
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.float64)
    u = rng.uniform(-0.5, 0.5, n)
    v = rng.uniform(-0.5, 0.5, n)
    z = 1.0 - (2.0 * i + 1.0) / n + u / n
    z = np.clip(z, -1.0, 1.0)
    phi = i * (np.pi * (3.0 - np.sqrt(5.0))) + v * mean_spacing(n)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    pts = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return np.ascontiguousarray(pts)


def cube_points(n: int, seed: int = SEED_POINTS) -> np.ndarray:
    """(n, 3) float64 C-contiguous uniform points in the unit cube."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.uniform(0.0, 1.0, (n, 3)))


def rhs(n: int, nrhs: int = 1, seed: int = SEED_RHS) -> np.ndarray:
    """(n, nrhs) float64 Fortran-ordered right-hand sides, x ~ U(-1, 1)."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.uniform(-1.0, 1.0, (n, nrhs)))


def codec_values(n: int, dyn_range: float = 1e3, zero_frac: float = 0.0,
                 neg_frac: float = 0.5, seed: int = SEED_CODEC) -> np.ndarray:
    """n float64 values, |v| log-uniform in [1, dyn_range] times a random scale.

    A fraction ``zero_frac`` is set to exactly zero and a fraction ``neg_frac``
    is negative.  The overall scale is drawn log-uniform in [1e-3, 1e3].
    """
    rng = np.random.default_rng(seed)
    scale = 10.0 ** rng.uniform(-3.0, 3.0)
    mag = scale * np.exp(rng.uniform(0.0, np.log(dyn_range), n))
    sign = np.where(rng.uniform(size=n) < neg_frac, -1.0, 1.0)
    v = sign * mag
    if zero_frac > 0:
        v[rng.uniform(size=n) < zero_frac] = 0.0
    return v


def orthonormal_columns(n: int, k: int, seed: int) -> np.ndarray:
    """(n, k) random matrix with orthonormal columns (QR of a Gaussian matrix)."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return np.asfortranarray(q)


def decaying_spectrum(k: int, ratio: float, seed: int) -> np.ndarray:
    """k positive singular values decaying geometrically from 1 to about ``ratio``."""
    rng = np.random.default_rng(seed)
    if k == 1:
        return np.ones(1)
    base = np.geomspace(1.0, ratio, k)
    return np.sort(base * np.exp(rng.uniform(-0.1, 0.1, k)))[::-1].copy()
