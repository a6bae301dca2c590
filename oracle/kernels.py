"""Matrix entries of the model problems.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's model problem is the Galerkin Laplace single-layer potential on the
unit sphere (Sec. 2.1, eqn. slp / matcoeff).  Point-kernel stand-ins are used:

* Laplace: a_ij = 1 / (4 pi |p_i - p_j|) for i != j and a_ii = 1 / (4 pi h),
  h = sqrt(4 pi / N) the mean spacing of N points on the unit sphere.
* Matern nu = 3/2: a_ij = (1 + sqrt3 r / l) exp(-sqrt3 r / l), r = |p_i - p_j|,
  l the length scale (diagonal 1).
* Row-weighted Laplace (a non-symmetric matrix diag(w) A for the adjoint
  product, remark after Alg. 3): w_i times the Laplace entry, w_i = 1 + x_i / 2
  with x_i the first coordinate of point i.
"""
from __future__ import annotations

import numpy as np

LAPLACE = "laplace"
MATERN = "matern"
LAPLACE_W = "laplace_w"


def _dist(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    d0 = p[:, None, 0] - q[None, :, 0]
    d1 = p[:, None, 1] - q[None, :, 1]
    d2 = p[:, None, 2] - q[None, :, 2]
    return np.sqrt((d0 * d0 + d1 * d1) + d2 * d2)


def entries(kind: str, pts: np.ndarray, rows: np.ndarray, cols: np.ndarray,
            param: float) -> np.ndarray:
    """Dense sub-matrix A[rows, cols] (original point indices), FP64.

    ``param`` is the diagonal spacing h for Laplace and the length scale for Matern.
    """
    if kind == LAPLACE_W:
        w = 1.0 + 0.5 * pts[rows, 0]
        return w[:, None] * entries(LAPLACE, pts, rows, cols, param)
    r = _dist(pts[rows], pts[cols])
    same = rows[:, None] == cols[None, :]
    if kind == LAPLACE:
        with np.errstate(divide="ignore"):
            a = 1.0 / (4.0 * np.pi * r)
        a[same] = 1.0 / (4.0 * np.pi * param)
        return a
    if kind == MATERN:
        t = np.sqrt(3.0) * r / param
        a = (1.0 + t) * np.exp(-t)
        a[same] = 1.0
        return a
    raise ValueError(kind)


def default_param(kind: str, n: int) -> float:
    """Laplace: the mean spacing sqrt(4 pi / N); Matern: length scale 0.1."""
    if kind in (LAPLACE, LAPLACE_W):
        return float(np.sqrt(4.0 * np.pi / n))
    return 0.1
