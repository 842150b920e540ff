"""Dense brute force of one Galerkin step, straight from the integral definitions.

TEST INFRASTRUCTURE ONLY. Used on tiny grids (8 x 8 and similar) to pin the
oracle's closed-form deposit and its banded mass-matrix solves.

Sec. III defines, for basis functions Lambda centred on the nodes,
    Lambda_{j j'} = int dx dp  L(x - x_j) L(p - p_j) L(x - x_j') L(p - p_j')
    Delta_{k j'}  = int dx dp  L(x - x_k - dx_k) L(p - p_k - dp_k) L(x - x_j') L(p - p_j')
    w_fin = Lambda^{-1} Delta^T w_in.
Here every 1-D overlap integral is evaluated by Gauss-Legendre quadrature on
the pieces between the breakpoints of the two piecewise-polynomial factors
(exact for these polynomial degrees), with no closed form. Along the periodic
coordinate the basis functions are periodised, so the integral over one
period equals the sum over periodic images of the integral over the real
line. Along the open momentum axis the basis functions are not truncated and
the integral runs over the real line. The dense system is solved by LU.
"""
from __future__ import annotations

import numpy as np

_GL_X, _GL_W = np.polynomial.legendre.leggauss(4)


def basis_value(kind: str, t: np.ndarray) -> np.ndarray:
    """Unit-spacing basis: 'box' = top-hat of width 1, 'tent' = hat of half-width 1,
    'cubic' = the cubic B-spline (pieces (4 - 6 t^2 + 3 |t|^3)/6 on |t| < 1, (2 - |t|)^3/6 on
    1 <= |t| < 2)."""
    t = np.abs(t)
    if kind == "box":
        return np.where(t < 0.5, 1.0, np.where(t == 0.5, 0.5, 0.0))
    if kind == "tent":
        return np.where(t < 1.0, 1.0 - t, 0.0)
    if kind == "cubic":
        return np.where(t < 1.0, (4.0 - 6.0 * t ** 2 + 3.0 * t ** 3) / 6.0,
                        np.where(t < 2.0, (2.0 - t) ** 3 / 6.0, 0.0))
    raise ValueError(kind)


def _breaks(kind: str, c: float):
    if kind == "box":
        return [c - 0.5, c + 0.5]
    if kind == "cubic":
        return [c - 2.0, c - 1.0, c, c + 1.0, c + 2.0]
    return [c - 1.0, c, c + 1.0]


def overlap_line(kind: str, a: float, b: float) -> float:
    """int_R L(t - a) L(t - b) dt for unit spacing, by piecewise quadrature."""
    pts = sorted(set(_breaks(kind, a) + _breaks(kind, b)))
    total = 0.0
    for s, e in zip(pts[:-1], pts[1:]):
        if e <= s:
            continue
        mid, half = 0.5 * (s + e), 0.5 * (e - s)
        t = mid + half * _GL_X
        total += half * np.sum(_GL_W * basis_value(kind, t - a) * basis_value(kind, t - b))
    return float(total)


def overlap_periodic(kind: str, a: float, b: float, period: int) -> float:
    """Overlap of two periodised basis functions over one period (unit spacing)."""
    total = 0.0
    base = round((a - b) / period)
    for m in range(base - 2, base + 3):
        total += overlap_line(kind, a, b + m * period)
    return total


def dense_step(nx: int, np_: int, hx: float, hp: float, kind: str, u: np.ndarray,
               v: np.ndarray, w_in: np.ndarray, lumped: bool = False):
    """One step from the integral definitions.

    u, v: pushed node positions in cell units ((x' - x0)/hx, (p' - p0)/hp), [np][nx].
    Returns w_fin [np][nx].
    """
    n = nx * np_
    lam_x = np.array([[hx * overlap_periodic(kind, float(i), float(k), nx) for k in range(nx)]
                      for i in range(nx)])
    lam_p = np.array([[hp * overlap_line(kind, float(j), float(k)) for k in range(np_)]
                      for j in range(np_)])
    lam = np.kron(lam_p, lam_x)          # index (j, i) -> j * nx + i
    delta = np.zeros((n, n))
    uf, vf = u.ravel(), v.ravel()
    for k in range(n):
        dx = np.array([hx * overlap_periodic(kind, uf[k], float(i), nx) for i in range(nx)])
        dp = np.array([hp * overlap_line(kind, vf[k], float(j)) for j in range(np_)])
        delta[k, :] = np.kron(dp, dx)
    rhs = delta.T @ w_in.ravel()
    if lumped:
        # lumping: each row of Lambda replaced by its sum over the unbounded
        # lattice, hx * hp (the tent basis is a partition of unity)
        lam = np.eye(n) * hx * hp
    return np.linalg.solve(lam, rhs).reshape(np_, nx)
