"""Coefficients of the kernels' arctangent (atan01 in hjcd_internal.cuh and
its packed copy atan_poly2 in k_ccd.cu).

atan(t) on [0, 1] is approximated as t * P(t^2) with P of degree 7.  The
coefficients minimise the largest absolute error max |t P(t^2) - atan(t)| over
a dense grid of [0, 1] -- a linear program in the eight coefficients and the
error bound (the discrete minimax, the Chebyshev approximation of the
equioscillation theorem on the grid), solved by scipy's HiGHS.  Printed with
ten significant digits, highest degree first (the kernels' Horner order):

    python paper_2510_07514_gb300/csrc/fit_atan.py
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linprog

DEGREE = 7  # of P in s = t^2


def fit(points: int = 4001) -> tuple[np.ndarray, float]:
    """(coefficients c_0..c_DEGREE of P, lowest degree first; the LP's error bound)."""
    # Chebyshev-spaced points cluster at the ends of [0, 1], where the error peaks first
    t = 0.5 - 0.5 * np.cos(np.pi * np.arange(points) / (points - 1))
    A = t[:, None] * (t[:, None] ** 2) ** np.arange(DEGREE + 1)[None, :]
    f = np.arctan(t)
    # variables (c_0 .. c_D, z): minimise z subject to -z <= A c - f <= z
    ones = np.ones((points, 1))
    A_ub = np.vstack([np.hstack([A, -ones]), np.hstack([-A, -ones])])
    b_ub = np.concatenate([f, -f])
    cost = np.zeros(DEGREE + 2)
    cost[-1] = 1.0
    res = linprog(cost, A_ub=A_ub, b_ub=b_ub, bounds=[(None, None)] * (DEGREE + 2), method="highs")
    if not res.success:
        raise RuntimeError(res.message)
    return res.x[:-1], float(res.x[-1])


def formatted(c: np.ndarray) -> list[str]:
    """The coefficients as they appear in the kernels' source, highest degree first."""
    return [f"{v:.9e}" for v in c[::-1]]


if __name__ == "__main__":
    c, z = fit()
    print(f"max |t P(t^2) - atan t| on the grid: {z:.3e}")
    for s in formatted(c):
        print(f"{s}f")
