"""Oracle linear solver: textbook unpreconditioned conjugate gradients (Sec. 2.5, Sec. 3.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def cg(A, b, x0, rtol, max_iter):
    """Hestenes-Stiefel CG without preconditioner.

    Stops as soon as the recursively updated residual satisfies ||r||^2 < rtol^2 ||b||^2 (the
    relative-residual test ||b - Ax|| / ||b|| < rtol), or after max_iter iterations.  b = 0 gives
    x = 0 in zero iterations.  Returns (x, iterations, ||r|| / ||b||).
    """
    b = np.asarray(b, dtype=np.float64)
    bb = float(b @ b)
    if bb == 0.0:
        return np.zeros_like(b), 0, 0.0
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A @ x
    p = r.copy()
    rr = float(r @ r)
    tol2 = rtol * rtol * bb
    k = 0
    while rr >= tol2 and k < max_iter:
        q = A @ p
        alpha = rr / float(p @ q)
        x += alpha * p
        r -= alpha * q
        rr_new = float(r @ r)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        k += 1
    return x, k, float(np.sqrt(rr / bb))
