"""Oracle: iterative refinement and the accuracy metrics of eq. (error).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* ``refine``: x0 = A_approx^-1 b; then r = b - A x (FP64), x += A_approx^-1 r,
  until ||r||_F <= rtol ||b||_F or ``maxit`` corrections (the factor used as a
  preconditioner for FP64 iterative refinement; the paper uses GMRES instead).
* ``relerr`` = ||A - A_approx|| / ||A|| and ``errsolve`` = ||I - A_approx^-1 A||
  (eq. error), spectral norms estimated by power iteration on B^* B with a
  seeded start block (30 iterations or 1e-3 relative change).
* ``solve_error_bound``: the right side of eq. (err_solve_cond).
"""
from __future__ import annotations

import numpy as np

from . import rsrs


def refine(fac, op, b: np.ndarray, rtol: float = 1e-12, maxit: int = 20):
    b = np.asarray(b, dtype=np.float64)
    x = rsrs.solve(fac, b)
    bn = np.linalg.norm(b)
    hist = []
    for it in range(maxit + 1):
        r = b - op.matvec(x)
        rel = np.linalg.norm(r) / bn
        hist.append(rel)
        if rel <= rtol or it == maxit:
            break
        x = x + rsrs.solve(fac, r)
    return x, hist


def _power(apply_b, apply_bt, n, iters=30, tol=1e-3, seed=7):
    v = np.random.default_rng(seed).standard_normal(n)
    v /= np.linalg.norm(v)
    est = 0.0
    for _ in range(iters):
        w = apply_bt(apply_b(v))
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        new = np.sqrt(nw)
        v = w / nw
        if est and abs(new - est) <= tol * est:
            est = new
            break
        est = new
    return est


def relerr(fac, op, iters=30):
    n = fac.n
    num = _power(lambda v: op.matvec(v) - rsrs.apply(fac, v),
                 lambda v: op.matvec(v, adjoint=True) - rsrs.apply(fac, v, adjoint=True), n, iters)
    den = _power(lambda v: op.matvec(v), lambda v: op.matvec(v, adjoint=True), n, iters)
    return num / den


def errsolve(fac, op, iters=30):
    n = fac.n
    return _power(lambda v: v - rsrs.solve(fac, op.matvec(v)),
                  lambda v: v - op.matvec(rsrs.solve(fac, v, adjoint=True), adjoint=True), n, iters)


def solve_error_bound(eps: float, cond: float) -> float:
    """Bound of eq. (err_solve_cond) on ||x - x~|| / ||x|| when relerr <= eps."""
    return 2.0 * eps * cond / (1.0 - eps * cond)
