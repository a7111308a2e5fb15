"""Oracle: iterative refinement and the accuracy metrics of eq. (error).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* ``refine``: x0 = A_approx^-1 b; then r = b - A x (FP64), x += A_approx^-1 r,
  until ||r||_F <= rtol ||b||_F or ``maxit`` corrections (the factor used as a
  preconditioner for FP64 iterative refinement; the paper uses GMRES instead).
* ``relerr`` = ||A - A_approx|| / ||A|| and ``errsolve`` = ||I - A_approx^-1 A||
  (eq. error), spectral norms estimated by power iteration on B^* B with a
  seeded start block (30 iterations or 1e-3 relative change).
* ``solve_error_bound``: the right side of eq. (err_solve_cond).
* ``gmres``: restarted, right-preconditioned GMRES with the factor as preconditioner (the Krylov
  method of the paper's experiments, Sec. 5), one right-hand side.
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


def gmres(matvec, precond, b: np.ndarray, rtol: float = 1e-12, restart: int = 30, maxit: int = 60):
    """Restarted GMRES(restart) (Saad and Schultz 1986) for A x = b with a right preconditioner:
    solve A M^-1 y = b by Arnoldi on A M^-1 (modified Gram-Schmidt), minimise ||beta e1 - H y||
    with Givens rotations, x = x0 + M^-1 V y; restart from the true residual.  The factor is the
    preconditioner (M^-1 = A_approx^-1) as in the paper's experiments, which report GMRES iteration
    counts.  One right-hand side; returns x, the number of iterations (applications of M^-1) and
    the history [initial relative residual, per-iteration estimates, true residual per restart]."""
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    x = np.zeros(n)
    bn = np.linalg.norm(b)
    hist = []
    total = 0
    while True:
        r = b - matvec(x) if total else b.copy()
        beta = np.linalg.norm(r)
        hist.append(beta / bn)
        if beta / bn <= rtol or total >= maxit:
            return x, total, hist
        V = np.zeros((n, restart + 1))
        H = np.zeros((restart + 1, restart))
        V[:, 0] = r / beta
        g = np.zeros(restart + 1)
        g[0] = beta
        cs, sn = np.zeros(restart), np.zeros(restart)
        k = 0
        while k < restart and total < maxit:
            w = matvec(precond(V[:, k]))
            for i in range(k + 1):
                H[i, k] = V[:, i] @ w
                w = w - H[i, k] * V[:, i]
            H[k + 1, k] = np.linalg.norm(w)
            V[:, k + 1] = w / H[k + 1, k] if H[k + 1, k] > 0 else 0.0
            for i in range(k):
                a, c2 = H[i, k], H[i + 1, k]
                H[i, k], H[i + 1, k] = cs[i] * a + sn[i] * c2, -sn[i] * a + cs[i] * c2
            rho = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = (H[k, k] / rho, H[k + 1, k] / rho) if rho > 0 else (1.0, 0.0)
            H[k, k], H[k + 1, k] = rho, 0.0
            g[k + 1], g[k] = -sn[k] * g[k], cs[k] * g[k]
            k += 1
            total += 1
            hist.append(abs(g[k]) / bn)
            if abs(g[k]) / bn <= rtol:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k]) if k else np.zeros(0)
        x = x + precond(V[:, :k] @ y)
