"""Oracle: the linear-algebra building blocks of Sec. 2, in plain FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* ``null(M)``   -- orthonormal basis of the null space of a wide l x s matrix
  (eq. null), taken as the trailing s-l columns of the complete Q of a
  Householder QR of M^T (LAPACK through numpy, a library primitive).
* ``pinv_right(Y, M)`` -- Y M^dagger for a wide full-row-rank M, through the
  reduced QR of M^T: M^T = Q R gives M^dagger = Q R^-T (eq. pinvformula).
* ``cpqr_id(M, k, tau)`` -- row interpolative decomposition of M (eq. id_def)
  by column-pivoted Householder QR of M^T stopped after k steps (Sec. 2.3:
  "standard pivoted QR with a greedy approach").  Column norms are recomputed
  from scratch every step; an exact tie goes to the lowest original column.
  Once the largest remaining residual norm is <= tau |R_00| (or <= an absolute
  ``floor``, the rounding level of the sketch) the remaining columns are
  numerically dependent: the rest of the k skeletons are taken in
  ascending original order (a choice among noise-level residuals would not be
  reproducible), and T = R11^-1 R12 is computed with the rows of those
  dependent pivots set to zero (truncated back-substitution; an all-zero sketch
  gives T = 0).
* ``lu`` -- LU with partial pivoting (LAPACK getrf via scipy).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def null(m: np.ndarray) -> np.ndarray:
    l, s = m.shape
    if l >= s:
        raise ValueError("null space needs more columns than rows")
    q, _ = np.linalg.qr(m.T, mode="complete")
    return q[:, l:]


def pinv_right(y: np.ndarray, m: np.ndarray) -> np.ndarray:
    """y @ pinv(m) for m (l x s, l <= s) of full row rank."""
    q, r = np.linalg.qr(m.T, mode="reduced")
    # y Q R^-T = (R^-1 (y Q)^T)^T
    return sla.solve_triangular(r, (y @ q).T, lower=False).T


def cpqr_id(m: np.ndarray, k: int, tau: float, record: dict | None = None, floor: float = 0.0):
    """Row ID of m (b x c): returns (skel, red, T) with m[red] ~= T^T m[skel].

    Pivots whose residual norm is <= tau |R_00| or <= ``floor`` (an absolute noise level) are
    numerically dependent: they are taken in ascending original order and their rows of T are
    zero (truncated back-substitution).

    skel: k row indices in pivot order; red: the other rows, ascending;
    T: k x (b-k) interpolation matrix.  ``record`` (a dict) receives, per pivot
    step, the runner-up row and the gap between the two largest residual norms
    relative to |R_00| (diagnostics for comparing implementations at near-ties).
    """
    a = np.array(m.T, dtype=np.float64, copy=True)  # c x b: pivot over columns = rows of m
    c, b = a.shape
    perm = np.arange(b)
    r00 = None
    j0 = k
    for j in range(k):
        norms = np.sqrt(np.sum(a[j:, j:] ** 2, axis=0))
        best = norms.max()
        if best <= floor or (r00 is not None and best <= tau * r00) or best == 0.0:
            j0 = min(j0, j)
        if j0 <= j:  # dependent: lowest remaining original index
            p = j + int(np.argmin(perm[j:]))
        else:
            cand = np.nonzero(norms == best)[0]
            p = j + cand[np.argmin(perm[j + cand])]
        if record is not None:
            # distance from the dependence thresholds: largest residual / max(floor, tau |R_00|)
            thr = max(floor, tau * r00 if r00 is not None else 0.0)
            record.setdefault("margin", []).append(best / thr if thr > 0 else np.inf)
            order = np.argsort(-norms, kind="stable")
            second = norms[order[1]] if len(order) > 1 else 0.0
            ref = r00 if r00 else best
            record.setdefault("gap", []).append((best - second) / ref if ref else 0.0)
            record.setdefault("runner", []).append(int(perm[j + order[1]]) if len(order) > 1 else -1)
            record.setdefault("dependent", []).append(bool(j0 <= j))
            shortfall = np.full(b, np.inf)  # (best - norm) / |R_00| of every remaining row
            shortfall[perm[j:]] = (best - norms) / ref if ref else 0.0
            record.setdefault("shortfall", []).append(shortfall)
        if p != j:
            a[:, [j, p]] = a[:, [p, j]]
            perm[[j, p]] = perm[[p, j]]
        x = a[j:, j]
        alpha = np.linalg.norm(x)
        if r00 is None:
            r00 = alpha
        if alpha == 0.0:
            continue
        sign = 1.0 if x[0] >= 0 else -1.0
        v = x.copy()
        v[0] += sign * alpha
        v /= np.linalg.norm(v)
        a[j:, j:] -= 2.0 * np.outer(v, v @ a[j:, j:])
    r11 = np.triu(a[:k, :k])
    r12 = a[:k, k:]
    t = np.zeros((k, b - k))
    if j0 > 0:
        t[:j0] = sla.solve_triangular(r11[:j0, :j0], r12[:j0], lower=False)
    skel = perm[:k].copy()
    red = np.sort(perm[k:])
    # columns of t follow perm[k:]; reorder them to ascending red
    order = np.argsort(perm[k:])
    t = t[:, order]
    return skel, red, t


def lu(a: np.ndarray):
    return sla.lu_factor(a)


def lu_solve(f, rhs: np.ndarray, trans: int = 0) -> np.ndarray:
    return sla.lu_solve(f, rhs, trans=trans)
