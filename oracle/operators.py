"""Oracle: the matrices A and their products, written out plainly in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Kernel matrices (Sec. 3, with the diagonal reading of the workloads):
    A = shift * I + scale * K,   K_ij = G(x_i, x_j) for i != j,  K_ii = 0,
    G = log|x - y| in 2D,  G = 1/|x - y| in 3D.
A is symmetric, so A* = A.  The sketches Y = A Omega, Z = A* Psi of eq.
(rand_sample_setting) are formed by row blocks of the dense matrix.

The 7-point operator (not in the paper; stands in for the PDE-derived matrices
of Exp. 3): cell-centred finite volumes on an n^3 grid of cells of [0,1]^3,
(A u)_i = sum over the 6 faces of beta_f (u_i - u_j) with beta_f the harmonic
mean 2 b_i b_j / (b_i + b_j) of the two cell coefficients, and beta_f = 2 b_i on
a boundary face (u = 0 beyond the wall).  It is symmetric positive definite.
"""
from __future__ import annotations

import numpy as np


def kernel_entries(kind: str, xi: np.ndarray, xj: np.ndarray, ii: np.ndarray, jj: np.ndarray) -> np.ndarray:
    """K(x_i, x_j) for the index sets ii (rows) and jj (cols); zero where ii == jj."""
    diff = xi[:, None, :] - xj[None, :, :]
    r = np.sqrt(np.sum(diff * diff, axis=2))
    same = ii[:, None] == jj[None, :]
    r = np.where(same, 1.0, r)
    if kind == "log2d":
        k = np.log(r)
    elif kind == "invr3d":
        k = 1.0 / r
    else:
        raise ValueError(kind)
    return np.where(same, 0.0, k)


class KernelOperator:
    """A = shift*I + scale*K over the points, applied densely by row blocks."""

    def __init__(self, kind: str, points: np.ndarray, shift: float, scale: float, block: int = 1024):
        self.kind = kind
        self.points = np.asarray(points, dtype=np.float64)
        self.n = self.points.shape[0]
        self.shift = shift
        self.scale = scale
        self.block = block

    def rows(self, idx: np.ndarray) -> np.ndarray:
        """Dense rows A[idx, :]."""
        idx = np.asarray(idx)
        allj = np.arange(self.n)
        a = self.scale * kernel_entries(self.kind, self.points[idx], self.points, idx, allj)
        a[np.arange(len(idx)), idx] += self.shift
        return a

    def dense(self) -> np.ndarray:
        return self.rows(np.arange(self.n))

    def matvec(self, x: np.ndarray, adjoint: bool = False) -> np.ndarray:
        """A x (A symmetric, so the adjoint is the same product)."""
        x = np.asarray(x, dtype=np.float64)
        out = np.empty_like(x)
        for i0 in range(0, self.n, self.block):
            idx = np.arange(i0, min(self.n, i0 + self.block))
            out[idx] = self.rows(idx) @ x
        return out


class Stencil7Operator:
    """7-point variable-coefficient operator on an n^3 cell grid (x fastest)."""

    def __init__(self, n_side: int, coef: np.ndarray):
        self.m = n_side
        self.n = n_side ** 3
        self.b = np.asarray(coef, dtype=np.float64).reshape(n_side, n_side, n_side)  # [z, y, x]

    def matvec(self, x: np.ndarray, adjoint: bool = False) -> np.ndarray:
        m = self.m
        x = np.asarray(x, dtype=np.float64)
        shp = x.shape
        u = x.reshape((m, m, m) + shp[1:])
        b = self.b
        out = np.zeros_like(u)
        for axis in range(3):
            bb = b
            # interior faces along this axis
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[axis] = slice(0, m - 1)
            hi[axis] = slice(1, m)
            bl, bh = bb[tuple(lo)], bb[tuple(hi)]
            beta = 2.0 * bl * bh / (bl + bh)
            beta = beta.reshape(beta.shape + (1,) * (u.ndim - 3))
            flux = beta * (u[tuple(lo)] - u[tuple(hi)])
            out[tuple(lo)] += flux
            out[tuple(hi)] -= flux
            # boundary faces (Dirichlet wall half a cell away)
            for end in (0, m - 1):
                e = [slice(None)] * 3
                e[axis] = slice(end, end + 1)
                be = 2.0 * bb[tuple(e)]
                be = be.reshape(be.shape + (1,) * (u.ndim - 3))
                out[tuple(e)] += be * u[tuple(e)]
        return out.reshape(shp)

    def dense(self) -> np.ndarray:
        return self.matvec(np.eye(self.n))


def make_operator(problem) -> KernelOperator | Stencil7Operator:
    if problem.kernel == "stencil7":
        return Stencil7Operator(problem.grid_side, problem.coefficients())
    return KernelOperator(problem.kernel, problem.points, problem.diag_shift, problem.scale)


def sample(op, omega: np.ndarray, psi: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Y = A Omega and Z = A* Psi (eq. rand_sample_setting)."""
    return op.matvec(omega), op.matvec(psi, adjoint=True)
