"""Seeded synthetic workloads for RSRS.

This module is shared by the CPU oracle's tests, the GPU tests and ``bench.py``.
It draws inputs and nothing else: point sets, Gaussian test matrices Omega/Psi,
right-hand sides and the PDE coefficient field.  It holds no step of the method
(no tree, no kernel evaluation, no linear algebra), so that the oracle and the
CUDA path share only their inputs.

Every draw comes from ``numpy.random.default_rng([seed, cfg, problem, stream])``
with the stream numbers below, so that any one array can be regenerated alone.

The five workloads follow the shapes of the paper's experiments (Sec. 5):
a 2D uniform grid and 2D/3D uniform random point clouds for the kernel matrices
of Sec. 3 / Exp. 1 (log kernel in 2D, 1/r in 3D), a batch of independent 2D
problems, and a 3D 7-point variable-coefficient operator standing in for the
PDE-derived matrices of Exp. 3.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 20231101

STREAM_POINTS = 0
STREAM_OMEGA = 1
STREAM_PSI = 2
STREAM_RHS = 3
STREAM_COEF = 4
STREAM_SIZES = 5


def rng_for(cfg: int, problem: int, stream: int, seed: int = MASTER_SEED) -> np.random.Generator:
    return np.random.default_rng([seed, cfg, problem, stream])


def grid_points_2d(n_side: int) -> np.ndarray:
    """Cell centres (i+1/2)/n_side of an n_side x n_side grid in [0,1]^2, row-major in (y, x)."""
    c = (np.arange(n_side, dtype=np.float64) + 0.5) / n_side
    yy, xx = np.meshgrid(c, c, indexing="ij")
    return np.ascontiguousarray(np.stack([xx.ravel(), yy.ravel()], axis=1))


def grid_points_3d(n_side: int) -> np.ndarray:
    """Cell centres of an n_side^3 grid in [0,1]^3, ordered with x fastest."""
    c = (np.arange(n_side, dtype=np.float64) + 0.5) / n_side
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    return np.ascontiguousarray(np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1))


def uniform_points(n: int, d: int, rng: np.random.Generator) -> np.ndarray:
    return np.ascontiguousarray(rng.random((n, d)))


def gaussian(n: int, s: int, rng: np.random.Generator) -> np.ndarray:
    """Standard normal n x s matrix, row-major (one point's s samples contiguous)."""
    return np.ascontiguousarray(rng.standard_normal((n, s)))


@dataclass
class Problem:
    """One RSRS problem instance: geometry, operator kind and sizes."""

    name: str
    cfg: int
    problem: int
    d: int
    kernel: str  # "log2d", "invr3d" or "stencil7"
    points: np.ndarray  # N x d
    leaf: int
    k: int
    s_cfg: int
    nrhs: int
    diag_shift: float = 1.0
    scale: float = 0.0  # A = diag_shift*I + scale*K
    grid_side: int = 0  # stencil7 only
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.points.shape[0]

    def omega(self, s: int) -> np.ndarray:
        return gaussian(self.n, s, rng_for(self.cfg, self.problem, STREAM_OMEGA))

    def psi(self, s: int) -> np.ndarray:
        return gaussian(self.n, s, rng_for(self.cfg, self.problem, STREAM_PSI))

    def rhs(self) -> np.ndarray:
        """N x nrhs right-hand sides, column-major (Fortran order) as the C ABI expects."""
        g = rng_for(self.cfg, self.problem, STREAM_RHS).standard_normal((self.nrhs, self.n))
        return np.asfortranarray(g.T)

    def coefficients(self) -> np.ndarray:
        """Per-cell coefficient b = exp(g), g ~ N(0, 0.5^2) iid (stencil7 only)."""
        g = rng_for(self.cfg, self.problem, STREAM_COEF).normal(0.0, 0.5, self.n)
        return np.exp(g)


def kernel_problem(cfg: int, name: str, points: np.ndarray, kernel: str, leaf: int, k: int,
                   s_cfg: int, nrhs: int, problem: int = 0) -> Problem:
    n = points.shape[0]
    return Problem(name=name, cfg=cfg, problem=problem, d=points.shape[1], kernel=kernel,
                   points=points, leaf=leaf, k=k, s_cfg=s_cfg, nrhs=nrhs,
                   diag_shift=1.0, scale=1.0 / n)


def cell_log_mean(h: float) -> float:
    """Mean of log|x| over the square cell [-h/2, h/2]^2: log(h/sqrt(2)) - 3/2 + pi/4 (from
    int_0^a int_0^a log(x^2 + y^2) dx dy = a^2 (log(2 a^2) - 3 + pi/2) with a = h/2)."""
    return float(np.log(h / np.sqrt(2.0)) - 1.5 + np.pi / 4.0)


def exp1_problem(n_side: int = 284, k: int = 40, nrhs: int = 1) -> Problem:
    """The matrix of the paper's Experiment 1 (Sec. 5.1, eq. Aentries_exp1): collocation points on
    the uniform n_side x n_side grid of the unit square (cell centres), A_ij = log|x_i - x_j| / N for
    i != j and A_ii = the integral of log|x| over the point's cell (h^2 = 1/N times the cell mean),
    leaf m = 4k (c_cap = 4) and n_samples = s of the sample bound (1520 at N = 80,656, k = 40)."""
    pts = grid_points_2d(n_side)
    n = pts.shape[0]
    h = 1.0 / n_side
    return Problem(name=f"exp1_grid{n_side}_k{k}", cfg=91, problem=0, d=2, kernel="log2d", points=pts,
                   leaf=4 * k, k=k, s_cfg=0, nrhs=nrhs, diag_shift=cell_log_mean(h) / n, scale=1.0 / n)


def config(idx: int) -> list[Problem]:
    """The five named workloads (0-based), each a list of problems.

    0: 2D grid 64x64, log kernel, leaf 64, k=32, s=400, 1 RHS.
    1: 2D uniform random N=65536, log kernel, leaf 64, k=48, s=600, 16 RHS.
    2: 3D uniform random N=32768, 1/r kernel, leaf 64, k=64, s=1600, 32 RHS.
    3: 64 independent 2D problems, N ~ U{2048..16384}, leaf 64, k=32, s=400, 1 RHS each.
    4: 7-point variable-coefficient operator on a 64^3 grid, leaf 8^3, k=96, s=2000, 8 RHS.
    """
    if idx == 0:
        return [kernel_problem(0, "grid2d_N4096_k32", grid_points_2d(64), "log2d", 64, 32, 400, 1)]
    if idx == 1:
        pts = uniform_points(65536, 2, rng_for(1, 0, STREAM_POINTS))
        return [kernel_problem(1, "rand2d_N65536_k48", pts, "log2d", 64, 48, 600, 16)]
    if idx == 2:
        pts = uniform_points(32768, 3, rng_for(2, 0, STREAM_POINTS))
        return [kernel_problem(2, "rand3d_N32768_k64", pts, "invr3d", 64, 64, 1600, 32)]
    if idx == 3:
        sizes = rng_for(3, 0, STREAM_SIZES).integers(2048, 16384, size=64, endpoint=True)
        out = []
        for p, n in enumerate(sizes):
            pts = uniform_points(int(n), 2, rng_for(3, p, STREAM_POINTS))
            out.append(kernel_problem(3, f"batch2d_p{p}_N{int(n)}_k32", pts, "log2d", 64, 32, 400, 1,
                                      problem=p))
        return out
    if idx == 4:
        pts = grid_points_3d(64)
        pr = Problem(name="stencil7_64cube_k96", cfg=4, problem=0, d=3, kernel="stencil7", points=pts,
                     leaf=512, k=96, s_cfg=2000, nrhs=8, diag_shift=0.0, scale=1.0, grid_side=64)
        return [pr]
    raise ValueError(f"no workload {idx}")


def small_problem(n_side: int = 0, n: int = 0, d: int = 2, kernel: str = "log2d", leaf: int = 16,
                  k: int = 8, nrhs: int = 2, seed_problem: int = 0, cfg: int = 90) -> Problem:
    """Small seeded problems for tests: a 2D grid (n_side) or n uniform random points in d dims."""
    if n_side:
        pts = grid_points_2d(n_side) if d == 2 else grid_points_3d(n_side)
    else:
        pts = uniform_points(n, d, rng_for(cfg, seed_problem, STREAM_POINTS))
    return kernel_problem(cfg, f"small_{kernel}_{pts.shape[0]}", pts, kernel, leaf, k, 0, nrhs,
                          problem=seed_problem)


# ---- counter-based draws matching the library's device generator ---------------------------
# Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of the multiply-xor round with
# multipliers 0xD2511F53, 0xCD9E8D57 and key increments 0x9E3779B9, 0xBB67AE85.  Counter =
# (q mod 2^32, q >> 32, stream, 0), key = (seed mod 2^32, seed >> 32).  Each output block gives two
# 53-bit uniforms u1 = (a + 1) 2^-53 in (0, 1] and u2 = b 2^-53 from its two 64-bit halves, and the
# Box-Muller pair r cos(2 pi u2), r sin(2 pi u2) with r = sqrt(-2 log u1).  Entry (i, c) of an
# N x s test matrix is member (i*s + c) mod 2 of pair (i*s + c) // 2 (stream 0: Omega, 1: Psi).

def _philox4x32_10(c0, c1, c2, c3, k0, k1):
    m0, m1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
    w0, w1 = np.uint32(0x9E3779B9), np.uint32(0xBB67AE85)
    mask = np.uint64(0xFFFFFFFF)
    for _ in range(10):
        p0 = m0 * c0.astype(np.uint64)
        p1 = m1 * c2.astype(np.uint64)
        n0 = (p1 >> np.uint64(32)).astype(np.uint32) ^ c1 ^ k0
        n2 = (p0 >> np.uint64(32)).astype(np.uint32) ^ c3 ^ k1
        c1 = (p1 & mask).astype(np.uint32)
        c3 = (p0 & mask).astype(np.uint32)
        c0, c2 = n0, n2
        k0 = np.uint32((int(k0) + int(w0)) & 0xFFFFFFFF)
        k1 = np.uint32((int(k1) + int(w1)) & 0xFFFFFFFF)
    return c0, c1, c2, c3


def philox_gaussian(n: int, s: int, seed: int, stream: int) -> np.ndarray:
    """The N x s standard normal test matrix the library draws on the device for (seed, stream)."""
    g = np.arange(n * s, dtype=np.uint64)
    q = g >> np.uint64(1)
    c0 = (q & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    c1 = (q >> np.uint64(32)).astype(np.uint32)
    c2 = np.full_like(c0, np.uint32(stream))
    c3 = np.zeros_like(c0)
    k0 = np.uint32(seed & 0xFFFFFFFF)
    k1 = np.uint32((seed >> 32) & 0xFFFFFFFF)
    o0, o1, o2, o3 = _philox4x32_10(c0, c1, c2, c3, k0, k1)
    a = ((o0.astype(np.uint64) << np.uint64(32)) | o1.astype(np.uint64)) >> np.uint64(11)
    b = ((o2.astype(np.uint64) << np.uint64(32)) | o3.astype(np.uint64)) >> np.uint64(11)
    u1 = (a.astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = b.astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.where((g & np.uint64(1)) == 0, r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2))
    return z.reshape(n, s)
