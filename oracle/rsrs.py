"""Oracle: Algorithm 1 (randomized strong recursive skeletonization), literally, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

``factor`` takes the sketch quartet {Y, Z, Omega, Psi} of eq.
(rand_sample_setting) and walks the tree from the deepest level to level 1.
For each compressed box B, in the processing order of ``oracle.tree.Schedule``:

1. B_act, N_act  -- active indices of B and of its neighbours (eq. BNactive).
2. Y'_B = Y_B null([Om_B; Om_N]),  Z'_B = Z_B null([Psi_B; Psi_N])
   (eq. nullYZ, Algorithm 1), with the full null space (s - l columns).
3. [R u S, T] = id([Y'_B | Z'_B]): the ID of the concatenation, as prescribed
   for a simultaneous row/column skeleton in Sec. 3.1 (eq.
   skel_lowrank_simult); rank k' = min(k, b).
4. E/F updates: Y_R -= T^T Y_S, Z_R -= T^T Z_S, Om_S += T Om_R,
   Psi_S += T Psi_R (eq. orth_sparsifying and Sec. 4.3).
5. Block extraction on the updated ("hatted") sketches (eq. pinvYZ):
   [X_RR X_RS X_RN] = Y_R pinv([Om_B; Om_N]) and
   [X_RR X_SR X_NR]^T = Z_R pinv([Psi_B; Psi_N]); X_RR, X_RS, X_RN are taken
   from the Y side and X_SR, X_NR from the Z side.
6. L and U of eq. (LUstrong) from an LU of X_RR, and the updates
   Y <- L Y, Om <- U^-1 Om, Z <- U^* Z, Psi <- L^-* Psi (Algorithm 1).
7. R leaves the active set.

Then the remaining active block is extracted densely,
A~_{Bt Bt} = Y_Bt pinv(Om_Bt), and LU-factorised.  ``solve``/``apply`` use the
factorization of eqs. (Afact) and (Ainvfact); the adjoints follow by taking
the adjoint of every factor.  Everything is indexed by original point number.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import linalg as la
from .tree import Schedule, Tree

EPS = np.finfo(np.float64).eps


def id_tau(b: int, s: int) -> float:
    """Residual, relative to |R_00|, below which the remaining CPQR pivots are numerically dependent
    (Sec. 2.3's greedy pivoted QR, stopped at the fixed rank k' of Sec. 4.5): 64 eps max(b, 2s)
    bounds the rounding of the Householder steps on a b x 2s sketch."""
    return 64.0 * EPS * max(b, 2 * s)


def nullification_rounding(s: int) -> float:
    """Rounding level, relative to the largest row of [Y_B | Z_B] before nullification, of a box's
    nullified sketch when its far field is exactly zero (Sec. 4.1): every entry of Y_B times a null
    basis (or the projector onto it) is a sum of s products of a row of norm |Y_i| with a unit
    vector, rounded to about eps |Y_i|, so a row of the 2s-column concatenation keeps about
    eps sqrt(2s) |Y_i| of rounding.  What the near field leaves behind is at most this."""
    return EPS * np.sqrt(2.0 * s)


@dataclass
class BoxFactor:
    box_id: int
    level: int
    colour: int
    B: np.ndarray  # active indices of the box before compression (tree order)
    S: np.ndarray  # skeletons, pivot order
    R: np.ndarray  # redundant, tree order
    N: np.ndarray  # active neighbour indices (tree order)
    T: np.ndarray  # k' x r
    XRR: np.ndarray
    lu: tuple
    LcS: np.ndarray  # X_SR X_RR^-1   (k' x r)
    LcN: np.ndarray  # X_NR X_RR^-1   (n x r)
    UcS: np.ndarray  # X_RR^-1 X_RS   (r x k')
    UcN: np.ndarray  # X_RR^-1 X_RN   (r x n)
    XRR_z: np.ndarray = None  # X_RR as estimated from the Z side (diagnostic)
    pivot_gap: np.ndarray = None  # per CPQR step: (largest - second residual norm) / |R_00|
    pivot_runner: np.ndarray = None  # per CPQR step: the runner-up point
    pivot_dependent: np.ndarray = None  # per CPQR step: taken by the dependent-pivot rule
    pivot_shortfall: np.ndarray = None  # per CPQR step and box point: (largest - its residual) / |R_00|
    pivot_margin: np.ndarray = None  # per CPQR step: largest residual / the dependence threshold


@dataclass
class Factor:
    n: int
    k: int
    s: int
    boxes: list = field(default_factory=list)
    root: np.ndarray = None  # B_t (tree order)
    root_A: np.ndarray = None
    root_lu: tuple = None


def _tree_sorted(idx: np.ndarray, pos: np.ndarray) -> np.ndarray:
    return idx[np.argsort(pos[idx], kind="stable")]


def factor(tree: Tree, sched: Schedule, Y, Z, Om, Ps, trace=None, max_steps: int | None = None) -> Factor:
    """Algorithm 1 on copies of the sketch quartet.  ``trace`` (a list) receives per-box dumps.

    ``max_steps`` stops after that many compressed boxes and skips the root (used
    only to time a bounded sample of a large workload)."""
    Y, Z, Om, Ps = (np.array(a, dtype=np.float64, copy=True) for a in (Y, Z, Om, Ps))
    n, s = Y.shape
    k = sched.k
    fac = Factor(n=n, k=k, s=s)
    act = {b.id: b.pts.copy() for b in tree.boxes if b.is_leaf}
    steps_by_level = {}
    for st in sched.steps:
        steps_by_level.setdefault(st["level"], []).append(st)
    for level in range(tree.depth, 0, -1):
        for b in tree.levels.get(level, []):
            if not b.is_leaf:
                act[b.id] = np.concatenate([act[c.id] for c in b.children])
        for st in steps_by_level.get(level, []):
            if max_steps is not None and len(fac.boxes) >= max_steps:
                return fac
            box = st["box"]
            Bact = act[box.id]
            Nact = (np.concatenate([act[c.id] for c in st["nbrs"]]) if st["nbrs"]
                    else np.zeros(0, dtype=np.int64))
            BN = np.concatenate([Bact, Nact])
            b, l = len(Bact), len(BN)
            assert b == st["b"] and l == st["b"] + st["n"]
            # step 2: block nullification
            Yp = Y[Bact] @ la.null(Om[BN])
            Zp = Z[Bact] @ la.null(Ps[BN])
            # step 3: ID of the concatenation
            kp = min(k, b)
            rec = {}
            # pivots are numerically dependent below tau |R_00| (the fixed-rank greedy ID), or below
            # the rounding level of the nullification itself, scaled by the largest row of [Y_B | Z_B]
            # before nullification: a box whose far field is exactly zero (a sparse operator's box
            # before fill-in reaches it) then has only dependent pivots and T = 0
            tau = id_tau(b, s)
            scale2 = np.sum(Y[Bact] ** 2, axis=1) + np.sum(Z[Bact] ** 2, axis=1)
            floor = nullification_rounding(s) * np.sqrt(np.max(scale2))
            skel, red, T = la.cpqr_id(np.hstack([Yp, Zp]), kp, tau, record=rec, floor=floor)
            S, R = Bact[skel], Bact[red]
            # step 4: sparsification E, F
            Y[R] -= T.T @ Y[S]
            Z[R] -= T.T @ Z[S]
            Om[S] += T @ Om[R]
            Ps[S] += T @ Ps[R]
            # step 5: block extraction on the hatted sketches
            Xy = la.pinv_right(Y[R], Om[BN])
            Xz = la.pinv_right(Z[R], Ps[BN])
            cN = np.arange(b, l)
            XRR, XRS, XRN = Xy[:, red], Xy[:, skel], Xy[:, cN]
            XSR, XNR = Xz[:, skel].T, Xz[:, cN].T
            # step 6: block elimination
            f = la.lu(XRR)
            UcS, UcN = la.lu_solve(f, XRS), la.lu_solve(f, XRN)
            LcS = la.lu_solve(f, XSR.T, trans=1).T
            LcN = la.lu_solve(f, XNR.T, trans=1).T
            YR = Y[R].copy()
            Y[S] -= LcS @ YR
            Y[Nact] -= LcN @ YR
            Om[R] += UcS @ Om[S] + UcN @ Om[Nact]
            ZR = Z[R].copy()
            Z[S] -= UcS.T @ ZR
            Z[Nact] -= UcN.T @ ZR
            Ps[R] += LcS.T @ Ps[S] + LcN.T @ Ps[Nact]
            # step 7: R leaves the active set
            act[box.id] = _tree_sorted(S, tree.pos)
            bf = BoxFactor(box_id=box.id, level=level, colour=st["colour"], B=Bact, S=S, R=R, N=Nact,
                           T=T, XRR=XRR, lu=f, LcS=LcS, LcN=LcN, UcS=UcS, UcN=UcN, XRR_z=Xz[:, red].T,
                           pivot_gap=np.array(rec.get("gap", [])),
                           pivot_runner=Bact[np.array(rec.get("runner", []), dtype=np.int64)]
                           if rec.get("runner") else np.zeros(0, dtype=np.int64),
                           pivot_dependent=np.array(rec.get("dependent", []), dtype=bool),
                           pivot_shortfall=np.array(rec.get("shortfall", [])),
                           pivot_margin=np.array(rec.get("margin", [])))
            fac.boxes.append(bf)
            if trace is not None:
                trace.append(dict(box=bf, Yp=Yp, Zp=Zp, scale2=scale2))
    if tree.depth == 0:
        Bt = np.arange(n)
    else:
        Bt = np.concatenate([act[b.id] for b in tree.levels[1]])
    Bt = _tree_sorted(Bt, tree.pos)
    fac.root = Bt
    fac.root_A = la.pinv_right(Y[Bt], Om[Bt])
    fac.root_lu = la.lu(fac.root_A)
    fac.final = dict(Y=Y, Z=Z, Om=Om, Ps=Ps)
    return fac


def sweep_inv(fac: Factor, f: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """V_M^-1 ... V_1^-1 f (V^-1 = L E), or for the adjoint W_M^-* ... W_1^-* f (W^-* = U^* F^*)."""
    x = np.array(f, dtype=np.float64, copy=True)
    for bf in fac.boxes:
        R, S, N = bf.R, bf.S, bf.N
        x[R] -= bf.T.T @ x[S]
        xR = x[R].copy()
        x[S] -= (bf.UcS.T if adjoint else bf.LcS) @ xR
        x[N] -= (bf.UcN.T if adjoint else bf.LcN) @ xR
    return x


def diag_solve(fac: Factor, f: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """P D^-1 P^T f: the X_RR blocks and the root block."""
    x = np.array(f, dtype=np.float64, copy=True)
    for bf in fac.boxes:
        x[bf.R] = la.lu_solve(bf.lu, x[bf.R], trans=1 if adjoint else 0)
    x[fac.root] = la.lu_solve(fac.root_lu, x[fac.root], trans=1 if adjoint else 0)
    return x


def sweep_inv_down(fac: Factor, f: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """W_1^-1 ... W_M^-1 f (W^-1 = F U), or for the adjoint V_1^-* ... V_M^-* f (V^-* = E^* L^*)."""
    x = np.array(f, dtype=np.float64, copy=True)
    for bf in reversed(fac.boxes):
        R, S, N = bf.R, bf.S, bf.N
        if not adjoint:
            x[R] -= bf.UcS @ x[S] + bf.UcN @ x[N]
        else:
            x[R] -= bf.LcS.T @ x[S] + bf.LcN.T @ x[N]
        x[S] -= bf.T @ x[R]
    return x


def solve(fac: Factor, f: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """A_approx^-1 f (eq. Ainvfact): upward pass, block-diagonal solve, downward pass."""
    return sweep_inv_down(fac, diag_solve(fac, sweep_inv(fac, f, adjoint), adjoint), adjoint)


def sweep_fwd(fac: Factor, f: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """W_M ... W_1 f (W = U^-1 F^-1), or for the adjoint V_M^* ... V_1^* f (V^* = L^-* E^-*)."""
    x = np.array(f, dtype=np.float64, copy=True)
    for bf in fac.boxes:
        R, S, N = bf.R, bf.S, bf.N
        x[S] += bf.T @ x[R]
        if not adjoint:
            x[R] += bf.UcS @ x[S] + bf.UcN @ x[N]
        else:
            x[R] += bf.LcS.T @ x[S] + bf.LcN.T @ x[N]
    return x


def diag_apply(fac: Factor, f: np.ndarray, adjoint: bool = False) -> np.ndarray:
    x = np.array(f, dtype=np.float64, copy=True)
    for bf in fac.boxes:
        x[bf.R] = (bf.XRR.T if adjoint else bf.XRR) @ x[bf.R]
    x[fac.root] = (fac.root_A.T if adjoint else fac.root_A) @ x[fac.root]
    return x


def sweep_fwd_down(fac: Factor, f: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """V_1 ... V_M f (V = E^-1 L^-1), or for the adjoint W_1^* ... W_M^* f (W^* = F^-* U^-*)."""
    x = np.array(f, dtype=np.float64, copy=True)
    for bf in reversed(fac.boxes):
        R, S, N = bf.R, bf.S, bf.N
        xR = x[R].copy()
        x[S] += (bf.UcS.T if adjoint else bf.LcS) @ xR
        x[N] += (bf.UcN.T if adjoint else bf.LcN) @ xR
        x[R] += bf.T.T @ x[S]
    return x


def apply(fac: Factor, f: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """A_approx f (eq. Afact)."""
    return sweep_fwd_down(fac, diag_apply(fac, sweep_fwd(fac, f, adjoint), adjoint), adjoint)


def build(problem, omega=None, psi=None, s: int | None = None, p: int | None = None, op=None,
          trace=None):
    """Tree, schedule, sketches and factor for a ``workloads.Problem``.

    Returns (tree, schedule, factor, (Y, Z, Omega, Psi)).
    """
    from .operators import make_operator, sample

    tree = Tree(problem.points, problem.leaf)
    sched = Schedule(tree, problem.k, p)
    if s is None:
        s = max(problem.s_cfg, sched.s_req)
    if s < sched.s_req:
        raise ValueError(f"undersampled: s={s} < s_req={sched.s_req}")
    omega = problem.omega(s) if omega is None else omega
    psi = problem.psi(s) if psi is None else psi
    op = make_operator(problem) if op is None else op
    Y, Z = sample(op, omega, psi)
    fac = factor(tree, sched, Y, Z, omega, psi, trace=trace)
    return tree, sched, fac, (Y, Z, omega, psi)
