"""Pins for the oracle's tree, neighbour lists, colouring and sample bound (Sec. 3, Sec. 4.5)."""
import numpy as np
import pytest

import workloads as W
from oracle.tree import Schedule, Tree


def _leaves(tr):
    return [b for b in tr.boxes if b.is_leaf]


@pytest.mark.parametrize("pts_fn,leaf", [
    (lambda: W.grid_points_2d(32), 16),
    (lambda: W.uniform_points(3000, 2, W.rng_for(91, 0, 0)), 20),
    (lambda: W.uniform_points(3000, 3, W.rng_for(92, 0, 0)), 24),
    (lambda: np.vstack([W.uniform_points(1500, 2, W.rng_for(93, 0, 0)) * 0.05,
                        W.uniform_points(500, 2, W.rng_for(93, 1, 0))]), 12),
])
def test_tree_partition_and_balance(pts_fn, leaf):
    pts = pts_fn()
    tr = Tree(pts, leaf)
    leaves = _leaves(tr)
    allpts = np.sort(np.concatenate([b.pts for b in leaves]))
    assert np.array_equal(allpts, np.arange(len(pts)))  # every point in exactly one leaf
    assert all(len(b.pts) <= leaf for b in leaves)
    # every box holds exactly the points of its children
    for b in tr.boxes:
        if not b.is_leaf:
            assert np.array_equal(np.sort(np.concatenate([c.pts for c in b.children])), b.pts)
    # points lie inside their leaf's cube (brute force on the geometry)
    for b in leaves:
        h = 1.0 / (1 << b.level)
        lo = np.array(b.coord) * h
        inside = (pts[b.pts] >= lo - 1e-15) & (pts[b.pts] <= lo + h + 1e-15)
        assert inside.all()
    # 2:1 balance between adjacent leaves
    for a in leaves:
        for c in leaves:
            if Tree.touches(a, c):
                assert abs(a.level - c.level) <= 1
    # tree order: each box is a contiguous range of tree positions
    for b in tr.boxes:
        pos = np.sort(tr.pos[b.pts])
        assert pos[0] == b.first_pos and pos[-1] == b.first_pos + len(b.pts) - 1


def test_uniform_grid_neighbour_counts():
    tr = Tree(W.grid_points_2d(64), 64)  # 8 x 8 leaves at level 3
    assert tr.depth == 3
    cands = tr.candidates(3)
    for b in tr.levels[3]:
        nb = tr.neighbours(b, cands)
        i, j = b.coord
        expect = (min(i + 1, 7) - max(i - 1, 0) + 1) * (min(j + 1, 7) - max(j - 1, 0) + 1) - 1
        assert len(nb) == expect
        # brute force on the geometry: centres at most one box width apart in each axis
        for c in cands:
            close = max(abs(c.coord[0] - i), abs(c.coord[1] - j)) <= 1 and c is not b
            assert close == (c in nb)


@pytest.mark.parametrize("leaf,k", [(16, 4), (64, 32)])
def test_colouring_is_conflict_free(leaf, k):
    tr = Tree(W.uniform_points(4000, 2, W.rng_for(94, 0, 0)), leaf)
    sc = Schedule(tr, k)
    by = {}
    for st in sc.steps:
        by.setdefault((st["level"], st["colour"]), []).append(st)
    for group in by.values():
        seen = set()
        for st in group:
            closed = {st["box"].id} | {c.id for c in st["nbrs"]}
            assert not (closed & seen)
            seen |= closed


@pytest.mark.parametrize("k", [40, 60])
def test_paper_sample_count_grid(k):
    """Exp. 1 prints n_samples = 37k + p (1520 at k=40, 2280 at k=60) for the 2D grid, m = 4k."""
    tr = Tree(W.grid_points_2d(284), 4 * k)  # N = 80,656, the smallest grid of the paper's table
    sc = Schedule(tr, k, p=k)
    assert sc.s_req == 37 * k + k
    assert {40: 1520, 60: 2280}[k] == sc.s_req


def test_uniform_3d_sample_count():
    """Eq. (s_uniform): s = (6^d + 1) k + p for a uniform 3D tree with 2^d k active points per tree box."""
    k = 2
    tr = Tree(W.grid_points_3d(32), 16)  # leaves of 8 points at level 4; level-3 boxes hold 8k active
    sc = Schedule(tr, k, p=k)
    assert sc.s_req == (6 ** 3 + 1) * k + k


def test_sizes_and_root():
    tr = Tree(W.grid_points_2d(64), 64)
    sc = Schedule(tr, 32)
    assert sc.root_size == 16 * 32  # 16 level-2 boxes keep k skeletons each
    assert sc.s_req >= sc.root_size + sc.p
    # sizes are consistent: b = sum of children's k', r = b - k'
    for st in sc.steps:
        assert st["r"] == st["b"] - st["kp"] and st["kp"] == min(32, st["b"])
