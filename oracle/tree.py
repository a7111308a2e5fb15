"""Oracle: quad/octree, neighbour lists, processing order and sample bound.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Geometry of Sec. 3 (tree, adjacency, near/far field), the active counts of
Sec. 4.4 and the sample bound s_B of Sec. 4.5, written plainly in Python with no shared code
with the CUDA library's own tree builder, so that the two can be compared.

Readings where the paper is silent:
* root cube: [0,1]^d when every point lies in it, else the bounding cube of the
  points anchored at the per-dimension minimum;
* points are binned by integer coordinates floor((x-lo)/side * 2^20), clamped;
* a box with more than ``leaf_cap`` points is split into 2^d children in Morton
  order (x bit lowest); empty children are not created;
* 2:1 balance (Sec. 3): a leaf is split while an adjacent leaf is two or more
  levels deeper;
* at level l the active points are partitioned among the level-l boxes and the
  not-yet-processed leaves of coarser levels; a box's neighbours are those of
  them that touch it (face, edge or corner), excluding itself;
* a box is compressed only when it has more than k active points and a
  non-empty far field; boxes of one level are processed colour by colour,
  colours from a greedy colouring (Morton order) of the graph in which two
  boxes conflict when their closed neighbourhoods intersect, and by ascending
  Morton key inside a colour;
* s_req = max over compressed boxes of (b + n at processing time) + k + p,
  and at least |B_t| + p for the final active set B_t: its pseudoinverse needs
  s >= |B_t| (Sec. 4.4), and the same oversampling p as the boxes' least-squares
  problems keeps Omega_Bt well conditioned (a square Gaussian block has a
  condition number in the 1e3..1e6 range, which turns sketch rounding into a
  large error in the root block).
"""
from __future__ import annotations

import numpy as np

LMAX = 20  # integer resolution of the binning: 2^20 cells per side


def _morton(coord: tuple[int, ...]) -> int:
    key = 0
    for bit in range(LMAX + 1):
        for dim, c in enumerate(coord):
            key |= ((c >> bit) & 1) << (bit * len(coord) + dim)
    return key


class Box:
    __slots__ = ("id", "level", "coord", "parent", "children", "pts", "first_pos")

    def __init__(self, bid, level, coord, parent, pts):
        self.id = bid
        self.level = level
        self.coord = coord
        self.parent = parent
        self.children = []
        self.pts = pts  # original indices, ascending
        self.first_pos = -1

    @property
    def is_leaf(self):
        return not self.children


class Tree:
    """Adaptive 2^d-tree over N points with leaf capacity ``leaf_cap``."""

    def __init__(self, points: np.ndarray, leaf_cap: int):
        points = np.asarray(points, dtype=np.float64)
        self.points = points
        self.n, self.d = points.shape
        self.leaf_cap = leaf_cap
        lo = points.min(axis=0)
        hi = points.max(axis=0)
        if lo.min() >= 0.0 and hi.max() <= 1.0:
            lo = np.zeros(self.d)
            side = 1.0
        else:
            side = float((hi - lo).max())
            if side <= 0.0:
                side = 1.0
        u = np.floor(((points - lo) / side) * float(1 << LMAX))
        self.icoord = np.clip(u, 0, (1 << LMAX) - 1).astype(np.int64)
        self.boxes: list[Box] = []
        root = self._new_box(0, (0,) * self.d, None, np.arange(self.n))
        stack = [root]
        while stack:
            b = stack.pop()
            if len(b.pts) > leaf_cap and b.level < LMAX:
                self._split(b)
                stack.extend(b.children)
        self._balance()
        self._finish()

    # -- construction -------------------------------------------------
    def _new_box(self, level, coord, parent, pts):
        b = Box(len(self.boxes), level, coord, parent, pts)
        self.boxes.append(b)
        return b

    def _split(self, b: Box):
        shift = LMAX - b.level - 1
        cc = self.icoord[b.pts] >> shift  # child-level coords
        child_idx = np.zeros(len(b.pts), dtype=np.int64)
        for dim in range(self.d):
            child_idx |= (cc[:, dim] - 2 * b.coord[dim]) << dim
        for c in range(1 << self.d):
            sel = b.pts[child_idx == c]
            if len(sel) == 0:
                continue
            coord = tuple(2 * b.coord[dim] + ((c >> dim) & 1) for dim in range(self.d))
            b.children.append(self._new_box(b.level + 1, coord, b, np.sort(sel)))

    @staticmethod
    def touches(a: Box, b: Box) -> bool:
        """Closed boxes a and b share at least a corner (and are distinct, not nested)."""
        L = max(a.level, b.level)
        sa, sb = L - a.level, L - b.level
        for dim in range(len(a.coord)):
            lo_a, hi_a = a.coord[dim] << sa, (a.coord[dim] + 1) << sa
            lo_b, hi_b = b.coord[dim] << sb, (b.coord[dim] + 1) << sb
            if lo_a > hi_b or lo_b > hi_a:
                return False
        return True

    @staticmethod
    def _extent(boxes):
        """Closed integer extents [lo, hi] of boxes at resolution 2^LMAX (len x d arrays)."""
        lv = np.array([b.level for b in boxes], dtype=np.int64)[:, None]
        c = np.array([b.coord for b in boxes], dtype=np.int64).reshape(len(boxes), -1)
        return c << (LMAX - lv), (c + 1) << (LMAX - lv)

    def _balance(self):
        changed = True
        while changed:
            changed = False
            leaves = [b for b in self.boxes if b.is_leaf]
            lo, hi = self._extent(leaves)
            lvl = np.array([b.level for b in leaves])
            to_split = []
            for i, a in enumerate(leaves):
                deep = lvl >= a.level + 2
                if not deep.any():
                    continue
                t = np.all((lo[deep] <= hi[i]) & (lo[i] <= hi[deep]), axis=1)
                if t.any():
                    to_split.append(a)
            for a in to_split:
                self._split(a)
                changed = True

    def _finish(self):
        # tree order: depth-first, children in Morton order, points ascending in a leaf
        order = []

        def dfs(b):
            b.first_pos = len(order)
            if b.is_leaf:
                order.extend(b.pts.tolist())
            for c in b.children:
                dfs(c)

        dfs(self.boxes[0])
        self.perm = np.array(order, dtype=np.int64)  # tree position -> original index
        self.pos = np.empty(self.n, dtype=np.int64)
        self.pos[self.perm] = np.arange(self.n)
        self.depth = max(b.level for b in self.boxes)
        self.levels = {}
        for b in self.boxes:
            self.levels.setdefault(b.level, []).append(b)
        for lv in self.levels.values():
            lv.sort(key=lambda b: _morton(b.coord))

    # -- per-level geometry --------------------------------------------
    def candidates(self, level: int) -> list[Box]:
        """Boxes that partition the active points at ``level``."""
        out = list(self.levels.get(level, []))
        out += [b for b in self.boxes if b.is_leaf and b.level < level]
        return out

    def neighbours(self, box: Box, cands: list[Box], ext=None) -> list[Box]:
        lo, hi = self._extent(cands) if ext is None else ext
        blo, bhi = self._extent([box])
        t = np.all((lo <= bhi[0]) & (blo[0] <= hi), axis=1)
        nb = [cands[i] for i in np.nonzero(t)[0] if cands[i] is not box]
        nb.sort(key=lambda c: c.first_pos)
        return nb


class Schedule:
    """Processing order and sizes of Algorithm 1 on a tree, for rank k and oversampling p.

    ``steps`` lists, level by level from the deepest to 1, the compressed boxes
    in processing order as dicts with keys: box, level, colour, nbrs, b, n, kp, r.
    """

    def __init__(self, tree: Tree, k: int, p: int | None = None):
        self.tree = tree
        self.k = k
        self.p = k if p is None else p
        act = {b.id: len(b.pts) for b in tree.boxes if b.is_leaf}
        self.steps = []
        self.n_colours = {}
        for level in range(tree.depth, 0, -1):
            boxes = tree.levels.get(level, [])
            for b in boxes:
                if not b.is_leaf:
                    act[b.id] = sum(act[c.id] for c in b.children)
            cands = tree.candidates(level)
            ext = tree._extent(cands)
            nbrs = {b.id: tree.neighbours(b, cands, ext) for b in boxes}
            comp = [b for b in boxes
                    if act[b.id] > k and len(cands) > 1 + len(nbrs[b.id])]
            # greedy colouring on the closed-neighbourhood conflict graph, Morton order
            members = {}
            for b in comp:
                for c in [b] + nbrs[b.id]:
                    members.setdefault(c.id, []).append(b.id)
            colour = {}
            for b in comp:  # already Morton-sorted
                used = set()
                for c in [b] + nbrs[b.id]:
                    for o in members[c.id]:
                        if o in colour:
                            used.add(colour[o])
                col = 0
                while col in used:
                    col += 1
                colour[b.id] = col
            ncol = max(colour.values()) + 1 if colour else 0
            self.n_colours[level] = ncol
            for col in range(ncol):
                for b in comp:
                    if colour[b.id] != col:
                        continue
                    bb = act[b.id]
                    n = sum(act[c.id] for c in nbrs[b.id])
                    kp = min(k, bb)
                    self.steps.append(dict(box=b, level=level, colour=col, nbrs=nbrs[b.id],
                                           b=bb, n=n, kp=kp, r=bb - kp))
                    act[b.id] = kp
        self.root_size = sum(act[b.id] for b in tree.levels[1]) if tree.depth >= 1 else tree.n
        if tree.depth == 0:
            self.root_size = tree.n
        self.max_l = max((st["b"] + st["n"] for st in self.steps), default=0)
        self.s_req = max(self.max_l + self.k + self.p if self.steps else 0, self.root_size + self.p)
