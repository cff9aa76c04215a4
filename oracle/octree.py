"""Octree clusters over RWG edge midpoints, admissibility and the block tree
(Sec. II, Eq. 10 and Eq. 13: Z = Z_N + Z_F, near-field at leaf level, far
field at all levels).

Readings (the paper uses a binary tree with leaves >= 0.5 lambda and leaves
eta of Eq. 10 open):
  * root = bounding cube of the midpoints (centre of the bounding box, side =
    largest extent); a node splits into 8 while it holds more than leaf_max
    unknowns (and is shallower than MAX_DEPTH); a point goes to the upper half
    of an axis when its coordinate is >= the node centre; children are visited
    in Morton order (index bx + 2 by + 4 bz); empty children are dropped;
  * unknowns inside a leaf keep ascending original index; leaves are numbered
    in depth-first order, which is also the elimination order;
  * admissible = the two cells do not touch (no shared face, edge or vertex),
    tested exactly on integer cell coordinates; this yields the 26-neighbour
    near field the complexity analysis assumes (Sec. IV);
  * with a constant eta > 0, Eq. 10 in the paper's form on top of that:
    admissible when the cells do not touch and min(diam) <= eta dist, diam
    the cell diagonal (sqrt 3 edge) and dist the distance between the two
    cubes, evaluated exactly on the integer cell coordinates as
    3 min(edge)^2 <= eta^2 sum(gap^2) (so ties, e.g. a one-cell diagonal gap
    at eta = 1, are far);
  * block recursion from (root, root): admissible -> far; two leaves -> near;
    otherwise split the non-leaf side(s).

Pinned by: near + far blocks tile the N x N index square exactly once;
admissible cells are geometrically separated; every near pair touches.
"""
from dataclasses import dataclass, field

import numpy as np

MAX_DEPTH = 21


@dataclass
class Node:
    level: int
    ijk: tuple
    start: int                 # first position in leaf (permuted) order
    count: int
    children: list = field(default_factory=list)
    leaf: int = -1             # leaf number, -1 for inner nodes


class Octree:
    def __init__(self, points, leaf_max, eta=0.0):
        pts = np.asarray(points, dtype=np.float64)
        self.leaf_max = int(leaf_max)
        self.eta = float(eta or 0.0)
        lo = pts.min(axis=0)
        hi = pts.max(axis=0)
        centre = (lo + hi) / 2.0
        half = float((hi - lo).max()) / 2.0
        if half == 0.0:
            half = 1.0
        self.origin = centre - half
        self.size = 2.0 * half
        self.pts = pts
        self.nodes = []
        self.perm = []
        self.leaves = []       # node ids of leaves in depth-first order
        self._build(list(range(len(pts))), 0, (0, 0, 0))
        self.perm = np.array(self.perm, dtype=np.int64)
        self.leaf_off = np.array([self.nodes[n].start for n in self.leaves] +
                                 [len(pts)], dtype=np.int64)

    def _build(self, idx, level, ijk):
        nid = len(self.nodes)
        node = Node(level, ijk, len(self.perm), len(idx))
        self.nodes.append(node)
        if len(idx) <= self.leaf_max or level >= MAX_DEPTH:
            node.leaf = len(self.leaves)
            self.leaves.append(nid)
            self.perm.extend(idx)
            return nid
        cell = self.size / (2 ** level)
        centre = [self.origin[a] + (ijk[a] + 0.5) * cell for a in range(3)]
        buckets = [[] for _ in range(8)]
        for i in idx:
            p = self.pts[i]
            c = ((1 if p[0] >= centre[0] else 0) |
                 (2 if p[1] >= centre[1] else 0) |
                 (4 if p[2] >= centre[2] else 0))
            buckets[c].append(i)
        for c in range(8):
            if buckets[c]:
                cijk = (2 * ijk[0] + (c & 1), 2 * ijk[1] + ((c >> 1) & 1),
                        2 * ijk[2] + ((c >> 2) & 1))
                node.children.append(self._build(buckets[c], level + 1, cijk))
        return nid

    @property
    def n_leaves(self):
        return len(self.leaves)

    def touching(self, s, t):
        """Cells of nodes s and t share at least a vertex (exact integers)."""
        a, b = self.nodes[s], self.nodes[t]
        sa = 1 << (MAX_DEPTH - a.level)
        sb = 1 << (MAX_DEPTH - b.level)
        for ax in range(3):
            lo_a, hi_a = a.ijk[ax] * sa, (a.ijk[ax] + 1) * sa
            lo_b, hi_b = b.ijk[ax] * sb, (b.ijk[ax] + 1) * sb
            if lo_a > hi_b or lo_b > hi_a:
                return False
        return True

    def near_pair(self, s, t):
        """Not admissible: the cells touch or, for eta > 0, fail
        min(diam) <= eta dist (Eq. 10), on exact integer coordinates."""
        if self.touching(s, t):
            return True
        if self.eta <= 0.0:
            return False
        a, b = self.nodes[s], self.nodes[t]
        sa = 1 << (MAX_DEPTH - a.level)
        sb = 1 << (MAX_DEPTH - b.level)
        D = 0
        for ax in range(3):
            lo_a, hi_a = a.ijk[ax] * sa, (a.ijk[ax] + 1) * sa
            lo_b, hi_b = b.ijk[ax] * sb, (b.ijk[ax] + 1) * sb
            g = max(0, lo_b - hi_a, lo_a - hi_b)
            D += g * g
        m = float(min(sa, sb))
        return not (3.0 * m * m <= (self.eta * self.eta) * float(D))

    def blocks(self):
        """Return (near, far): near = list of (leaf_i, leaf_j) over all ordered
        pairs; far = list of (node_s, node_t) over all ordered pairs."""
        near, far = [], []
        stack = [(0, 0)]
        while stack:
            s, t = stack.pop()
            if not self.near_pair(s, t):
                far.append((s, t))
                continue
            ns, nt = self.nodes[s], self.nodes[t]
            if ns.leaf >= 0 and nt.leaf >= 0:
                near.append((ns.leaf, nt.leaf))
            elif ns.leaf >= 0:
                stack.extend((s, c) for c in reversed(nt.children))
            elif nt.leaf >= 0:
                stack.extend((c, t) for c in reversed(ns.children))
            else:
                stack.extend((cs, ct) for cs in reversed(ns.children)
                             for ct in reversed(nt.children))
        return near, far

    def upper_blocks(self):
        """Near pairs with i <= j and far pairs whose row cluster starts before
        the column cluster, each sorted; the other half is the transpose."""
        near, far = self.blocks()
        near_u = sorted({(i, j) for (i, j) in near if i <= j})
        far_u = sorted((s, t) for (s, t) in far
                       if self.nodes[s].start < self.nodes[t].start)
        far_u.sort(key=lambda st: (self.nodes[st[0]].start, self.nodes[st[1]].start,
                                   self.nodes[st[0]].count, self.nodes[st[1]].count))
        return near_u, far_u
