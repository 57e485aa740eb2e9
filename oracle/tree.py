"""Cluster tree and block tree (oracle; test infrastructure only).

Section 2, Def. "Cluster tree": every node t carries a label t^ (an index
set); the labels of the sons partition the label of the father; the root is
labelled by the whole index set.  Section 2, Def. "Block tree": the root is
(root, root); a subdivided block (t, s) has the sons sons(t) x sons(s); its
leaves partition I x J and split into admissible leaves L+ and inadmissible
leaves L-.

Construction rules (the paper leaves them open; these readings are shared
with the library by specification only, never by code):

* geometric bisection: a cluster with more than ``leaf_size`` indices is
  split along the longest axis of the bounding box of its points (ties go to
  the lowest axis) at the midpoint; indices whose coordinate is below the
  midpoint go to the first son, the others to the second, keeping their
  order.  A split that would leave one son empty is not made;
* clusters are numbered in depth-first preorder, root 0;
* admissibility of (t, s): dist(t, s) > 0 and
  max(diam t, diam s) <= eta * dist(t, s), with the Euclidean diameter of
  the (optionally padded) bounding box and the Euclidean box-box distance;
* a block is subdivided while it is inadmissible and both clusters have
  sons; blocks are numbered in depth-first preorder with the sons ordered
  (t1,s1), (t1,s2), (t2,s1), (t2,s2).
"""
from __future__ import annotations

import math

import numpy as np


class ClusterTree:
    """Binary cluster tree by geometric bisection (Section 2)."""

    def __init__(self, points: np.ndarray, leaf_size: int, pad: float = 0.0):
        self.points = np.asarray(points, dtype=np.float64)
        self.n, self.dim = self.points.shape
        self.leaf_size = int(leaf_size)
        self.pad = float(pad)
        # per-cluster lists, indexed by cluster id (DFS preorder)
        self.idx = []        # original indices in the label, in tree order
        self.sons = []       # [] or [t1, t2]
        self.father = []     # -1 for the root
        self.level = []
        self.lo = []         # padded bounding box used for admissibility
        self.hi = []
        self._build(np.arange(self.n, dtype=np.int64), -1, 0)
        self.n_clusters = len(self.idx)
        # tree order of the indices = concatenation of leaf labels in DFS order
        self.perm = np.concatenate([self.idx[t] for t in range(self.n_clusters) if not self.sons[t]])
        pos = np.empty(self.n, dtype=np.int64)
        pos[self.perm] = np.arange(self.n)
        # a label is a contiguous range of the tree order; its offset is the
        # smallest tree position of its indices
        self.offset = [int(pos[self.idx[t]].min()) if len(self.idx[t]) else 0 for t in range(self.n_clusters)]
        self.size = [len(self.idx[t]) for t in range(self.n_clusters)]
        # number of clusters in the subtree rooted at t (#T_t)
        self.subtree_count = [0] * self.n_clusters
        for t in reversed(range(self.n_clusters)):
            self.subtree_count[t] = 1 + sum(self.subtree_count[s] for s in self.sons[t])

    def _build(self, idx: np.ndarray, father: int, level: int) -> int:
        t = len(self.idx)
        pts = self.points[idx]
        lo = pts.min(axis=0)
        hi = pts.max(axis=0)
        self.idx.append(idx)
        self.sons.append([])
        self.father.append(father)
        self.level.append(level)
        self.lo.append(lo - self.pad)
        self.hi.append(hi + self.pad)
        if len(idx) > self.leaf_size:
            ext = hi - lo
            axis = 0
            for a in range(self.dim):
                if ext[a] > ext[axis]:
                    axis = a
            mid = 0.5 * (lo[axis] + hi[axis])
            first = idx[pts[:, axis] < mid]
            second = idx[~(pts[:, axis] < mid)]
            if len(first) > 0 and len(second) > 0:
                t1 = self._build(first, t, level + 1)
                t2 = self._build(second, t, level + 1)
                self.sons[t] = [t1, t2]
        return t

    def is_leaf(self, t: int) -> bool:
        return not self.sons[t]

    def descendants(self, t: int) -> list:
        """All clusters of the subtree T_t (t included), DFS preorder."""
        out = [t]
        for s in self.sons[t]:
            out += self.descendants(s)
        return out

    def predecessors(self, t: int) -> list:
        """pred(t) of Section 4, ordered from the root down to t."""
        path = []
        while t >= 0:
            path.append(t)
            t = self.father[t]
        return path[::-1]

    def diam(self, t: int) -> float:
        return math.sqrt(float(np.sum((self.hi[t] - self.lo[t]) ** 2)))

    def dist_to(self, other: "ClusterTree", t: int, s: int) -> float:
        """Euclidean distance between the box of t (here) and of s (in other)."""
        gap = np.maximum(0.0, np.maximum(other.lo[s] - self.hi[t], self.lo[t] - other.hi[s]))
        return math.sqrt(float(np.sum(gap ** 2)))


class BlockTree:
    """Block tree T_{I x J} with admissible / inadmissible leaves (Section 2)."""

    ADM, NEAR, SUB = 1, 2, 0

    def __init__(self, rows: ClusterTree, cols: ClusterTree, eta: float):
        self.rows = rows
        self.cols = cols
        self.eta = float(eta)
        self.row = []     # row cluster of each block
        self.col = []     # column cluster
        self.kind = []    # SUB / ADM / NEAR
        self.sons = []
        self.father = []
        self._build(0, 0, -1)
        self.n_blocks = len(self.row)
        self.admissible = [b for b in range(self.n_blocks) if self.kind[b] == self.ADM]
        self.inadmissible = [b for b in range(self.n_blocks) if self.kind[b] == self.NEAR]
        # row(t) and the column analogue col(s): admissible leaves by cluster
        self.row_blocks = [[] for _ in range(rows.n_clusters)]
        self.col_blocks = [[] for _ in range(cols.n_clusters)]
        for b in self.admissible:
            self.row_blocks[self.row[b]].append(b)
            self.col_blocks[self.col[b]].append(b)

    def admissible_pair(self, t: int, s: int) -> bool:
        d = self.rows.dist_to(self.cols, t, s)
        return d > 0.0 and max(self.rows.diam(t), self.cols.diam(s)) <= self.eta * d

    def _build(self, t: int, s: int, father: int) -> int:
        b = len(self.row)
        self.row.append(t)
        self.col.append(s)
        self.sons.append([])
        self.father.append(father)
        if self.admissible_pair(t, s):
            self.kind.append(self.ADM)
        elif self.rows.is_leaf(t) or self.cols.is_leaf(s):
            self.kind.append(self.NEAR)
        else:
            self.kind.append(self.SUB)
            for t1 in self.rows.sons[t]:
                for s1 in self.cols.sons[s]:
                    self.sons[b].append(self._build(t1, s1, b))
        return b

    def descendants(self, b: int) -> list:
        out = [b]
        for c in self.sons[b]:
            out += self.descendants(c)
        return out

