"""H^2-matrix representation (oracle; test infrastructure only).

Section 2, Def. "Cluster basis" and Eq. (nested): a nested cluster basis
stores V_t only for leaves and a transfer matrix E_t for every non-root
cluster, with V_t|_{t'} = V_{t'} E_{t'} for every son t' of t.  Ranks may
differ from cluster to cluster, so E_t is k_t x k_{t+}.

Section 2, Def. "H^2-matrix" and Eq. (vsw): every admissible leaf b = (t, s)
is G|_{t x s} = V_t S_b W_s^*; inadmissible leaves are stored densely.
All matrices are float64 numpy arrays indexed by cluster or block id; rows
of a cluster basis follow the tree order of the cluster's label.
"""
from __future__ import annotations

import copy

import numpy as np

from .tree import BlockTree, ClusterTree


class ClusterBasis:
    """Nested cluster basis: leaf matrices, transfer matrices, ranks."""

    def __init__(self, tree: ClusterTree):
        self.tree = tree
        self.rank = [0] * tree.n_clusters
        self.leaf = {}       # t -> (#t x k_t) for leaves
        self.transfer = {}   # t -> (k_t x k_{t+}) for non-root clusters

    def dense(self, t: int) -> np.ndarray:
        """V_t as an explicit #t x k_t matrix, expanded through Eq. (nested)."""
        if self.tree.is_leaf(t):
            return self.leaf[t]
        parts = [self.dense(s) @ self.transfer[s] for s in self.tree.sons[t]]
        return np.vstack(parts)

    @classmethod
    def from_canonical(cls, tree: ClusterTree, ranks, leaf_data, transfer_data):
        cb = cls(tree)
        cb.rank = [int(r) for r in ranks]
        pos = 0
        for t in range(tree.n_clusters):
            if tree.is_leaf(t):
                m, k = tree.size[t], cb.rank[t]
                cb.leaf[t] = np.array(leaf_data[pos:pos + m * k]).reshape((m, k), order="F")
                pos += m * k
        assert pos == len(leaf_data)
        pos = 0
        for t in range(1, tree.n_clusters):
            k, kf = cb.rank[t], cb.rank[tree.father[t]]
            cb.transfer[t] = np.array(transfer_data[pos:pos + k * kf]).reshape((k, kf), order="F")
            pos += k * kf
        assert pos == len(transfer_data)
        return cb

    def to_canonical(self):
        leaf = [self.leaf[t].ravel(order="F") for t in range(self.tree.n_clusters) if self.tree.is_leaf(t)]
        tr = [self.transfer[t].ravel(order="F") for t in range(1, self.tree.n_clusters)]
        cat = lambda xs: np.concatenate(xs) if xs else np.zeros(0)
        return np.array(self.rank, dtype=np.int32), cat(leaf), cat(tr)


class H2Matrix:
    """H^2-matrix: row basis V, column basis W, couplings S_b, nearfield."""

    def __init__(self, blocks: BlockTree, V: ClusterBasis, W: ClusterBasis):
        self.blocks = blocks
        self.V = V
        self.W = W
        self.S = {}      # admissible leaf b -> k_t x l_s
        self.N = {}      # inadmissible leaf b -> #t x #s

    def copy(self) -> "H2Matrix":
        other = H2Matrix(self.blocks, copy.deepcopy(self.V), copy.deepcopy(self.W))
        other.V.tree = self.V.tree
        other.W.tree = self.W.tree
        other.S = {b: s.copy() for b, s in self.S.items()}
        other.N = {b: n.copy() for b, n in self.N.items()}
        return other

    def set_couplings(self, data):
        pos = 0
        for b in self.blocks.admissible:
            k = self.V.rank[self.blocks.row[b]]
            l = self.W.rank[self.blocks.col[b]]
            self.S[b] = np.array(data[pos:pos + k * l]).reshape((k, l), order="F")
            pos += k * l
        assert pos == len(data)

    def set_nearfield(self, data):
        pos = 0
        for b in self.blocks.inadmissible:
            m = self.V.tree.size[self.blocks.row[b]]
            n = self.W.tree.size[self.blocks.col[b]]
            self.N[b] = np.array(data[pos:pos + m * n]).reshape((m, n), order="F")
            pos += m * n
        assert pos == len(data)

    def block_dense(self, b: int) -> np.ndarray:
        """Z|_{t x s} of any block-tree node, in tree order (Eq. (vsw))."""
        bt = self.blocks
        kind = bt.kind[b]
        if kind == BlockTree.ADM:
            return self.V.dense(bt.row[b]) @ self.S[b] @ self.W.dense(bt.col[b]).T
        if kind == BlockTree.NEAR:
            return self.N[b]
        t, s = bt.row[b], bt.col[b]
        out = np.zeros((self.V.tree.size[t], self.W.tree.size[s]))
        t_off, s_off = self.V.tree.offset[t], self.W.tree.offset[s]
        for c in bt.sons[b]:
            tc, sc = bt.row[c], bt.col[c]
            r0 = self.V.tree.offset[tc] - t_off
            c0 = self.W.tree.offset[sc] - s_off
            out[r0:r0 + self.V.tree.size[tc], c0:c0 + self.W.tree.size[sc]] = self.block_dense(c)
        return out

    def dense(self) -> np.ndarray:
        """The whole matrix in tree order (rows and columns permuted)."""
        return self.block_dense(0)
