"""Per-block parity of assembled H^2 matrices (test helper, no oracle code).

The tolerance of the GPU parity tests is stated per assembled block: for
every leaf b = (t, s) of the block tree,

    ||Z_gpu|_b - Z_ref|_b||_F <= tol * ||Z_ref|_b||_F,

so that an error confined to one block of small norm cannot hide behind the
norm of the whole matrix.  A block whose reference is exactly zero is
compared against the norm of the whole reference instead (there is no
relative scale to use).

Two forms:

* ``blockwise_dense``: both matrices given densely (tree order), every leaf
  block sliced out (small problems);
* ``blockwise_h2``: both given as H^2 containers; an admissible block is
  compared in compressed form: with orthonormal bases Q_V of [V1 V2] and
  Q_W of [W1 W2], ||V1 S1 W1^* - V2 S2 W2^*||_F equals the norm of the small
  matrix (Q_V^* V1) S1 (W1^* Q_W) - (Q_V^* V2) S2 (W2^* Q_W), formed without
  squaring (large problems, where the dense blocks would not fit).
"""
from __future__ import annotations

import numpy as np

from dense_ref import basis_dense


def leaf_blocks(bt):
    return sorted(list(bt.admissible) + list(bt.inadmissible))


def blockwise_dense(G: np.ndarray, R: np.ndarray, bt, rt, ct, blocks=None, floor=0.0):
    """Worst per-block relative error and the block where it occurs.
    ``floor`` (absolute) is added to every block's norm: blocks whose
    reference is at the rounding level of the whole matrix (structural
    zeros computed as +-1e-30) have no relative scale of their own."""
    total = float(np.linalg.norm(R))
    worst, where = 0.0, -1
    for b in (leaf_blocks(bt) if blocks is None else blocks):
        t, s = bt.row[b], bt.col[b]
        r0, c0 = rt.offset[t], ct.offset[s]
        gb = G[r0:r0 + rt.size[t], c0:c0 + ct.size[s]]
        rb = R[r0:r0 + rt.size[t], c0:c0 + ct.size[s]]
        den = float(np.linalg.norm(rb)) + floor
        if den == 0.0:
            den = total if total > 0 else 1.0
        e = float(np.linalg.norm(gb - rb)) / den
        if not (e <= worst):
            worst, where = e, b
    return worst, where


def assert_blockwise_dense(G, R, bt, rt, ct, tol, what="", floor=0.0):
    worst, where = blockwise_dense(G, R, bt, rt, ct, floor=floor)
    assert worst <= tol, ("per-block relative error", what, where, worst)
    return worst


class _BasisCache:
    def __init__(self, tree, basis):
        self.tree, self.basis, self.mem = tree, basis, {}

    def __call__(self, t):
        if t not in self.mem:
            self.mem[t] = basis_dense(self.tree, self.basis, t)
        return self.mem[t]


def blockwise_h2(got, ref, blocks):
    """Worst per-block relative error over the given leaf blocks of two H^2
    containers with the same block tree (bases may differ)."""
    bt = ref.blocks
    rt, ct = ref.V.tree, ref.W.tree
    gv, gw = _BasisCache(rt, got.V), _BasisCache(ct, got.W)
    rv, rw = _BasisCache(rt, ref.V), _BasisCache(ct, ref.W)
    worst, where = 0.0, -1
    for b in blocks:
        t, s = bt.row[b], bt.col[b]
        if bt.kind[b] == bt.NEAR:
            diff = float(np.linalg.norm(got.N[b] - ref.N[b]))
            den = float(np.linalg.norm(ref.N[b]))
        elif bt.kind[b] == bt.ADM:
            # orthonormal bases QV, QW of the stacked row and column bases;
            # the difference lives in range(QV) x range(QW), so its norm is
            # that of a small matrix, formed without squaring
            V1, V2, W1, W2 = gv(t), rv(t), gw(s), rw(s)
            QV = np.linalg.qr(np.hstack([V1, V2]))[0]
            QW = np.linalg.qr(np.hstack([W1, W2]))[0]
            M1 = (QV.T @ V1) @ got.S[b] @ (W1.T @ QW)
            M2 = (QV.T @ V2) @ ref.S[b] @ (W2.T @ QW)
            diff = float(np.linalg.norm(M1 - M2))
            den = float(np.linalg.norm(M2))
        else:
            raise ValueError("not a leaf block: %d" % b)
        if den == 0.0:
            den = 1.0
        e = diff / den
        if not (e <= worst):
            worst, where = e, b
    return worst, where
