"""Dense restatements used as pins (test helper, no oracle code).

Everything here works on explicit dense matrices built straight from the
definitions of Section 2, so that the oracle's structured recursions can be
checked against them on small problems.
"""
from __future__ import annotations

import math

import numpy as np


def basis_dense(tree, basis, t):
    """V_t from Eq. (nested) written as a product along each leaf-to-t path:
    rows of a leaf l below t are V_l E_l E_{l+} ... E_{t'} (t' the son of t)."""
    out = np.zeros((tree.size[t], basis.rank[t]))
    stack = [t]
    while stack:
        c = stack.pop()
        if tree.sons[c]:
            stack.extend(tree.sons[c])
            continue
        M = basis.leaf[c]
        x = c
        while x != t:
            M = M @ basis.transfer[x]
            x = tree.father[x]
        r0 = tree.offset[c] - tree.offset[t]
        out[r0:r0 + tree.size[c]] = M
    return out


def block(D, tree_r, tree_c, t, s):
    r0, c0 = tree_r.offset[t], tree_c.offset[s]
    return D[r0:r0 + tree_r.size[t], c0:c0 + tree_c.size[s]]


def weighted_block_row(Zt, Z, t, row_side=True):
    """Z~_t of Section 4 with block-relative weights, as a dense matrix.

    Row side: [omega_b Z~|_{t x s} for every admissible b = (t*, s) with
    t* in pred(t)], omega_b = sqrt(#T_{t*}) / ||Z~|_{t* x s}||_F.  Column side:
    the same for Z~^* with the column tree.
    """
    bt = Z.blocks
    rt, ctr = Z.V.tree, Z.W.tree
    tree = rt if row_side else ctr
    lists = bt.row_blocks if row_side else bt.col_blocks
    cols = []
    x = t
    while x >= 0:
        for b in lists[x]:
            tb, sb = bt.row[b], bt.col[b]
            full = block(Zt, rt, ctr, tb, sb)
            nrm = np.linalg.norm(full)
            om = math.sqrt(tree.subtree_count[x]) / nrm if nrm > 0 else 0.0
            if row_side:
                r0 = rt.offset[t] - rt.offset[tb]
                cols.append(om * full[r0:r0 + rt.size[t], :])
            else:
                c0 = ctr.offset[t] - ctr.offset[sb]
                cols.append(om * full[:, c0:c0 + ctr.size[t]].T)
        x = tree.father[x]
    if not cols:
        return np.zeros((tree.size[t], 0))
    return np.hstack(cols)
