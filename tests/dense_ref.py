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


def basis_row(tree, basis, leaf_of, i, t):
    """Row of V_t at tree position i (i inside t^), via Eq. (nested)."""
    c = leaf_of[i]
    row = basis.leaf[c][i - tree.offset[c]]
    while c != t:
        row = row @ basis.transfer[c]
        c = tree.father[c]
    return row


def leaf_index(tree):
    """leaf_of[i] = leaf cluster containing tree position i."""
    out = np.zeros(tree.n, dtype=np.int64)
    for c in range(tree.n_clusters):
        if not tree.sons[c]:
            out[tree.offset[c]:tree.offset[c] + tree.size[c]] = c
    return out


def entries(Z, I, J):
    """Entries Z[I[k], J[k]] (tree positions) of an H^2 matrix, one by one:
    descend the block tree to the leaf containing (i, j) and evaluate
    V_t S_b W_s^* there (Eq. (vsw)) or read the nearfield block."""
    bt = Z.blocks
    rt, ct = Z.V.tree, Z.W.tree
    lr, lc = leaf_index(rt), leaf_index(ct)
    out = np.zeros(len(I))
    for k, (i, j) in enumerate(zip(I, J)):
        b = 0
        while bt.kind[b] == bt.SUB:
            for c in bt.sons[b]:
                t, s = bt.row[c], bt.col[c]
                if rt.offset[t] <= i < rt.offset[t] + rt.size[t] and ct.offset[s] <= j < ct.offset[s] + ct.size[s]:
                    b = c
                    break
        t, s = bt.row[b], bt.col[b]
        if bt.kind[b] == bt.ADM:
            v = basis_row(rt, Z.V, lr, i, t)
            w = basis_row(ct, Z.W, lc, j, s)
            out[k] = v @ Z.S[b] @ w
        else:
            out[k] = Z.N[b][i - rt.offset[t], j - ct.offset[s]]
    return out
