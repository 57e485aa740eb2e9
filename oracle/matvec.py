"""H^2-matrix times a block of vectors (oracle; test infrastructure only).

Y <- alpha Z X + beta Y with the rows of X and Y in tree order and one
right-hand side per column.  Z is the sum over the admissible leaves
b = (t, s) of V_t S_b W_s^* (Section 2, Eq. (vsw)) and the dense
inadmissible leaves.  Because the bases are nested (Section 2, Eq.
(nested)), the products with W_s^* and with V_t are formed once per
cluster:

1. forward transformation, sons before fathers: xh_s = W_s^* X|_s for a
   leaf, xh_s = sum over the sons s' of E_{s'}^* xh_{s'} above;
2. coupling: yh_t = sum over the admissible leaves b = (t, s) of S_b xh_s;
3. backward transformation, fathers before sons: yh_{t'} += E_{t'} yh_t
   for every son t' of t, and Y|_t += V_t yh_t at the leaves;
4. nearfield: Y|_t += N_b X|_s for the inadmissible leaves b = (t, s).

The multiplication (Section 3) uses this product where one factor block is
a leaf: X|_{t x s} V_s is formed by k such products (Section 6, Case 2).
Plain numpy, cluster by cluster; it shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np

from .h2 import H2Matrix


def matvec(Z: H2Matrix, X, alpha: float = 1.0, beta: float = 0.0, Y=None) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    V, W, bt = Z.V, Z.W, Z.blocks
    rt, ct = V.tree, W.tree
    nrhs = X.shape[1]
    # 1. forward transformation (a son's id is larger than its father's)
    xh = {}
    for s in reversed(range(ct.n_clusters)):
        if ct.is_leaf(s):
            o, m = ct.offset[s], ct.size[s]
            xh[s] = W.leaf[s].T @ X[o:o + m]
        else:
            acc = np.zeros((W.rank[s], nrhs))
            for c in ct.sons[s]:
                acc = acc + W.transfer[c].T @ xh[c]
            xh[s] = acc
    # 2. coupling
    yh = {t: np.zeros((V.rank[t], nrhs)) for t in range(rt.n_clusters)}
    for b in bt.admissible:
        yh[bt.row[b]] = yh[bt.row[b]] + Z.S[b] @ xh[bt.col[b]]
    # 3. backward transformation (fathers first) and the leaves' rows
    out = np.zeros((rt.size[0], nrhs))
    for t in range(rt.n_clusters):
        for c in rt.sons[t]:
            yh[c] = yh[c] + V.transfer[c] @ yh[t]
        if rt.is_leaf(t):
            o, m = rt.offset[t], rt.size[t]
            out[o:o + m] += V.leaf[t] @ yh[t]
    # 4. nearfield
    for b in bt.inadmissible:
        t, s = bt.row[b], bt.col[b]
        out[rt.offset[t]:rt.offset[t] + rt.size[t]] += Z.N[b] @ X[ct.offset[s]:ct.offset[s] + ct.size[s]]
    res = alpha * out
    if beta != 0.0:
        Yv = np.asarray(Y, dtype=np.float64)
        res = res + beta * (Yv[:, None] if Yv.ndim == 1 else Yv)
    return res[:, 0] if vec else res
