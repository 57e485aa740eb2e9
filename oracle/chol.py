"""Approximate Cholesky factorisation A ~ L L^* of a symmetric positive
definite H^2 matrix (oracle; test infrastructure only, imported by tests/,
__graft_entry__.smoke() and bench.py's oracle timings alone).

The paper's experiments (Section 7) precondition with an approximate
Cholesky factorisation built by the algorithms of Section 3: the block
recursion of the LR factorisation, with the lower factor's transpose in
place of the upper factor, every low-rank term added through the local
update of Section 5.  Readings (the paper gives the LR recursion in full
and says only that Cholesky is built the same way):

1. On a diagonal block d = (t, t) with sons t1, t2:
   L11 = chol(A11); L21 = A21 L11^-* ; A22 <- A22 - L21 L21^* ;
   L22 = chol(A22).  The factor is the lower triangle of the matrix;
   the strictly upper nearfield is never read.  A term X|_x (X|_x)^* whose
   x is a leaf reaches a subdivided diagonal target whole: it is added to
   the block, both triangles, by one local update, so the strictly upper
   admissible blocks hold the transposed counterparts of such terms (and
   the shared cluster bases carry them).
2. A leaf: dense Cholesky of its lower triangle (positive diagonal), its
   strictly upper part set to zero.
3. L21 = A21 L11^-* block by block: X [L11 0; L21 L22]^* = [Y1 Y2] gives
   X1 = Y1 L11^-*, Y2 <- Y2 - X1 L21^*, X2 = Y2 L22^-* (recursion over the
   sons of the column cluster, row sons in order).  An admissible leaf
   X = V_t S W_s^* becomes V_t (L^-1 W_s S^*)^*: S set to zero and the
   factor pair (V_t, L^-1 W_s S^*) added by one local update.  A block
   whose basis on either side has rank 0 is zero and stays zero.
4. The product Z|_z += alpha X|_x (X|_y)^* with the second factor read
   transposed: the transpose of an admissible block V_r S W_s^* is
   W_s S^* V_r^*, of a dense leaf its transpose, of a subdivided block the
   transposes of its sons.  The recursion over the sons, the terms from
   the matrix at the start of the product, their grouping per target,
   the temporaries and the dense factor pairs are those of the LR's
   product (readings 1 to 3 of ``oracle.lr``).  For a diagonal target only
   the son blocks on or below the diagonal are computed.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from .lr import _apply_update, _compress, _Ctx, _factor_pair, _place, _son
from .tree import BlockTree


def chol_dense(M: np.ndarray) -> np.ndarray:
    """Lower triangular L with L L^* = M (the lower triangle of M is read),
    column by column; the strictly upper part of the result is zero."""
    A = np.tril(np.array(M, dtype=np.float64))
    n = A.shape[0]
    for k in range(n):
        d = A[k, k] - A[k, :k] @ A[k, :k]
        if not d > 0.0:
            raise ValueError("matrix not positive definite")
        A[k, k] = np.sqrt(d)
        A[k + 1:, k] = (A[k + 1:, k] - A[k + 1:, :k] @ A[k, :k]) / A[k, k]
    return A


# ------------------------------------------- dense solves with the factor
def lsolve_n(Z, d, Y):
    """X with L|_{t x t} X = Y (lower with its diagonal; d = (t, t))."""
    bt = Z.blocks
    if bt.kind[d] == BlockTree.NEAR:
        return solve_triangular(Z.N[d], Y, lower=True)
    tree = Z.V.tree
    t = bt.row[d]
    t1, t2 = tree.sons[t]
    n1 = tree.size[t1]
    X1 = lsolve_n(Z, _son(bt, d, t1, t1), Y[:n1])
    Y2 = Y[n1:] - Z.block_dense(_son(bt, d, t2, t1)) @ X1
    X2 = lsolve_n(Z, _son(bt, d, t2, t2), Y2)
    return np.vstack([X1, X2])


def ltsolve(Z, d, Y):
    """X with L|_{t x t}^* X = Y."""
    bt = Z.blocks
    if bt.kind[d] == BlockTree.NEAR:
        return solve_triangular(Z.N[d], Y, lower=True, trans="T")
    tree = Z.V.tree
    t = bt.row[d]
    t1, t2 = tree.sons[t]
    n1 = tree.size[t1]
    X2 = ltsolve(Z, _son(bt, d, t2, t2), Y[n1:])
    Y1 = Y[:n1] - Z.block_dense(_son(bt, d, t2, t1)).T @ X2
    X1 = ltsolve(Z, _son(bt, d, t1, t1), Y1)
    return np.vstack([X1, X2])


# ------------------------------ product with the second factor transposed
def _case2_t(Z, alpha, x, yh):
    """Term alpha X|_x (Z|_yh)^* when x or yh is a leaf: x = (t, s),
    yh = (r, s), the product (t, r)."""
    bt = Z.blocks
    t, s, r = bt.row[x], bt.col[x], bt.row[yh]
    if bt.kind[yh] == BlockTree.ADM:
        # (Z|_yh)^* = W_s S^* V_r^*
        Xt = Z.block_dense(x) @ Z.W.dense(s)
        return ("lr", alpha * (Xt @ Z.S[yh].T), Z.V.dense(r))
    if bt.kind[x] == BlockTree.ADM:
        # V_t S_x W_s^* (Z|_yh)^* = V_t (Z|_yh W_s S_x^*)^*
        Yt = Z.block_dense(yh) @ Z.W.dense(s)
        return ("lr", Z.V.dense(t), alpha * (Yt @ Z.S[x].T))
    X, Yh = Z.block_dense(x), Z.block_dense(yh)
    return ("dense", alpha * (X @ Yh.T), alpha * X, Yh)


def _skip(bt, tree, z, t1, r1, lower):
    """A son (t1, r1) of a diagonal target strictly above the diagonal."""
    return lower and bt.row[z] == bt.col[z] and tree.offset[t1] < tree.offset[r1]


def _collect_t(Z, alpha, x, yh, z, out, lower):
    bt = Z.blocks
    if bt.kind[x] == BlockTree.SUB and bt.kind[yh] == BlockTree.SUB:
        t, s, r = bt.row[x], bt.col[x], bt.row[yh]
        tree = Z.V.tree
        if bt.kind[z] == BlockTree.SUB:
            for s1 in tree.sons[s]:
                for t1 in tree.sons[t]:
                    for r1 in tree.sons[r]:
                        if _skip(bt, tree, z, t1, r1, lower):
                            continue
                        _collect_t(Z, alpha, _son(bt, x, t1, s1), _son(bt, yh, r1, s1), _son(bt, z, t1, r1),
                                   out, lower)
            return
        assert bt.kind[z] == BlockTree.ADM, "inadmissible target of subdivided factors"
        temps = {}
        for s1 in tree.sons[s]:
            for t1 in tree.sons[t]:
                for r1 in tree.sons[r]:
                    _collect_virtual_t(Z, alpha, _son(bt, x, t1, s1), _son(bt, yh, r1, s1),
                                       temps.setdefault((t1, r1), []))
        for t1 in tree.sons[t]:
            for r1 in tree.sons[r]:
                out.append(("temp", z, temps.get((t1, r1), [])))
        return
    out.append(("term", z, (bt.row[x], bt.row[yh]), _case2_t(Z, alpha, x, yh)))


def _collect_virtual_t(Z, alpha, x, yh, bucket):
    bt = Z.blocks
    if bt.kind[x] == BlockTree.SUB and bt.kind[yh] == BlockTree.SUB:
        t, s, r = bt.row[x], bt.col[x], bt.row[yh]
        tree = Z.V.tree
        for s1 in tree.sons[s]:
            for t1 in tree.sons[t]:
                for r1 in tree.sons[r]:
                    _collect_virtual_t(Z, alpha, _son(bt, x, t1, s1), _son(bt, yh, r1, s1), bucket)
        return
    bucket.append(((bt.row[x], bt.row[yh]), _case2_t(Z, alpha, x, yh)))


def _pair(term):
    if term[0] == "lr":
        return term[1], term[2]
    return _factor_pair(term[1], term[2], term[3])


def _mul_t(C: _Ctx, alpha, x, yh, z, lower):
    """Z|_z += alpha Z|_x (Z|_yh)^* (reading 4); terms from the matrix at
    the start, grouped per target that is not an inadmissible leaf."""
    Z = C.Z
    bt = Z.blocks
    out = []
    _collect_t(Z, alpha, x, yh, z, out, lower)
    groups = {}
    for item in out:
        if item[0] == "term" and bt.kind[item[1]] != BlockTree.NEAR:
            groups.setdefault(item[1], []).append(item[3])
    for item in out:
        if item[0] == "term":
            z1, term = item[1], item[3]
            if bt.kind[z1] == BlockTree.NEAR:
                if term[0] == "lr":
                    Z.N[z1] = Z.N[z1] + term[1] @ term[2].T
                else:
                    Z.N[z1] = Z.N[z1] + term[1]
                continue
            terms = groups.pop(z1, None)
            if terms is None:
                continue
            pairs = [_pair(tm) for tm in terms]
            _apply_update(C, z1, np.hstack([a for a, _ in pairs]), np.hstack([b_ for _, b_ in pairs]))
        else:
            z1, bucket = item[1], item[2]
            if not bucket:
                continue
            As, Bs = [], []
            for cl, term in bucket:
                A, B = _place(Z, z1, cl, *_pair(term))
                As.append(A)
                Bs.append(B)
            A, B = _compress(np.hstack(As), np.hstack(Bs), C.eps)
            _apply_update(C, z1, A, B)


# ------------------------------------------------------- the factorisation
def _chol_rsolve(C: _Ctx, d, x):
    """Z|_x <- Z|_x L|_{s x s}^-* in place, x = (t, s), d = (s, s)."""
    Z = C.Z
    bt = Z.blocks
    if bt.kind[x] == BlockTree.NEAR:
        Z.N[x] = lsolve_n(Z, d, Z.N[x].T).T
        return
    t, s = bt.row[x], bt.col[x]
    if bt.kind[x] == BlockTree.ADM:
        if Z.S[x].size == 0:          # a rank-0 basis: the block is zero
            return
        Bh = lsolve_n(Z, d, Z.W.dense(s) @ Z.S[x].T)      # L^-1 W_s S^*
        Vt = Z.V.dense(t)
        Z.S[x] = np.zeros_like(Z.S[x])
        _apply_update(C, x, Vt, Bh)
        return
    tree = Z.V.tree
    s1, s2 = tree.sons[s]
    for t1 in tree.sons[t]:
        _chol_rsolve(C, _son(bt, d, s1, s1), _son(bt, x, t1, s1))
    for t1 in tree.sons[t]:
        _mul_t(C, -1.0, _son(bt, x, t1, s1), _son(bt, d, s2, s1), _son(bt, x, t1, s2), lower=False)
    for t1 in tree.sons[t]:
        _chol_rsolve(C, _son(bt, d, s2, s2), _son(bt, x, t1, s2))


def _chol(C: _Ctx, d):
    Z = C.Z
    bt = Z.blocks
    if bt.kind[d] == BlockTree.NEAR:
        Z.N[d] = chol_dense(Z.N[d])
        return
    tree = Z.V.tree
    t = bt.row[d]
    t1, t2 = tree.sons[t]
    d11, d21, d22 = _son(bt, d, t1, t1), _son(bt, d, t2, t1), _son(bt, d, t2, t2)
    _chol(C, d11)
    _chol_rsolve(C, d11, d21)
    _mul_t(C, -1.0, d21, d21, d22, lower=True)
    _chol(C, d22)


def chol_factor(Z, eps: float, cap=32, rank_cap=None):
    """Factorise the symmetric positive definite H^2 matrix Z (one tree for
    rows and columns) in place: on return its lower triangle holds L with
    A ~ L L^*.  Returns statistics."""
    C = _Ctx(Z, eps, cap, rank_cap)
    _chol(C, 0)
    return {"updates": C.updates, "max_rank": C.max_rank}


def lower(Z) -> np.ndarray:
    """The factor L of a Cholesky-factorised matrix as a dense array (tree
    order): the lower triangle of the assembled matrix."""
    return np.tril(Z.dense())


def chol_solve(Z, b):
    """x with L L^* x = b (tree order; b a vector or n x m)."""
    b = np.asarray(b, dtype=np.float64)
    B = b.reshape(b.shape[0], -1)
    X = ltsolve(Z, 0, lsolve_n(Z, 0, B))
    return X.reshape(b.shape)
