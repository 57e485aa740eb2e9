"""H^2-LR factorisation, block substitutions and the H^2 product (oracle;
test infrastructure only).

Section 3 of the paper, step by step, on ONE H^2 matrix that holds A on
entry and L (strictly lower part, unit diagonal implied) and R (upper part
with the diagonal) on exit, all blocks sharing the row basis V and the
column basis W of that matrix (the factorisation is done in place).

* lr(t): a leaf (t, t) is factorised by Gaussian elimination without
  pivoting (Doolittle); otherwise, with sons t1, t2: lr(t1); solve
  L11 R12 = A12 (forward substitution); solve L21 R11 = A21; A22 <- A22 -
  L21 R12 (the product); lr(t2).
* forward substitution L X = Y splits X, Y by the sons of t: X1 from
  L11 X1 = Y1, then L22 X2 = Y2 - L21 X1; X R = Y likewise by the sons of
  the column cluster.
* the product Z|_{t x r} += alpha X|_{t x s} Y|_{s x r}: the eight
  sub-products when X and Y are subdivided (Case 1 of Section 6); a
  low-rank term when X or Y is an admissible leaf, X V_s S W_r^* or
  V_t S (Y^* W_s)^* (Case 2); a dense term when both are inadmissible.
  Low-rank terms enter the H^2 matrix through the local low-rank update of
  Section 5 (``oracle.update``), dense terms are added to inadmissible
  leaves.

Readings of what the paper leaves open (also listed in the design notes):

1. A product's terms are all computed from the matrix as it is when the
   product starts, then added in the order the recursion produces them (X
   and Y share bases with Z here, so an update of Z would otherwise change
   the representation of later factors within the product).  The terms
   for one target block that is not an inadmissible leaf are added
   together: their factor pairs, in the recursion's order, form one factor
   pair, added by one local update where the block's first term stands.
2. Target (t, r) an admissible leaf while X and Y are subdivided: the
   sub-products go to temporaries (t', r'), t' in sons(t), r' in sons(r)
   (deeper sub-products are summed into their temporary exactly); each
   temporary is one factor pair, truncated by SVD to the smallest rank with
   sum_{i>r} sigma_i^2 <= (eps/2)^2 sum_i sigma_i^2, extended by zeros to
   t x r and added by one local update: at most four updates.
3. A dense term P for a target that is not an inadmissible leaf is written
   as a factor pair through its smallest dimension (X, Y^* when the inner
   cluster is the smallest, else (P, I) or (I, P^*)).
4. Forward substitution on an admissible leaf Y = V_t S W_s^*: X =
   (L^-1 V_t S) W_s^*, stored by setting S to zero and adding
   (L^-1 V_t S) W_s^* with a local update; X R = Y likewise with
   V_t (R^-* W_s S^*)^*.  A block whose basis has rank 0 on either side is
   zero; it stays zero and takes no update.
5. An update of rank u is applied in consecutive column groups of at most
   u_max columns (u_max = 32 minus the largest rank among the clusters of
   both subtrees, at least 1 and at most 31), each group one local update;
   with u_max = None the update is applied whole.
6. The approximate inverse (Remark on inversion) is built in a second H^2
   matrix C with the same trees, starting from zero (every rank 0); the
   blocks B12 = A11^-1 A12 and B21 = A21 A11^-1 go to a third zero matrix
   T, the Schur complement S = A22 - A21 B12 overwrites A22 (A is consumed),
   and the six products run in the order of the Remark, each one product
   of Section 3.  A leaf is inverted by Doolittle's LU and two triangular
   solves with the identity.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from .tree import BlockTree
from .update import apply_delta, local_update


class _Ctx:
    def __init__(self, Z, eps, cap, rank_cap=None):
        self.Z = Z
        self.eps = float(eps)
        self.rank_cap = rank_cap
        self.cap = cap
        self.updates = 0
        self.max_rank = 0


# ---------------------------------------------------------------- helpers
def _son(bt, b, t, s):
    """The son of block b with row cluster t and column cluster s."""
    for c in bt.sons[b]:
        if bt.row[c] == t and bt.col[c] == s:
            return c
    raise KeyError((b, t, s))


def lu_doolittle(M: np.ndarray) -> np.ndarray:
    """L (unit lower, strictly below the diagonal) and R (upper with the
    diagonal) of M = L R, in one array; Gaussian elimination without
    pivoting."""
    A = np.array(M, dtype=np.float64)
    n = A.shape[0]
    for k in range(n):
        if A[k, k] == 0.0:
            raise ZeroDivisionError("zero pivot")
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A


def _apply_update(C: _Ctx, b: int, A: np.ndarray, B: np.ndarray):
    """Z|_b <- trunc_eps(Z|_b + A B^*), in column groups (reading 5)."""
    Z = C.Z
    u = A.shape[1]
    if u == 0:
        return
    bt = Z.blocks
    j = 0
    while j < u:
        if C.cap is None:
            w = u
        else:
            kmax = 0
            for t in Z.V.tree.descendants(bt.row[b]):
                kmax = max(kmax, Z.V.rank[t])
            for s in Z.W.tree.descendants(bt.col[b]):
                kmax = max(kmax, Z.W.rank[s])
            w = max(1, min(C.cap - 1, C.cap - kmax))
        w = min(w, u - j)
        d = local_update(Z, b, A[:, j:j + w], B[:, j:j + w], C.eps, max_rank=C.rank_cap)
        Z2 = apply_delta(Z, d)
        Z.V, Z.W, Z.S, Z.N = Z2.V, Z2.W, Z2.S, Z2.N
        C.updates += 1
        C.max_rank = max(C.max_rank, max(Z.V.rank), max(Z.W.rank))
        j += w


def _factor_pair(P, x_cols=None, y_rows=None):
    """A dense term as a factor pair through its smallest dimension (reading 3)."""
    m, n = P.shape
    if x_cols is not None and x_cols.shape[1] <= min(m, n):
        return x_cols, y_rows
    if m <= n:
        return np.eye(m), P.T.copy()
    return P, np.eye(n)


# ----------------------------------------------------- product (Section 3)
def _case2(ZX, ZY, alpha, x, y):
    """Term alpha X|_x Y|_y when x or y is a leaf (Section 6, Case 2), as
    ('lr', A, B) or ('dense', P, X, Y) with P = alpha X Y; X = ZX, Y = ZY
    (the same matrix in the factorisation)."""
    bt = ZX.blocks
    t, s, r = bt.row[x], bt.col[x], bt.col[y]
    if bt.kind[y] == BlockTree.ADM:
        Xt = ZX.block_dense(x) @ ZY.V.dense(s)               # X|_{t x s} V_s
        return ("lr", alpha * (Xt @ ZY.S[y]), ZY.W.dense(r))
    if bt.kind[x] == BlockTree.ADM:
        Yt = ZY.block_dense(y).T @ ZX.W.dense(s)             # Y|_{s x r}^* W_s
        return ("lr", ZX.V.dense(t), alpha * (Yt @ ZX.S[x].T))
    X, Y = ZX.block_dense(x), ZY.block_dense(y)
    return ("dense", alpha * (X @ Y), alpha * X, Y.T)


def _collect(ZX, ZY, alpha, x, y, z, out):
    """Terms of Z|_z += alpha X|_x Y|_y in the order of the recursion."""
    Z = ZX
    bt = Z.blocks
    if bt.kind[x] == BlockTree.SUB and bt.kind[y] == BlockTree.SUB:
        t, s, r = bt.row[x], bt.col[x], bt.col[y]
        tree = Z.V.tree
        if bt.kind[z] == BlockTree.SUB:
            for s1 in tree.sons[s]:
                for t1 in tree.sons[t]:
                    for r1 in tree.sons[r]:
                        _collect(ZX, ZY, alpha, _son(bt, x, t1, s1), _son(bt, y, s1, r1), _son(bt, z, t1, r1),
                                 out)
            return
        assert bt.kind[z] == BlockTree.ADM, "inadmissible target of subdivided factors"
        temps = {}
        for s1 in tree.sons[s]:
            for t1 in tree.sons[t]:
                for r1 in tree.sons[r]:
                    _collect_virtual(ZX, ZY, alpha, _son(bt, x, t1, s1), _son(bt, y, s1, r1),
                                     temps.setdefault((t1, r1), []))
        for t1 in tree.sons[t]:
            for r1 in tree.sons[r]:
                out.append(("temp", z, temps.get((t1, r1), [])))
        return
    out.append(("term", z, (bt.row[x], bt.col[y]), _case2(ZX, ZY, alpha, x, y)))


def _collect_virtual(ZX, ZY, alpha, x, y, bucket):
    Z = ZX
    bt = Z.blocks
    if bt.kind[x] == BlockTree.SUB and bt.kind[y] == BlockTree.SUB:
        t, s, r = bt.row[x], bt.col[x], bt.col[y]
        tree = Z.V.tree
        for s1 in tree.sons[s]:
            for t1 in tree.sons[t]:
                for r1 in tree.sons[r]:
                    _collect_virtual(ZX, ZY, alpha, _son(bt, x, t1, s1), _son(bt, y, s1, r1), bucket)
        return
    bucket.append(((bt.row[x], bt.col[y]), _case2(ZX, ZY, alpha, x, y)))


def _place(Z, z, cl, A, B):
    """Extend factors of a term on clusters cl = (t', r') by zeros to z."""
    tree = Z.V.tree
    bt = Z.blocks
    t, r = bt.row[z], bt.col[z]
    Ax = np.zeros((tree.size[t], A.shape[1]))
    Bx = np.zeros((tree.size[r], B.shape[1]))
    a0 = tree.offset[cl[0]] - tree.offset[t]
    b0 = tree.offset[cl[1]] - tree.offset[r]
    Ax[a0:a0 + A.shape[0]] = A
    Bx[b0:b0 + B.shape[0]] = B
    return Ax, Bx


def _compress(A, B, eps):
    """Factor pair of A B^* truncated by SVD (reading 2)."""
    if A.shape[1] == 0:
        return A, B
    QA, RA = np.linalg.qr(A)
    QB, RB = np.linalg.qr(B)
    U, sig, Vt = np.linalg.svd(RA @ RB.T)
    total = float(np.sum(sig ** 2))
    if total == 0.0:
        return A[:, :0], B[:, :0]
    thr = (0.5 * eps) ** 2 * total
    r = len(sig)
    tail = 0.0
    while r > 0 and tail + sig[r - 1] ** 2 <= thr:
        tail += sig[r - 1] ** 2
        r -= 1
    return QA @ (U[:, :r] * sig[:r]), QB @ Vt[:r].T


def _apply_term(C: _Ctx, z, term):
    Z = C.Z
    bt = Z.blocks
    if term[0] == "lr":
        A, B = term[1], term[2]
        if bt.kind[z] == BlockTree.NEAR:
            Z.N[z] = Z.N[z] + A @ B.T
        else:
            _apply_update(C, z, A, B)
    else:
        P, X, Yt = term[1], term[2], term[3]
        if bt.kind[z] == BlockTree.NEAR:
            Z.N[z] = Z.N[z] + P
        else:
            A, B = _factor_pair(P, X, Yt)
            _apply_update(C, z, A, B)


def _mul(C: _Ctx, alpha, x, y, z, ZX=None, ZY=None):
    """Z|_z += alpha X|_x Y|_y (reading 1: terms from the matrices at the
    start); X, Y default to Z itself (the factorisation in place)."""
    out = []
    _collect(C.Z if ZX is None else ZX, C.Z if ZY is None else ZY, alpha, x, y, z, out)
    bt = C.Z.blocks
    groups = {}
    for item in out:
        if item[0] == "term" and bt.kind[item[1]] != BlockTree.NEAR:
            groups.setdefault(item[1], []).append(item[3])
    for item in out:
        if item[0] == "term":
            z1 = item[1]
            if bt.kind[z1] == BlockTree.NEAR:
                _apply_term(C, z1, item[3])
                continue
            terms = groups.pop(z1, None)
            if terms is None:        # added with the block's first term
                continue
            As, Bs = [], []
            for term in terms:
                if term[0] == "lr":
                    A, B = term[1], term[2]
                else:
                    A, B = _factor_pair(term[1], term[2], term[3])
                As.append(A)
                Bs.append(B)
            _apply_update(C, z1, np.hstack(As), np.hstack(Bs))
        else:
            z1, bucket = item[1], item[2]
            if not bucket:
                continue
            As, Bs = [], []
            for cl, term in bucket:
                if term[0] == "lr":
                    A, B = term[1], term[2]
                else:
                    A, B = _factor_pair(term[1], term[2], term[3])
                A, B = _place(C.Z, z1, cl, A, B)
                As.append(A)
                Bs.append(B)
            A, B = _compress(np.hstack(As), np.hstack(Bs), C.eps)
            _apply_update(C, z1, A, B)


# ---------------------------------------------- substitutions (Section 3)
def lsolve_dense(Z, d, Y):
    """X with L|_{t x t} X = Y (d = block (t, t), Y dense #t x m)."""
    bt = Z.blocks
    if bt.kind[d] == BlockTree.NEAR:
        return solve_triangular(Z.N[d], Y, lower=True, unit_diagonal=True)
    tree = Z.V.tree
    t = bt.row[d]
    t1, t2 = tree.sons[t]
    n1 = tree.size[t1]
    X1 = lsolve_dense(Z, _son(bt, d, t1, t1), Y[:n1])
    Y2 = Y[n1:] - Z.block_dense(_son(bt, d, t2, t1)) @ X1
    X2 = lsolve_dense(Z, _son(bt, d, t2, t2), Y2)
    return np.vstack([X1, X2])


def usolve_dense(Z, d, Y):
    """X with R|_{t x t} X = Y (upper triangular with the diagonal)."""
    bt = Z.blocks
    if bt.kind[d] == BlockTree.NEAR:
        return solve_triangular(Z.N[d], Y, lower=False)
    tree = Z.V.tree
    t = bt.row[d]
    t1, t2 = tree.sons[t]
    n1 = tree.size[t1]
    X2 = usolve_dense(Z, _son(bt, d, t2, t2), Y[n1:])
    Y1 = Y[:n1] - Z.block_dense(_son(bt, d, t1, t2)) @ X2
    X1 = usolve_dense(Z, _son(bt, d, t1, t1), Y1)
    return np.vstack([X1, X2])


def rsolve_dense(Z, d, Y):
    """X with X R|_{s x s} = Y (Y dense m x #s)."""
    bt = Z.blocks
    if bt.kind[d] == BlockTree.NEAR:
        return solve_triangular(Z.N[d], Y.T, trans="T", lower=False).T
    tree = Z.V.tree
    s = bt.row[d]
    s1, s2 = tree.sons[s]
    n1 = tree.size[s1]
    X1 = rsolve_dense(Z, _son(bt, d, s1, s1), Y[:, :n1])
    Y2 = Y[:, n1:] - X1 @ Z.block_dense(_son(bt, d, s1, s2))
    X2 = rsolve_dense(Z, _son(bt, d, s2, s2), Y2)
    return np.hstack([X1, X2])


def _lsolve(C: _Ctx, d, x):
    """Z|_x <- L|_{t x t}^-1 Z|_x in place, x = (t, s), d = (t, t)."""
    Z = C.Z
    bt = Z.blocks
    if bt.kind[x] == BlockTree.NEAR:
        Z.N[x] = lsolve_dense(Z, d, Z.N[x])
        return
    t, s = bt.row[x], bt.col[x]
    if bt.kind[x] == BlockTree.ADM:
        if Z.S[x].size == 0:          # a rank-0 basis: the block is zero and stays zero
            return
        Xh = lsolve_dense(Z, d, Z.V.dense(t) @ Z.S[x])        # reading 4
        Ws = Z.W.dense(s)
        Z.S[x] = np.zeros_like(Z.S[x])
        _apply_update(C, x, Xh, Ws)
        return
    tree = Z.V.tree
    t1, t2 = tree.sons[t]
    for s1 in tree.sons[s]:
        _lsolve(C, _son(bt, d, t1, t1), _son(bt, x, t1, s1))
    for s1 in tree.sons[s]:
        _mul(C, -1.0, _son(bt, d, t2, t1), _son(bt, x, t1, s1), _son(bt, x, t2, s1))
    for s1 in tree.sons[s]:
        _lsolve(C, _son(bt, d, t2, t2), _son(bt, x, t2, s1))


def _rsolve(C: _Ctx, d, x):
    """Z|_x <- Z|_x R|_{s x s}^-1 in place, x = (t, s), d = (s, s)."""
    Z = C.Z
    bt = Z.blocks
    if bt.kind[x] == BlockTree.NEAR:
        Z.N[x] = rsolve_dense(Z, d, Z.N[x])
        return
    t, s = bt.row[x], bt.col[x]
    if bt.kind[x] == BlockTree.ADM:
        if Z.S[x].size == 0:          # a rank-0 basis: the block is zero and stays zero
            return
        Bh = rsolve_dense(Z, d, Z.S[x] @ Z.W.dense(s).T).T    # reading 4
        Vt = Z.V.dense(t)
        Z.S[x] = np.zeros_like(Z.S[x])
        _apply_update(C, x, Vt, Bh)
        return
    tree = Z.V.tree
    s1, s2 = tree.sons[s]
    for t1 in tree.sons[t]:
        _rsolve(C, _son(bt, d, s1, s1), _son(bt, x, t1, s1))
    for t1 in tree.sons[t]:
        _mul(C, -1.0, _son(bt, x, t1, s1), _son(bt, d, s1, s2), _son(bt, x, t1, s2))
    for t1 in tree.sons[t]:
        _rsolve(C, _son(bt, d, s2, s2), _son(bt, x, t1, s2))


def _lr(C: _Ctx, d):
    Z = C.Z
    bt = Z.blocks
    if bt.kind[d] == BlockTree.NEAR:
        Z.N[d] = lu_doolittle(Z.N[d])
        return
    tree = Z.V.tree
    t = bt.row[d]
    t1, t2 = tree.sons[t]
    d11, d12 = _son(bt, d, t1, t1), _son(bt, d, t1, t2)
    d21, d22 = _son(bt, d, t2, t1), _son(bt, d, t2, t2)
    _lr(C, d11)
    _lsolve(C, d11, d12)
    _rsolve(C, d11, d21)
    _mul(C, -1.0, d21, d12, d22)
    _lr(C, d22)


def lr_factor(Z, eps: float, cap=32, rank_cap=None):
    """Factorise the H^2 matrix Z (square, same tree for rows and columns)
    in place: on return Z holds L and R.  ``rank_cap``: at most that many
    columns per new cluster basis in every local update (the rank cap
    option, off by default).  Returns statistics."""
    C = _Ctx(Z, eps, cap, rank_cap)
    _lr(C, 0)
    return {"updates": C.updates, "max_rank": C.max_rank}


def lr_solve(Z, b):
    """x with L R x = b (tree order; b a vector or n x m)."""
    b = np.asarray(b, dtype=np.float64)
    B = b.reshape(b.shape[0], -1)
    X = usolve_dense(Z, 0, lsolve_dense(Z, 0, B))
    return X.reshape(b.shape)


def pcg(apply_A, b, precond, tol=1e-10, maxit=1000):
    """Preconditioned conjugate gradients from x0 = 0, stopped when the
    updated residual satisfies ||r|| <= tol ||b||.  Returns x and the number
    of iterations."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = float(np.linalg.norm(b))
    if nb == 0.0:
        return x, 0
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    for it in range(1, maxit + 1):
        q = apply_A(p)
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        if float(np.linalg.norm(r)) <= tol * nb:
            return x, it
        z = precond(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit


def power_error(apply_A, precond, n, iters=50, seed=0):
    """||I - P^-1 A||_2 estimated by the power iteration (Section 7's Err)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = v - precond(apply_A(v))
        lam = float(np.linalg.norm(w))
        if lam == 0.0:
            return 0.0
        v = w / lam
    return lam


def mul(Z, X, Y, alpha: float, x: int, y: int, z: int, eps: float, cap=32, rank_cap=None):
    """The product of Section 3, Z|_z <- Z|_z + alpha X|_x Y|_y, for blocks
    x = (t, s), y = (s, r), z = (t, r) of the block tree the three H^2
    matrices share (X or Y may be Z itself); low-rank terms enter Z through
    local updates with accuracy eps.  Z is modified in place; returns the
    number of updates."""
    C = _Ctx(Z, eps, cap, rank_cap)
    _mul(C, alpha, x, y, z, X, Y)
    return C.updates



# ------------------------------------------- inversion (Remark on inversion)
def zero_like(Z):
    """An H^2 matrix with Z's trees and every rank, coupling and nearfield
    entry zero (reading 6)."""
    from .h2 import ClusterBasis, H2Matrix
    V, W = ClusterBasis(Z.V.tree), ClusterBasis(Z.W.tree)
    for cb in (V, W):
        tr = cb.tree
        for t in range(tr.n_clusters):
            if tr.is_leaf(t):
                cb.leaf[t] = np.zeros((tr.size[t], 0))
            if t > 0:
                cb.transfer[t] = np.zeros((0, 0))
    out = H2Matrix(Z.blocks, V, W)
    bt = Z.blocks
    out.S = {b: np.zeros((0, 0)) for b in bt.admissible}
    out.N = {b: np.zeros((Z.V.tree.size[bt.row[b]], Z.W.tree.size[bt.col[b]])) for b in bt.inadmissible}
    return out


def leaf_inverse(M: np.ndarray) -> np.ndarray:
    """M^-1 of a dense diagonal leaf: Doolittle's LU, then R^-1 L^-1 I."""
    F = lu_doolittle(M)
    n = F.shape[0]
    Y = solve_triangular(F, np.eye(n), lower=True, unit_diagonal=True)
    return solve_triangular(F, Y, lower=False)


def _inv(C: _Ctx, A, Cm, T, d):
    """Cm|_d <- (A|_d)^-1 for a diagonal block d (Remark on inversion)."""
    bt = A.blocks
    if bt.kind[d] == BlockTree.NEAR:
        Cm.N[d] = leaf_inverse(A.N[d])
        return
    t = bt.row[d]
    t1, t2 = A.V.tree.sons[t]
    d11, d12 = _son(bt, d, t1, t1), _son(bt, d, t1, t2)
    d21, d22 = _son(bt, d, t2, t1), _son(bt, d, t2, t2)
    _inv(C, A, Cm, T, d11)                                    # C11 = A11^-1
    C.updates += mul(T, Cm, A, 1.0, d11, d12, d12, C.eps, C.cap, C.rank_cap)    # B12 = A11^-1 A12
    C.updates += mul(T, A, Cm, 1.0, d21, d11, d21, C.eps, C.cap, C.rank_cap)    # B21 = A21 A11^-1
    C.updates += mul(A, A, T, -1.0, d21, d12, d22, C.eps, C.cap, C.rank_cap)    # S = A22 - A21 B12
    _inv(C, A, Cm, T, d22)                                    # C22 = S^-1
    C.updates += mul(Cm, T, Cm, -1.0, d12, d22, d12, C.eps, C.cap, C.rank_cap)  # C12 = -B12 C22
    C.updates += mul(Cm, Cm, T, -1.0, d22, d21, d21, C.eps, C.cap, C.rank_cap)  # C21 = -C22 B21
    C.updates += mul(Cm, Cm, T, -1.0, d12, d21, d11, C.eps, C.cap, C.rank_cap)  # C11 = C11 - C12 B21


def inverse(A, eps: float, cap=32, rank_cap=None):
    """The approximate inverse of the square H^2 matrix A (Remark on
    inversion, reading 6) as a new H^2 matrix with A's trees; A is consumed
    (its lower right blocks hold Schur complements on return).  Returns the
    inverse and statistics."""
    Cm, T = zero_like(A), zero_like(A)
    C = _Ctx(A, eps, cap, rank_cap)
    _inv(C, A, Cm, T, 0)
    return Cm, {"updates": C.updates}
