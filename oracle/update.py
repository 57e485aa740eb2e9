"""Local low-rank update of an H^2-matrix block (oracle; test infrastructure only).

Computes Z|_{t0 x s0} <- trunc_eps(Z|_{t0 x s0} + A B^*) for a block
b0 = (t0, s0) of the block tree, following Sections 4 and 5 step by step:

1. extension, Eq. (tildeZ_h2) restricted to the subtrees T_{t0}, T_{s0}
   (Section 5): V~_t = (V_t, A|_t), E~_t = diag(E_t, I) inside the subtree,
   E~_{t0} = [E_{t0}; 0], S~_b = diag(S_b, I) / [S_b; 0] / [S_b, 0];
2. basis R-factors V~_t = P_t R_t, leaf QR then QR of the stacked
   [R_{t1} E~_{t1}; R_{t2} E~_{t2}] (Section 4, "simple recursion");
   clusters outside the subtree have orthonormal bases and R = I;
3. weight matrices B~_t: R-factor of the stack of the blocks of row(t) and
   of the father's B~_{t+} E~_t^* (Section 4), top-down, taking every block
   of row(t) into account (Section 5) and starting from the ancestor path
   root -> t0+ of the unchanged matrix;
4. truncation bottom-up: leaf SVD of V~_t B~_t^* (Eq. (Qt_condensed)),
   inner SVD of V^_t B~_t^* with V^_t = [R_{t1} E~_{t1}; R_{t2} E~_{t2}]
   (Eq. (hatQt_condensed)), split of Q^_t into the new transfer matrices
   (Eq. (Qt_nested)), R_t = Q^_t^* V^_t;
5. reprojection of every affected coupling matrix, S_b <- R_t S~_b R_s^*,
   and the transfer commit E_{t0} <- R_{t0} [E_{t0}; 0] (Section 5);
6. dense addition of A|_t B|_s^* to the inadmissible leaves inside b0 (the
   paper does not spell this out; it is needed because b0 may be any block).

The column basis is handled "similarly, replacing Z~ by Z~^*" (Section 4).

Readings of points the paper leaves open (also listed in the design notes):

* the update rank u may differ from the cluster ranks: extensions use I_u;
* block-relative accuracy: a block b = (t, s) enters the row weights of t
  scaled by omega_b = sqrt(#T_t) / ||Z~|_b||_F and the column weights of s
  scaled by sqrt(#T_s) / ||Z~|_b||_F (#T_t = clusters in the subtree of t;
  omega_b = 0 for a zero block); each cluster keeps the smallest rank r with
  sum_{i>r} sigma_i^2 <= (eps/2)^2.  This bounds the error of every
  admissible block by ||Z~|_b - Z_new|_b||_F <= eps/sqrt(2) ||Z~|_b||_F;
* the weight inherited from the father of t0 is computed top-down from the
  root over the unchanged matrix and enters as B~_{t0+} [E_{t0}; 0]^*;
* an empty weight stack gives rank 0.
"""
from __future__ import annotations

import math

import numpy as np

from .h2 import H2Matrix
from .tree import BlockTree


def qr_r(M: np.ndarray) -> np.ndarray:
    """R-factor of a thin QR decomposition; min(rows, cols) x cols."""
    if M.shape[0] == 0 or M.shape[1] == 0:
        return np.zeros((0, M.shape[1]))
    return np.linalg.qr(M, mode="r")


def rank_rule(sigma: np.ndarray, eps: float) -> int:
    """Smallest r with sum_{i>=r} sigma_i^2 <= (eps/2)^2 (sigma descending)."""
    thr = (0.5 * eps) ** 2
    tail = 0.0
    r = len(sigma)
    while r > 0 and tail + sigma[r - 1] ** 2 <= thr:
        tail += sigma[r - 1] ** 2
        r -= 1
    return r


def rank_margin(sigma: np.ndarray, eps: float, r: int) -> float:
    """Relative distance of the rank decision from flipping (for test triage)."""
    thr = (0.5 * eps) ** 2
    tail_r = float(np.sum(sigma[r:] ** 2))
    if thr == 0.0:
        return math.inf
    if r == 0:
        return math.inf if tail_r == 0.0 else abs(thr - tail_r) / thr
    tail_next = tail_r + float(sigma[r - 1] ** 2)
    # keeping r is right because tail_next > thr >= tail_r
    lo = (thr - tail_r) / thr
    hi = (tail_next - thr) / thr
    return min(lo, hi)


class SideData:
    """Extended basis of one side restricted to a subtree (step 1)."""

    def __init__(self, basis, root: int, F: np.ndarray, tree):
        self.basis = basis
        self.tree = tree
        self.root = root
        self.sub = tree.descendants(root)          # DFS preorder
        self.inside = set(self.sub)
        self.u = F.shape[1]
        self.F = F
        off0 = tree.offset[root]
        self.K = {t: basis.rank[t] + self.u for t in self.sub}
        # V~_t for the leaves of the subtree: (V_t, F|_t)
        self.leaf_ext = {}
        for t in self.sub:
            if tree.is_leaf(t):
                r0 = tree.offset[t] - off0
                self.leaf_ext[t] = np.hstack([basis.leaf[t], F[r0:r0 + tree.size[t], :]])
        # E~_t = diag(E_t, I_u) inside, E~_{root} = [E_root; 0]
        self.E_ext = {}
        for t in self.sub:
            if t == 0:
                continue
            E = basis.transfer[t]
            if t == root:
                self.E_ext[t] = np.vstack([E, np.zeros((self.u, E.shape[1]))])
            else:
                k, kf = E.shape
                Ex = np.zeros((k + self.u, kf + self.u))
                Ex[:k, :kf] = E
                Ex[k:, kf:] = np.eye(self.u)
                self.E_ext[t] = Ex

    def r_factors(self) -> dict:
        """Step 2: R_t with V~_t = P_t R_t, bottom-up."""
        R = {}
        for t in reversed(self.sub):
            if self.tree.is_leaf(t):
                R[t] = qr_r(self.leaf_ext[t])
            else:
                R[t] = qr_r(np.vstack([R[s] @ self.E_ext[s] for s in self.tree.sons[t]]))
        return R


def extended_coupling(S: np.ndarray, t_in: bool, s_in: bool, u: int) -> np.ndarray:
    """S~_b of Eq. (tildeZ_h2) and its one-sided forms (Section 5)."""
    k, l = S.shape
    if t_in and s_in:
        X = np.zeros((k + u, l + u))
        X[:k, :l] = S
        X[k:, l:] = np.eye(u)
        return X
    if t_in:
        return np.vstack([S, np.zeros((u, l))])
    if s_in:
        return np.hstack([S, np.zeros((k, u))])
    return S


def local_update(Z: H2Matrix, b0: int, A: np.ndarray, B: np.ndarray, eps: float,
                 trace: dict | None = None, max_rank: int | None = None) -> dict:
    """One local low-rank update; returns the delta without modifying Z.

    ``max_rank`` (the rank cap option, off by default): every new cluster
    basis keeps at most that many of its leading singular directions.

    The delta holds the new ranks, leaf bases and transfer matrices of the
    clusters in T_{t0} (row) and T_{s0} (column), the new coupling matrices
    of every admissible block whose row lies in T_{t0} or whose column lies
    in T_{s0}, and the new nearfield blocks inside b0.  ``trace`` (if given)
    receives the intermediate matrices of steps 2-4.
    """
    bt = Z.blocks
    t0, s0 = bt.row[b0], bt.col[b0]
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    u = A.shape[1]
    assert B.shape[1] == u
    assert A.shape[0] == Z.V.tree.size[t0] and B.shape[0] == Z.W.tree.size[s0]

    # step 1: extension
    rs = SideData(Z.V, t0, A, Z.V.tree)
    cs = SideData(Z.W, s0, B, Z.W.tree)
    S_ext = {}
    for b in bt.admissible:
        t_in = bt.row[b] in rs.inside
        s_in = bt.col[b] in cs.inside
        if t_in or s_in:
            S_ext[b] = extended_coupling(Z.S[b], t_in, s_in, u)

    # step 2: basis R-factors of both sides
    RV = rs.r_factors()
    RW = cs.r_factors()

    def r_or_eye(R, side, c, k):
        return R[c] if c in side.inside else np.eye(k)

    # ||Z~|_b||_F = ||R_V,t S~_b R_W,s^*||_F for every block the weights touch
    def block_norm(b):
        t, s = bt.row[b], bt.col[b]
        Sx = S_ext.get(b, Z.S[b])
        Rt = r_or_eye(RV, rs, t, Sx.shape[0])
        Rs = r_or_eye(RW, cs, s, Sx.shape[1])
        return float(np.linalg.norm(Rt @ Sx @ Rs.T))

    # step 3: weights, row side (Z~) and column side (Z~^*)
    def weights(side, other, Rother, blocks_of, tree, transpose):
        # ancestor path root -> father of the subtree root, unchanged matrix
        B_prev = None
        path = tree.predecessors(side.root)[:-1]
        for a in path:
            rows = []
            for b in blocks_of[a]:
                nrm = block_norm(b)
                om = math.sqrt(tree.subtree_count[a]) / nrm if nrm > 0 else 0.0
                Sb = Z.S[b]
                rows.append(om * (Sb if transpose else Sb.T))
            if a != 0:
                rows.append(B_prev @ side.basis.transfer[a].T)
            B_prev = qr_r(np.vstack(rows)) if rows else np.zeros((0, side.basis.rank[a]))
        Bw = {}
        for t in side.sub:
            Kt = side.K[t]
            rows = []
            for b in blocks_of[t]:
                nrm = block_norm(b)
                om = math.sqrt(tree.subtree_count[t]) / nrm if nrm > 0 else 0.0
                o = bt.col[b] if not transpose else bt.row[b]
                Sx = S_ext.get(b, Z.S[b])
                Sx = Sx if transpose else Sx.T          # rows: other side's index
                Ro = r_or_eye(Rother, other, o, Sx.shape[0])
                rows.append(om * (Ro @ Sx))
            if t == side.root:
                if t != 0:
                    rows.append(B_prev @ side.E_ext[t].T)
            else:
                rows.append(Bw[tree.father[t]] @ side.E_ext[t].T)
            Bw[t] = qr_r(np.vstack(rows)) if rows else np.zeros((0, Kt))
        return Bw

    BV = weights(rs, cs, RW, bt.row_blocks, Z.V.tree, transpose=False)
    BW = weights(cs, rs, RV, bt.col_blocks, Z.W.tree, transpose=True)

    # step 4: truncation, bottom-up
    def truncate(side, Bw):
        tree = side.tree
        Rt, Q, Fnew, rank, sig, margin = {}, {}, {}, {}, {}, {}
        for t in reversed(side.sub):
            if tree.is_leaf(t):
                Vh = side.leaf_ext[t]
            else:
                Vh = np.vstack([Rt[s] @ side.E_ext[s] for s in tree.sons[t]])
            M = Vh @ Bw[t].T
            if M.shape[0] == 0 or M.shape[1] == 0:
                U = np.zeros((M.shape[0], 0))
                s_ = np.zeros(0)
            else:
                U, s_, _ = np.linalg.svd(M, full_matrices=False)
            r = rank_rule(s_, eps)
            if max_rank is not None and max_rank > 0:
                r = min(r, max_rank)
            Qh = U[:, :r]
            Rt[t] = Qh.T @ Vh
            rank[t] = r
            sig[t] = s_
            margin[t] = rank_margin(s_, eps, r)
            if tree.is_leaf(t):
                Q[t] = Qh
            else:
                r0 = 0
                for s in tree.sons[t]:
                    rs_ = rank[s]
                    Fnew[s] = Qh[r0:r0 + rs_, :]
                    r0 += rs_
        # transfer commit E_{t0} <- R_{t0} [E_{t0}; 0]
        if side.root != 0:
            Fnew[side.root] = Rt[side.root] @ side.E_ext[side.root]
        return Rt, Q, Fnew, rank, sig, margin

    RtV, QV, FV, rankV, sigV, marV = truncate(rs, BV)
    RtW, QW, FW, rankW, sigW, marW = truncate(cs, BW)

    # step 5: reprojection of every affected coupling matrix
    S_new = {}
    for b, Sx in S_ext.items():
        t, s = bt.row[b], bt.col[b]
        Rt = RtV[t] if t in rs.inside else np.eye(Sx.shape[0])
        Rs = RtW[s] if s in cs.inside else np.eye(Sx.shape[1])
        S_new[b] = Rt @ Sx @ Rs.T

    # step 6: nearfield leaves inside b0
    N_new = {}
    toff, soff = Z.V.tree.offset[t0], Z.W.tree.offset[s0]
    for b in bt.descendants(b0):
        if bt.kind[b] == BlockTree.NEAR:
            t, s = bt.row[b], bt.col[b]
            r0 = Z.V.tree.offset[t] - toff
            c0 = Z.W.tree.offset[s] - soff
            At = A[r0:r0 + Z.V.tree.size[t]]
            Bs = B[c0:c0 + Z.W.tree.size[s]]
            N_new[b] = Z.N[b] + At @ Bs.T

    if trace is not None:
        trace.update(dict(RV=RV, RW=RW, BV=BV, BW=BW, RtV=RtV, RtW=RtW, sigV=sigV, sigW=sigW,
                          marginV=marV, marginW=marW, rs=rs, cs=cs, S_ext=S_ext))
    return dict(b0=b0, t0=t0, s0=s0,
                V=dict(rank=rankV, leaf=QV, transfer=FV),
                W=dict(rank=rankW, leaf=QW, transfer=FW),
                S=S_new, N=N_new,
                margin=min([math.inf] + list(marV.values()) + list(marW.values())))


def apply_delta(Z: H2Matrix, delta: dict) -> H2Matrix:
    """Return a copy of Z with the delta of ``local_update`` committed."""
    out = Z.copy()
    for key, basis in (("V", out.V), ("W", out.W)):
        d = delta[key]
        for t, r in d["rank"].items():
            basis.rank[t] = r
        for t, q in d["leaf"].items():
            basis.leaf[t] = q
        for t, f in d["transfer"].items():
            basis.transfer[t] = f
    for b, s in delta["S"].items():
        out.S[b] = s
    for b, n in delta["N"].items():
        out.N[b] = n
    return out


def isolated_batch(Z: H2Matrix, blocks, A_list, B_list, eps: float) -> list:
    """Isolated batch: every update reads the same Z and yields its own delta."""
    return [local_update(Z, b, A, B, eps) for b, A, B in zip(blocks, A_list, B_list)]


def sequential_batch(Z: H2Matrix, blocks, A_list, B_list, eps: float) -> H2Matrix:
    """Sequential batch: the updates are applied one after the other, in order."""
    for b, A, B in zip(blocks, A_list, B_list):
        Z = apply_delta(Z, local_update(Z, b, A, B, eps))
    return Z
