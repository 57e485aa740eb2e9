"""Pins of the oracle's local low-rank update (Sections 4 and 5).

Each test checks the oracle against a fact that the paper or the
mathematics fixes, computed densely and independently of the oracle's
structured recursions:

* Eq. (tildeZ_h2) is exact: at eps = 0 the update reproduces Z + A B^*;
* one admissible block alone in its block row and column: the update is
  the truncated SVD of Z~|_b (Eckart-Young) with the same rank;
* basis R-factors: R_t^* R_t = V~_t^* V~_t;
* weights: V~_t B~_t^* B~_t V~_t^* = Z~_t Z~_t^* for the dense weighted
  block row Z~_t (Eq. (Zt_factors));
* truncation: the singular values equal those of the dense condensed block
  row; the new bases are orthonormal and nested;
* reprojection: S_b = Q_t^* Z~|_b Q_s (Section 2, optimal couplings);
* block-relative accuracy: ||Z~|_b - Z_new|_b|| <= eps/sqrt(2) ||Z~|_b||
  for every admissible block, unaffected couplings bit-unchanged.
"""
import math

import numpy as np
import pytest

import synth
from dense_ref import basis_dense, block, weighted_block_row
from oracle.h2 import ClusterBasis, H2Matrix
from oracle.tree import BlockTree, ClusterTree
from oracle.update import apply_delta, local_update
from problems import draw_updates, embed, oracle_problem


@pytest.fixture(scope="module")
def prob():
    Z, st, _ = oracle_problem(24, 6, seed=11, leaf=16)
    blocks, A, B = draw_updates(Z, st, 4, 3)
    return Z, blocks, A, B


def _extra_blocks(Z):
    """Root block, a subdivided block and an inadmissible leaf."""
    bt = Z.blocks
    sub = [b for b in range(1, bt.n_blocks) if bt.kind[b] == BlockTree.SUB]
    return [0, sub[len(sub) // 2], bt.inadmissible[len(bt.inadmissible) // 3]]


def _factors(Z, b, u, rng):
    bt = Z.blocks
    A = rng.standard_normal((Z.V.tree.size[bt.row[b]], u))
    B = rng.standard_normal((Z.W.tree.size[bt.col[b]], u))
    return A, B


def _all_cases(Z, blocks, A, B):
    rng = np.random.default_rng(5)
    cases = list(zip(blocks, A, B))
    for b in _extra_blocks(Z):
        cases.append((b,) + _factors(Z, b, 3, rng))
    return cases


def test_exact_at_eps_zero(prob):
    Z, blocks, A, B = prob
    D = Z.dense()
    for b, a, bb in _all_cases(Z, blocks, A, B):
        Zn = apply_delta(Z, local_update(Z, b, a, bb, 0.0))
        ref = D + embed(Z, b, a, bb)
        assert np.linalg.norm(Zn.dense() - ref) <= 1e-13 * np.linalg.norm(ref)


def test_dense_assembly_matches_path_products(prob):
    Z = prob[0]
    for t in range(Z.V.tree.n_clusters):
        np.testing.assert_allclose(Z.V.dense(t), basis_dense(Z.V.tree, Z.V, t), rtol=0, atol=1e-14)


def _two_group_problem(k, seed):
    """Two distant groups of 12 points: the block tree is the root split once
    into two nearfield diagonal blocks and two admissible off-diagonal ones."""
    rng = np.random.default_rng(seed)
    g1 = rng.uniform(0.0, 0.1, size=(12, 2))
    g2 = rng.uniform(0.9, 1.0, size=(12, 2))
    pts = np.vstack([g1, g2])
    ct = ClusterTree(pts, 12)
    bt = BlockTree(ct, ct, 2.0)
    assert ct.n_clusters == 3 and len(bt.admissible) == 2

    def basis():
        cb = ClusterBasis(ct)
        cb.rank = [k, k, k]
        for t in (1, 2):
            q, _ = np.linalg.qr(rng.standard_normal((12, k)))
            cb.leaf[t] = q
            cb.transfer[t] = np.linalg.qr(rng.standard_normal((2 * k, k)))[0][(t - 1) * k:t * k]
        return cb

    Z = H2Matrix(bt, basis(), basis())
    for b in bt.admissible:
        # singular values spread over 1 .. 1e-6
        U, _ = np.linalg.qr(rng.standard_normal((k, k)))
        Vv, _ = np.linalg.qr(rng.standard_normal((k, k)))
        Z.S[b] = U @ np.diag(np.logspace(0, -6, k)) @ Vv.T
    for b in bt.inadmissible:
        Z.N[b] = rng.standard_normal((12, 12))
    return Z


@pytest.mark.parametrize("eps", [1e-7, 1e-4, 1e-2, 0.3])
def test_single_block_is_truncated_svd(eps):
    k, u = 5, 2
    Z = _two_group_problem(k, seed=3)
    bt = Z.blocks
    b0 = bt.admissible[0]
    t0, s0 = bt.row[b0], bt.col[b0]
    rng = np.random.default_rng(9)
    A = 1e-3 * rng.standard_normal((12, u))
    B = rng.standard_normal((12, u))
    D = Z.dense()
    Zt = D + embed(Z, b0, A, B)
    d = local_update(Z, b0, A, B, eps)
    Zn = apply_delta(Z, d)
    blk = block(Zt, Z.V.tree, Z.W.tree, t0, s0)
    U, sig, Yt = np.linalg.svd(blk)
    # block-relative rank: smallest r with tail <= (eps/2)^2 ||Z~|_b||^2
    thr = (0.5 * eps * np.linalg.norm(blk)) ** 2
    r = len(sig)
    while r > 0 and np.sum(sig[r - 1:] ** 2) <= thr:
        r -= 1
    assert d["V"]["rank"][t0] == r and d["W"]["rank"][s0] == r
    best = (U[:, :r] * sig[:r]) @ Yt[:r]
    got = block(Zn.dense(), Z.V.tree, Z.W.tree, t0, s0)
    assert np.linalg.norm(got - best) <= 1e-12 * np.linalg.norm(blk)
    # nothing else moved
    other = Zn.dense() - got.sum() * 0
    mask = np.ones_like(D, dtype=bool)
    r0, c0 = Z.V.tree.offset[t0], Z.W.tree.offset[s0]
    mask[r0:r0 + 12, c0:c0 + 12] = False
    np.testing.assert_array_equal(other[mask], D[mask])


def _trace_case(Z, b, a, bb, eps):
    tr = {}
    d = local_update(Z, b, a, bb, eps, trace=tr)
    return d, tr


def _ext_dense(Z, side, t, F, root):
    tree = Z.V.tree if side == "V" else Z.W.tree
    basis = Z.V if side == "V" else Z.W
    r0 = tree.offset[t] - tree.offset[root]
    return np.hstack([basis_dense(tree, basis, t), F[r0:r0 + tree.size[t]]])


@pytest.mark.parametrize("eps", [1e-6, 0.5, 2.0])
def test_r_factors_and_weights_gram(prob, eps):
    Z, blocks, A, B = prob
    D = Z.dense()
    for b, a, bb in _all_cases(Z, blocks, A, B)[:5]:
        d, tr = _trace_case(Z, b, a, bb, eps)
        Zt = D + embed(Z, b, a, bb)
        for side, F, root, R, Bw in (("V", a, d["t0"], tr["RV"], tr["BV"]),
                                     ("W", bb, d["s0"], tr["RW"], tr["BW"])):
            for t in R:
                Vx = _ext_dense(Z, side, t, F, root)
                G = Vx.T @ Vx
                np.testing.assert_allclose(R[t].T @ R[t], G, rtol=0, atol=1e-12 * max(1.0, np.abs(G).max()))
                Zw = weighted_block_row(Zt, Z, t, row_side=(side == "V"))
                lhs = Vx @ (Bw[t].T @ Bw[t]) @ Vx.T
                rhs = Zw @ Zw.T
                np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-11 * max(1.0, np.abs(rhs).max()))


@pytest.mark.parametrize("eps", [1e-6, 0.5, 2.0])
def test_truncation_and_reprojection(prob, eps):
    Z, blocks, A, B = prob
    D = Z.dense()
    bt = Z.blocks
    for b, a, bb in _all_cases(Z, blocks, A, B):
        d, tr = _trace_case(Z, b, a, bb, eps)
        Zn = apply_delta(Z, d)
        Zt = D + embed(Z, b, a, bb)
        for side, sig in (("V", tr["sigV"]), ("W", tr["sigW"])):
            tree = Zn.V.tree if side == "V" else Zn.W.tree
            basis = Zn.V if side == "V" else Zn.W
            for t, s_ in sig.items():
                Q = basis_dense(tree, basis, t)
                # orthonormal new basis (nestedness is the representation itself)
                np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), rtol=0, atol=1e-12)
                Zw = weighted_block_row(Zt, Z, t, row_side=(side == "V"))
                if tree.sons[t]:
                    P = np.zeros((tree.size[t], 0))
                    blocks_ = []
                    for c in tree.sons[t]:
                        blocks_.append(basis_dense(tree, basis, c))
                    from scipy.linalg import block_diag
                    P = block_diag(*blocks_)
                    Cw = P.T @ Zw
                else:
                    Cw = Zw
                ref = np.linalg.svd(Cw, compute_uv=False) if Cw.size else np.zeros(0)
                n = min(len(ref), len(s_))
                scale = max(1.0, ref[0] if len(ref) else 1.0)
                np.testing.assert_allclose(s_[:n], ref[:n], rtol=0, atol=1e-11 * scale)
                assert np.all(ref[n:] <= 1e-11 * scale) and np.all(s_[n:] <= 1e-11 * scale)
        # reprojection: S_b = Q_t^* Z~|_b Q_s for every affected block
        for c, Snew in d["S"].items():
            t, s = bt.row[c], bt.col[c]
            Qt = basis_dense(Zn.V.tree, Zn.V, t)
            Qs = basis_dense(Zn.W.tree, Zn.W, s)
            ref = Qt.T @ block(Zt, Z.V.tree, Z.W.tree, t, s) @ Qs
            np.testing.assert_allclose(Snew, ref, rtol=0, atol=1e-11 * max(1.0, np.abs(ref).max()))
        # unaffected couplings are bit-unchanged; ranks never exceed k + u
        for c in bt.admissible:
            if c not in d["S"]:
                np.testing.assert_array_equal(Zn.S[c], Z.S[c])
        for side in ("V", "W"):
            for t, r in d[side]["rank"].items():
                assert r <= getattr(Z, side).rank[t] + a.shape[1]


@pytest.mark.parametrize("eps", [1e-6, 0.1, 0.5, 2.0])
def test_block_relative_error_bound(prob, eps):
    Z, blocks, A, B = prob
    D = Z.dense()
    bt = Z.blocks
    truncated = 0
    for b, a, bb in _all_cases(Z, blocks, A, B):
        d = local_update(Z, b, a, bb, eps)
        Zn = apply_delta(Z, d)
        Dn = Zn.dense()
        Zt = D + embed(Z, b, a, bb)
        for c in bt.admissible:
            t, s = bt.row[c], bt.col[c]
            ref = block(Zt, Z.V.tree, Z.W.tree, t, s)
            err = np.linalg.norm(block(Dn, Z.V.tree, Z.W.tree, t, s) - ref)
            assert err <= (eps / math.sqrt(2) + 1e-13) * np.linalg.norm(ref)
        for c in bt.inadmissible:
            t, s = bt.row[c], bt.col[c]
            np.testing.assert_allclose(block(Dn, Z.V.tree, Z.W.tree, t, s),
                                       block(Zt, Z.V.tree, Z.W.tree, t, s), rtol=0, atol=1e-13)
        truncated += sum(r < Z.V.rank[t] + a.shape[1] for t, r in d["V"]["rank"].items())
    if eps >= 0.5:
        assert truncated > 0   # the large tolerances really truncate


def test_near_range_update_is_compressed(prob):
    """A nearly inside range(V_t0) x range(W_s0): the new directions are
    below the tolerance and the ranks fall back to k (Eq. (Qt_condition))."""
    Z, blocks, _, _ = prob
    bt = Z.blocks
    b = blocks[0]
    t0, s0 = bt.row[b], bt.col[b]
    rng = np.random.default_rng(2)
    Vt = basis_dense(Z.V.tree, Z.V, t0)
    Ws = basis_dense(Z.W.tree, Z.W, s0)
    A = Vt @ rng.standard_normal((Vt.shape[1], 3)) + 1e-9 * rng.standard_normal((Vt.shape[0], 3))
    B = Ws @ rng.standard_normal((Ws.shape[1], 3))
    d = local_update(Z, b, A, B, 1e-4)
    assert all(r <= Z.V.rank[t] for t, r in d["V"]["rank"].items())
    Zn = apply_delta(Z, d)
    ref = Z.dense() + embed(Z, b, A, B)
    blk = block(ref, Z.V.tree, Z.W.tree, t0, s0)
    got = block(Zn.dense(), Z.V.tree, Z.W.tree, t0, s0)
    assert np.linalg.norm(got - blk) <= 1e-4 * np.linalg.norm(blk)
