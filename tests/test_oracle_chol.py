"""Pins of the oracle's approximate Cholesky factorisation (oracle.chol;
Section 7 builds its preconditioner this way, with the algorithms of
Section 3) -- CPU.

Against what the mathematics fixes:

* a dense leaf: L L^* = M, L lower with a positive diagonal, equal to
  numpy's Cholesky factor; an indefinite matrix is refused;
* without truncation every step is exact, so the factor is the Cholesky
  factor of the FEM matrix (numpy, dense), and the strictly upper
  nearfield is never read (scrambled, the factor keeps every bit);
* the product with the second factor read transposed, without
  truncation, adds exactly alpha X|_x (X|_y)^* (dense check), and for a
  diagonal target with ``lower`` only the blocks on or below the diagonal;
* at eps = 1e-4 the factor reproduces A to O(eps), L L^* is symmetric
  positive definite, and CG preconditioned by it converges in a few steps
  (Table 1: m = 3 at the paper's accuracies).
* without truncation the Cholesky factor is the LR's unit lower factor
  scaled by the square roots of the LR's pivots (A = L U with U = D L^*).
"""
import numpy as np
import pytest

import synth
from oracle.chol import _mul_t, chol_dense, chol_factor, chol_solve, lower
from oracle.fem import h2_from_sparse, stiffness
from oracle.lr import _Ctx, _son, pcg


def _fem(N, leaf, seed, M=4, dim=2):
    sigma = synth.checker_sigma(np.random.default_rng(seed), M, dim)
    K, pts = stiffness(N, dim, sigma, M)
    Z = h2_from_sparse(K, pts, leaf, 2.0, 1.0 / N)
    perm = Z.V.tree.perm
    return Z, K[perm][:, perm].toarray()


def test_chol_dense():
    rng = np.random.default_rng(0)
    G = rng.standard_normal((13, 13))
    M = G @ G.T + 13 * np.eye(13)
    L = chol_dense(M)
    assert np.array_equal(L, np.tril(L)) and (np.diag(L) > 0).all()
    assert np.abs(L @ L.T - M).max() <= 1e-13 * np.abs(M).max()
    assert np.abs(L - np.linalg.cholesky(M)).max() <= 1e-13 * np.abs(L).max()
    # only the lower triangle is read
    M2 = np.tril(M) + np.triu(rng.standard_normal((13, 13)), 1)
    assert np.array_equal(chol_dense(M2), L)
    with pytest.raises(ValueError):
        chol_dense(np.diag([1.0, -1.0, 2.0]))


@pytest.mark.parametrize("N,leaf,dim", [(12, 8, 2), (16, 16, 2), (8, 16, 3)])
def test_chol_without_truncation_is_dense_cholesky(N, leaf, dim):
    Z, A = _fem(N, leaf, seed=N + 3, M=2 if dim == 3 else 4, dim=dim)
    info = chol_factor(Z, 0.0, cap=None)
    L = lower(Z)
    ref = np.linalg.cholesky(A)
    assert np.linalg.norm(L - ref) <= 1e-12 * np.linalg.norm(ref)
    assert info["updates"] > 0 and info["max_rank"] > 0
    # the strictly upper nearfield is never read: scrambled, the factor
    # keeps every bit
    Z2, _ = _fem(N, leaf, seed=N + 3, M=2 if dim == 3 else 4, dim=dim)
    tr, bt = Z2.V.tree, Z2.blocks
    rng = np.random.default_rng(1)
    for b in bt.inadmissible:
        if tr.offset[bt.row[b]] < tr.offset[bt.col[b]]:
            Z2.N[b] = rng.standard_normal(Z2.N[b].shape)
        elif bt.row[b] == bt.col[b]:
            Z2.N[b] = Z2.N[b] + np.triu(rng.standard_normal(Z2.N[b].shape), 1)
    chol_factor(Z2, 0.0, cap=None)
    assert np.array_equal(lower(Z2), L)


@pytest.mark.parametrize("lower_only", [False, True])
def test_product_with_transposed_factor(lower_only):
    Z, A = _fem(16, 16, seed=11)
    chol_factor(Z, 0.0, cap=None)            # admissible blocks of rank > 0
    bt, tr = Z.blocks, Z.V.tree
    t1, t2 = tr.sons[0]
    d21, d22 = _son(bt, 0, t2, t1), _son(bt, 0, t2, t2)
    assert max(Z.V.rank) > 0
    before = Z.dense()
    r2 = slice(tr.offset[t2], tr.offset[t2] + tr.size[t2])
    r1 = slice(tr.offset[t1], tr.offset[t1] + tr.size[t1])
    X = before[r2, r1]
    want = before[r2, r2] - 0.5 * X @ X.T
    Z2 = Z.copy()
    C = _Ctx(Z2, 0.0, None)
    _mul_t(C, -0.5, d21, d21, d22, lower_only)
    got = Z2.dense()[r2, r2]
    if lower_only:
        # blocks on or below the diagonal get the product, the others stay
        for b in list(bt.admissible) + list(bt.inadmissible):
            t, s = bt.row[b], bt.col[b]
            if not (tr.offset[t] >= tr.offset[t2] and tr.offset[s] >= tr.offset[t2]):
                continue
            rt = slice(tr.offset[t] - tr.offset[t2], tr.offset[t] - tr.offset[t2] + tr.size[t])
            cs = slice(tr.offset[s] - tr.offset[t2], tr.offset[s] - tr.offset[t2] + tr.size[s])
            ref = want if tr.offset[t] >= tr.offset[s] else before[r2, r2]
            assert np.abs(got[rt, cs] - ref[rt, cs]).max() <= 1e-12 * np.abs(want).max(), b
    else:
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # the factor X itself is unchanged (terms from the matrix at the start)
    assert np.abs(Z2.dense()[r2, r1] - X).max() <= 1e-12 * np.abs(X).max()


def test_chol_truncated_is_a_preconditioner():
    Z, A = _fem(24, 16, seed=5)
    info = chol_factor(Z, 1e-4)
    L = lower(Z)
    n = A.shape[0]
    assert np.linalg.norm(A - L @ L.T) <= 1e-5 * np.linalg.norm(A)
    assert (np.diag(L) > 0).all()
    b = np.random.default_rng(2).standard_normal(n)
    x, it = pcg(lambda v: A @ v, b, lambda r: chol_solve(Z, r), 1e-10)
    assert it <= 5 and np.linalg.norm(A @ x - b) <= 1e-9 * np.linalg.norm(b)
    # fewer local updates than the LR of the same matrix (one triangle)
    from oracle.lr import lr_factor
    Z2, _ = _fem(24, 16, seed=5)
    assert info["updates"] < lr_factor(Z2, 1e-4)["updates"]


def test_chol_solve():
    Z, A = _fem(12, 8, seed=7)
    chol_factor(Z, 0.0, cap=None)
    B = np.random.default_rng(3).standard_normal((A.shape[0], 2))
    X = chol_solve(Z, B)
    assert np.linalg.norm(A @ X - B) <= 1e-10 * np.linalg.norm(B)


def test_chol_is_the_scaled_lr_without_truncation():
    """For a symmetric positive definite A, Doolittle's A = L U has
    U = D L^*, so the Cholesky factor is L D^(1/2): the two oracle
    factorisations, run without truncation, agree to rounding."""
    from oracle.lr import lr_factor
    Z1, A = _fem(16, 8, seed=13)
    Z2 = Z1.copy()
    chol_factor(Z1, 0.0, cap=None)
    lr_factor(Z2, 0.0, cap=None)
    D = Z2.dense()
    n = D.shape[0]
    Ld = np.tril(D, -1) + np.eye(n)
    d = np.diag(D)
    assert (d > 0).all()
    Lc = lower(Z1)
    assert np.linalg.norm(Lc - Ld * np.sqrt(d)) <= 1e-12 * np.linalg.norm(Lc)
