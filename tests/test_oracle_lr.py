"""Pins of the oracle's H^2-LR, substitutions, product and CG (oracle.lr) -- CPU.

Against what the mathematics fixes:

* Gaussian elimination without pivoting: L R = M with L unit lower and R
  upper triangular; equal to LAPACK's LU where it does not pivot;
* the H^2-LR at eps = 0 is exact (every local update is exact, Eq.
  (tildeZ_h2)), so it must equal dense Doolittle LU of the FEM matrix;
* at eps = 1e-4 the factor reproduces A to O(eps) and preconditions CG to
  a few steps (Table 1: m = 3 at the paper's accuracies);
* the product Z|_z += alpha X|_x Y|_y at eps = 0 changes exactly the
  target block, by the dense product (every kind of triple: subdivided
  target, admissible target of subdivided factors, low-rank and dense
  terms);
* block substitutions equal dense triangular solves with the same factor;
* CG: a diagonal matrix with three distinct eigenvalues needs three steps,
  an exact preconditioner one; the power iteration on a diagonal matrix
  gives max |1 - a_i / c| for the preconditioner c I.
"""
import numpy as np
import pytest
import scipy.linalg as la

import synth
from oracle.fem import h2_from_sparse, stiffness
from oracle.lr import (_Ctx, _mul, lr_factor, lr_solve, lsolve_dense, lu_doolittle, mul, pcg, power_error,
                       rsolve_dense, usolve_dense)
from oracle.tree import BlockTree
from problems import block_triples as _triples, oracle_problem


def _fem(N, leaf, seed=0, M=4):
    sigma = synth.checker_sigma(np.random.default_rng(seed), M, 2)
    K, pts = stiffness(N, 2, sigma, M)
    Z = h2_from_sparse(K, pts, leaf, 2.0, 1.0 / N)
    perm = Z.V.tree.perm
    return Z, K[perm][:, perm].toarray()


def test_doolittle():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((9, 9)) + 12 * np.eye(9)
    F = lu_doolittle(M)
    Lm, Rm = np.tril(F, -1) + np.eye(9), np.triu(F)
    assert np.abs(Lm @ Rm - M).max() <= 1e-13 * np.abs(M).max()
    P, L2, R2 = la.lu(M)
    assert np.array_equal(P, np.eye(9))          # diagonally dominant: no pivoting
    assert np.abs(Lm - L2).max() <= 1e-13 and np.abs(Rm - R2).max() <= 1e-12


@pytest.mark.parametrize("N,leaf", [(16, 16), (14, 8)])
def test_lr_without_truncation_is_dense_lu(N, leaf):
    Z, A = _fem(N, leaf, seed=N)
    info = lr_factor(Z, 0.0)
    D = Z.dense()
    ref = lu_doolittle(A)
    assert np.linalg.norm(D - ref) <= 1e-12 * np.linalg.norm(ref)
    assert info["updates"] > 0 and info["max_rank"] > 0


def test_lr_truncated_is_a_preconditioner():
    Z, A = _fem(32, 32, seed=3)
    lr_factor(Z, 1e-4)
    D = Z.dense()
    n = D.shape[0]
    Lm, Rm = np.tril(D, -1) + np.eye(n), np.triu(D)
    err = np.linalg.norm(A - Lm @ Rm) / np.linalg.norm(A)
    assert 0 < err <= 1e-5
    b = np.random.default_rng(1).standard_normal(n)
    x, it = pcg(lambda v: A @ v, b, lambda r: lr_solve(Z, r), 1e-10)
    assert it <= 5 and np.linalg.norm(A @ x - b) <= 1e-9 * np.linalg.norm(b)
    x0, it0 = pcg(lambda v: A @ v, b, lambda r: r, 1e-10)
    assert it0 > 10 * it


def test_substitutions_are_dense_triangular_solves():
    Z, A = _fem(16, 8, seed=5)
    lr_factor(Z, 0.0)
    D = Z.dense()
    n = D.shape[0]
    Lm, Rm = np.tril(D, -1) + np.eye(n), np.triu(D)
    Y = np.random.default_rng(2).standard_normal((n, 3))
    assert np.allclose(lsolve_dense(Z, 0, Y), la.solve_triangular(Lm, Y, lower=True), rtol=0, atol=1e-10)
    assert np.allclose(usolve_dense(Z, 0, Y), la.solve_triangular(Rm, Y), rtol=0, atol=1e-10)
    Yr = Y.T.copy()
    assert np.allclose(rsolve_dense(Z, 0, Yr), la.solve_triangular(Rm.T, Yr.T, lower=True).T, rtol=0, atol=1e-10)
    assert np.allclose(lr_solve(Z, Y), np.linalg.solve(A, Y), rtol=0, atol=1e-9)


def test_product_is_exact_without_truncation():
    Zo, _, _ = oracle_problem(16, 3, 77, 8)
    bt, ct = Zo.blocks, Zo.V.tree
    triples = _triples(bt, ct)
    kinds = {k[2] for k in triples}
    assert BlockTree.SUB in kinds and BlockTree.ADM in kinds and BlockTree.NEAR in kinds
    assert (BlockTree.SUB, BlockTree.SUB, BlockTree.ADM) in triples   # temporaries
    for key, (x, y, z) in triples.items():
        Z = Zo.copy()
        before = Z.dense()
        X, Y = Z.block_dense(x), Z.block_dense(y)
        _mul(_Ctx(Z, 0.0, None), -0.75, x, y, z)
        want = before.copy()
        t, r = bt.row[z], bt.col[z]
        want[ct.offset[t]:ct.offset[t] + ct.size[t], ct.offset[r]:ct.offset[r] + ct.size[r]] += -0.75 * X @ Y
        got = Z.dense()
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want), key


def test_product_of_three_matrices_is_exact_without_truncation():
    """Z|_z += alpha X|_x Y|_y with three different H^2 matrices on one tree
    (different bases and couplings): at eps = 0 exactly the dense product is
    added to the target block, for every combination of block kinds."""
    X, _, _ = oracle_problem(16, 3, 81, 8)
    Y, _, _ = oracle_problem(16, 4, 82, 8)
    Z0, _, _ = oracle_problem(16, 2, 83, 8)
    bt, ct = Z0.blocks, Z0.V.tree
    triples = _triples(bt, ct)
    for key, (x, y, z) in triples.items():
        Z = Z0.copy()
        before = Z.dense()
        Xb, Yb = X.block_dense(x), Y.block_dense(y)
        mul(Z, X, Y, 0.5, x, y, z, 0.0, cap=None)
        want = before.copy()
        t, r = bt.row[z], bt.col[z]
        want[ct.offset[t]:ct.offset[t] + ct.size[t], ct.offset[r]:ct.offset[r] + ct.size[r]] += 0.5 * Xb @ Yb
        got = Z.dense()
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want), key
        # X and Y are read only
        assert np.array_equal(X.block_dense(x), Xb) and np.array_equal(Y.block_dense(y), Yb)


def test_cg_step_counts():
    d = np.array([1.0] * 5 + [4.0] * 7 + [9.0] * 3)
    b = np.random.default_rng(0).standard_normal(len(d))
    x, it = pcg(lambda v: d * v, b, lambda r: r, 1e-12)
    assert it == 3 and np.allclose(d * x, b)
    x, it = pcg(lambda v: d * v, b, lambda r: r / d, 1e-12)
    assert it == 1


def test_power_error_closed_form():
    d = np.linspace(1.0, 3.0, 40)
    c = 2.5
    e = power_error(lambda v: d * v, lambda r: r / c, len(d), iters=400, seed=1)
    assert abs(e - np.max(np.abs(1 - d / c))) <= 1e-6


def test_rank_cap():
    """The rank cap option: no basis rank above it; a cap above every rank
    the factorisation reaches changes nothing."""
    Z, A = _fem(24, 16, seed=9)
    Z1, Z2 = Z.copy(), Z.copy()
    info = lr_factor(Z1, 1e-4)
    top = info["max_rank"]
    assert top > 4
    lr_factor(Z2, 1e-4, rank_cap=top)
    np.testing.assert_array_equal(Z1.dense(), Z2.dense())
    Z3 = Z.copy()
    info3 = lr_factor(Z3, 1e-4, rank_cap=4)
    assert max(Z3.V.rank) <= 4 and max(Z3.W.rank) <= 4 and info3["max_rank"] == 4
    # still a preconditioner, a weaker one
    D = Z3.dense()
    n = D.shape[0]
    Lm, Rm = np.tril(D, -1) + np.eye(n), np.triu(D)
    assert np.linalg.norm(A - Lm @ Rm) <= 1e-1 * np.linalg.norm(A)
