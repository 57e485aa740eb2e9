"""Pins of the oracle's approximate inverse (oracle.lr.inverse; the Remark
on inversion) -- CPU.

Against what the mathematics fixes:

* a leaf is inverted exactly: Doolittle LU and two triangular solves equal
  numpy's inverse on a diagonally dominant matrix;
* a zero matrix with A's trees is zero (every rank 0);
* without truncation every product of the recursion is exact, so the
  result is the inverse of the FEM matrix (dense, numpy);
* at eps = 1e-4 the result approximates the inverse to O(eps) and
  preconditions CG to a few steps (Table 1: m = 3 at the paper's
  accuracies).
"""
import numpy as np
import pytest

import synth
from oracle.fem import h2_from_sparse, stiffness
from oracle.lr import inverse, leaf_inverse, pcg, zero_like


def _fem(N, leaf, seed, M=4):
    sigma = synth.checker_sigma(np.random.default_rng(seed), M, 2)
    K, pts = stiffness(N, 2, sigma, M)
    Z = h2_from_sparse(K, pts, leaf, 2.0, 1.0 / N)
    perm = Z.V.tree.perm
    return Z, K[perm][:, perm].toarray()


def test_leaf_inverse():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((11, 11)) + 15 * np.eye(11)
    Minv = leaf_inverse(M)
    ref = np.linalg.inv(M)
    assert np.abs(Minv - ref).max() <= 1e-14 * np.abs(ref).max() * 11
    assert np.abs(Minv @ M - np.eye(11)).max() <= 1e-13


def test_zero_like_is_zero():
    Z, A = _fem(12, 8, seed=2)
    O = zero_like(Z)
    assert max(O.V.rank) == 0 and max(O.W.rank) == 0
    assert not O.dense().any()
    assert O.blocks is Z.blocks


@pytest.mark.parametrize("N,leaf", [(12, 8), (16, 16)])
def test_inverse_without_truncation_is_dense_inverse(N, leaf):
    Z, A = _fem(N, leaf, seed=N + 1)
    C, info = inverse(Z.copy(), 0.0, cap=None)
    ref = np.linalg.inv(A)
    assert np.linalg.norm(C.dense() - ref) <= 1e-12 * np.linalg.norm(ref)
    assert info["updates"] > 0


def test_inverse_truncated_is_a_preconditioner():
    Z, A = _fem(16, 16, seed=3)
    C, info = inverse(Z.copy(), 1e-4)
    D = C.dense()
    n = A.shape[0]
    err = np.linalg.norm(np.eye(n) - D @ A, 2)
    assert 0 < err <= 1e-2
    ref = np.linalg.inv(A)
    assert np.linalg.norm(D - ref) <= 1e-4 * np.linalg.norm(ref)
    b = np.random.default_rng(1).standard_normal(n)
    x, it = pcg(lambda v: A @ v, b, lambda r: D @ r, 1e-10)
    assert it <= 5 and np.linalg.norm(A @ x - b) <= 1e-9 * np.linalg.norm(b)
