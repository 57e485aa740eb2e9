"""Pins of the oracle's H^2 matrix-vector product (oracle/matvec.py).

Against the dense matrix assembled block by block through explicitly
expanded bases (H2Matrix.dense, Section 2 Eqs. (vsw) and (nested)), which
shares no step with the forward/backward transformations; several right-
hand sides at once; alpha, beta; rank-0 bases; a matrix after updates
(ranks differing between clusters).
"""
import numpy as np
import pytest

from oracle.matvec import matvec
from oracle.update import apply_delta, local_update
from problems import draw_updates, oracle_problem, oracle_problem_general


@pytest.mark.parametrize("N,k,leaf", [(20, 4, 16), (24, 6, 16), (32, 5, 32)])
def test_matvec_equals_dense(N, k, leaf):
    Zo, st, _ = oracle_problem(N, k, 301 + N, leaf)
    D = Zo.dense()
    rng = np.random.default_rng(N)
    X = rng.standard_normal((D.shape[1], 3))
    np.testing.assert_allclose(matvec(Zo, X), D @ X, rtol=0, atol=1e-12 * np.abs(D).sum(axis=1).max() * np.abs(X).max())
    x = X[:, 0]
    y = rng.standard_normal(D.shape[0])
    got = matvec(Zo, x, alpha=2.0, beta=-0.5, Y=y)
    np.testing.assert_allclose(got, 2.0 * (D @ x) - 0.5 * y, rtol=1e-12, atol=1e-12 * np.linalg.norm(D @ x))


def test_matvec_general_points_and_rank_zero():
    pts = np.random.default_rng(3).uniform(size=(400, 2))
    for k in (0, 5):
        Zo, _, _ = oracle_problem_general(pts, k, 307, 16)
        D = Zo.dense()
        X = np.random.default_rng(k).standard_normal((D.shape[1], 2))
        np.testing.assert_allclose(matvec(Zo, X), D @ X, rtol=0, atol=1e-12 * (np.abs(D).sum() + 1.0))


def test_matvec_after_updates_with_uneven_ranks():
    Zo, st, _ = oracle_problem(24, 5, 311, 16)
    blocks, A, B = draw_updates(Zo, st, 3, 2)
    Z = Zo
    for j, b0 in enumerate(blocks):
        Z = apply_delta(Z, local_update(Z, b0, A[j], B[j], 0.3))
    assert len(set(Z.V.rank)) > 1
    D = Z.dense()
    X = np.random.default_rng(5).standard_normal((D.shape[1], 4))
    np.testing.assert_allclose(matvec(Z, X), D @ X, rtol=0, atol=1e-11 * np.abs(D).sum(axis=1).max() * np.abs(X).max())
