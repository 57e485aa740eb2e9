"""Pins of the oracle's finite-element matrices (oracle.fem) -- CPU.

Against what the mathematics fixes, never the oracle's own formula:

* constant sigma: the P1 stiffness matrix on the diagonal-split square grid
  is the five-point stencil sigma (4, -1) and on Kuhn's tetrahedra of the
  cube the seven-point stencil sigma h (6, -1) (Kronecker sums of the 1-D
  second difference);
* variable sigma in 2D: the cotangent formula K_ab = -1/2 sum_e sigma_e
  cot(angle opposite ab in e), K_aa = -(sum of the row's other entries in
  the matrix before the boundary nodes are removed), assembled edge by edge;
* variable sigma in 3D: element matrices from gradients obtained by solving
  each tetrahedron's 4 x 4 interpolation system, summed element by element;
* row sums zero away from the boundary, symmetry, positive definiteness;
* the H^2 form: dense assembly equals the permuted matrix, every admissible
  block of the stiffness matrix is zero (support boxes), ranks 0.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle.fem import h2_from_sparse, stiffness


def _second_difference(n):
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()


def test_constant_sigma_2d_is_five_point_stencil():
    N, s = 7, 3.5
    K, _ = stiffness(N, 2, np.array([s]), 1)
    T, I = _second_difference(N - 1), sp.identity(N - 1)
    ref = s * (sp.kron(I, T) + sp.kron(T, I))
    assert abs(K - ref).max() <= 1e-13 * s


def test_constant_sigma_3d_is_seven_point_stencil():
    N, s = 5, 0.7
    K, _ = stiffness(N, 3, np.array([s]), 1)
    T, I = _second_difference(N - 1), sp.identity(N - 1)
    ref = s * (1.0 / N) * (sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I))
    assert abs(K - ref).max() <= 1e-13 * s


def _cotangent_2d(N, sigma, M):
    """Stiffness matrix by the cotangent formula, edge by edge (2D)."""
    nn = N + 1
    full = np.zeros((nn * nn, nn * nn))
    idx = lambda i, j: i + nn * j
    for j in range(N):
        for i in range(N):
            for tri in (((i, j), (i + 1, j), (i + 1, j + 1)), ((i, j), (i + 1, j + 1), (i, j + 1))):
                P = [np.array(v, dtype=float) / N for v in tri]
                c = sum(P) / 3.0
                sg = sigma[min(int(M * c[0]), M - 1) + M * min(int(M * c[1]), M - 1)]
                for a in range(3):
                    b_, o = (a + 1) % 3, (a + 2) % 3
                    u, v = P[a] - P[o], P[b_] - P[o]
                    cot = float(u @ v) / abs(u[0] * v[1] - u[1] * v[0])
                    ia, ib = idx(*tri[a]), idx(*tri[b_])
                    full[ia, ib] -= 0.5 * sg * cot
                    full[ib, ia] -= 0.5 * sg * cot
    np.fill_diagonal(full, 0.0)
    np.fill_diagonal(full, -full.sum(axis=1))
    keep = [idx(i, j) for j in range(1, N) for i in range(1, N)]
    return full[np.ix_(keep, keep)]


@pytest.mark.parametrize("N,M", [(6, 3), (8, 4), (5, 2)])
def test_variable_sigma_2d_cotangent_formula(N, M):
    sigma = synth.checker_sigma(np.random.default_rng(N + M), M, 2)
    K, _ = stiffness(N, 2, sigma, M)
    ref = _cotangent_2d(N, sigma, M)
    assert np.abs(K.toarray() - ref).max() <= 1e-12 * np.abs(ref).max()


def _brute_3d(N, sigma, M):
    nn = N + 1
    full = np.zeros((nn ** 3, nn ** 3))
    idx = lambda v: v[0] + nn * v[1] + nn * nn * v[2]
    for k, j, i in itertools.product(range(N), repeat=3):
        for order in itertools.permutations(range(3)):
            verts = [(i, j, k)]
            v = [i, j, k]
            for a in order:
                v[a] += 1
                verts.append(tuple(v))
            X = np.array(verts, dtype=float) / N
            # gradients from the interpolation system [1 x y z] c = e_a
            Msys = np.hstack([np.ones((4, 1)), X])
            C = np.linalg.solve(Msys, np.eye(4))          # column a = coefficients of lambda_a
            G = C[1:].T                                   # row a = grad lambda_a
            vol = abs(np.linalg.det(X[1:] - X[0])) / 6.0
            c = X.mean(axis=0)
            f = [min(int(M * c[q]), M - 1) for q in range(3)]
            sg = sigma[f[0] + M * f[1] + M * M * f[2]]
            ids = [idx(w) for w in verts]
            for a in range(4):
                for b_ in range(4):
                    full[ids[a], ids[b_]] += sg * vol * float(G[a] @ G[b_])
    keep = [idx((i, j, k)) for k in range(1, N) for j in range(1, N) for i in range(1, N)]
    return full[np.ix_(keep, keep)]


def test_variable_sigma_3d_element_sum():
    N, M = 4, 2
    sigma = synth.checker_sigma(np.random.default_rng(7), M, 3)
    K, _ = stiffness(N, 3, sigma, M)
    ref = _brute_3d(N, sigma, M)
    assert np.abs(K.toarray() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dim,N,M", [(2, 10, 4), (3, 6, 2)])
def test_row_sums_symmetry_definiteness(dim, N, M):
    sigma = synth.checker_sigma(np.random.default_rng(dim * N), M, dim)
    K, pts = stiffness(N, dim, sigma, M)
    D = K.toarray()
    assert np.abs(D - D.T).max() <= 1e-14 * np.abs(D).max()
    assert np.linalg.eigvalsh(D).min() > 0
    h = 1.0 / N
    inner = np.all((pts > 1.5 * h) & (pts < 1 - 1.5 * h), axis=1)
    assert inner.any()
    assert np.abs(D[inner].sum(axis=1)).max() <= 1e-12 * np.abs(D).max()


@pytest.mark.parametrize("dim,N,leaf", [(2, 32, 32), (2, 17, 8), (3, 10, 16)])
def test_h2_form_of_the_fem_matrix(dim, N, leaf):
    sigma = synth.checker_sigma(np.random.default_rng(1), 2, dim)
    K, pts = stiffness(N, dim, sigma, 2)
    Z = h2_from_sparse(K, pts, leaf, 2.0, 1.0 / N)
    perm = Z.V.tree.perm
    assert np.array_equal(Z.dense(), K[perm][:, perm].toarray())
    assert max(Z.V.rank) == 0 and len(Z.blocks.admissible) > 0
    # a nonzero planted in an admissible block is refused
    bt, tr = Z.blocks, Z.V.tree
    b0 = bt.admissible[len(bt.admissible) // 2]
    i, j = perm[tr.offset[bt.row[b0]]], perm[tr.offset[bt.col[b0]]]
    K2 = K.tolil()
    K2[i, j] = 1.0
    with pytest.raises(ValueError):
        h2_from_sparse(K2.tocsr(), pts, leaf, 2.0, 1.0 / N)


def test_checker_sigma_range():
    s = synth.checker_sigma(np.random.default_rng(0), 16, 2)
    assert s.shape == (256,) and s.min() >= 1e-2 and s.max() <= 1e2
    assert math.log10(s.max() / s.min()) > 3.5
