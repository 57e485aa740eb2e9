"""P1 finite-element stiffness matrices and their H^2 form (oracle; test
infrastructure only).

The model problem of the paper's experiments (Section 7, first model
problem; the PDE is stated in the introduction): -div(sigma grad u) = f on
the unit square (or cube), u = 0 on the boundary, piecewise linear nodal
basis functions on a regular mesh.  The paper uses sigma = 1; here sigma is
piecewise constant on an M x M (x M) checkerboard.  Readings (the paper
leaves these open):

* nodes x = (i/N, j/N[, k/N]); the interior nodes i, j, k = 1..N-1 are the
  unknowns, numbered x fastest; boundary nodes are eliminated (Dirichlet);
* 2D: every cell [i, i+1] x [j, j+1] is split along its diagonal from
  (i, j) to (i+1, j+1) into two triangles;
* 3D: every cell is split into Kuhn's six tetrahedra, one per order of the
  three axes, all sharing the cell's main diagonal;
* sigma_e = the checker value at the element's centroid: index
  floor(M * x_c) per axis, clamped to M - 1; the checker array is ordered
  x fastest;
* the element matrix of a simplex e is sigma_e |e| G G^*, with G the
  gradients of the barycentric coordinates (rows); an entry below 1e-12
  of the element's largest diagonal entry is set to zero: its exact value
  is zero (orthogonal gradients, the edge opposite a right angle), and the
  gradients of rounded node coordinates only leave noise of ~1e-17 there,
  which differs with the order of the arithmetic and, through the
  block-relative truncation of the factorisation, would turn into rank-one
  updates of rounding-level blocks.

The H^2 form (Section 2): cluster tree of the interior nodes with support
boxes (node box padded by h = 1/N per side), block tree with
admissibility max(diam) <= eta dist; every admissible block of the
stiffness matrix is then exactly zero, so the H^2 matrix has row and column
bases of rank 0 and the nonzeros live in the dense inadmissible leaves.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .h2 import ClusterBasis, H2Matrix
from .tree import BlockTree, ClusterTree


def _simplices(N: int, dim: int):
    """Vertex grid indices (multi-indices) of every simplex of the mesh."""
    cells = np.array(list(itertools.product(range(N), repeat=dim)))[:, ::-1]   # x fastest
    if dim == 2:
        # (i,j),(i+1,j),(i+1,j+1) and (i,j),(i+1,j+1),(i,j+1)
        loc = [((0, 0), (1, 0), (1, 1)), ((0, 0), (1, 1), (0, 1))]
    elif dim == 3:
        loc = []
        for order in itertools.permutations(range(3)):
            v = [0, 0, 0]
            path = [tuple(v)]
            for a in order:
                v[a] += 1
                path.append(tuple(v))
            loc.append(tuple(path))
    else:
        raise ValueError("dim must be 2 or 3")
    out = []
    for c in cells:
        for simplex in loc:
            out.append([tuple(c + np.array(v)) for v in simplex])
    return out


def stiffness(N: int, dim: int, sigma: np.ndarray, M: int):
    """Stiffness matrix (scipy CSR, interior nodes only) and the interior
    node coordinates (n x dim, rows in the unknowns' order)."""
    sigma = np.asarray(sigma, dtype=np.float64).ravel()
    assert sigma.size == M ** dim
    h = 1.0 / N
    nside = N + 1
    rows, cols, vals = [], [], []
    for simplex in _simplices(N, dim):
        X = np.array(simplex, dtype=np.float64) * h              # (dim+1) x dim
        J = (X[1:] - X[0]).T                                       # dim x dim
        vol = abs(np.linalg.det(J)) / (2.0 if dim == 2 else 6.0)
        Ginv = np.linalg.inv(J)                                    # rows: grad of lambda_1..dim
        G = np.vstack([-Ginv.sum(axis=0), Ginv])                   # (dim+1) x dim
        xc = X.mean(axis=0)
        idx = np.minimum((M * xc).astype(np.int64), M - 1)
        flat = idx[0] + M * idx[1] + (M * M * idx[2] if dim == 3 else 0)
        Ke = sigma[flat] * vol * (G @ G.T)
        # an entry whose exact value is zero (two vertices whose gradients
        # are orthogonal: the edge opposite a right angle) comes out of the
        # rounded gradients as noise; it is zero
        Ke[np.abs(Ke) <= 1e-12 * np.abs(np.diag(Ke)).max()] = 0.0
        glob = [sum(v[a] * nside ** a for a in range(dim)) for v in simplex]
        for a in range(dim + 1):
            for b in range(dim + 1):
                rows.append(glob[a])
                cols.append(glob[b])
                vals.append(Ke[a, b])
    full = sp.coo_matrix((vals, (rows, cols)), shape=(nside ** dim,) * 2).tocsr()
    # interior nodes, x fastest
    grid = np.array(list(itertools.product(range(1, N), repeat=dim)))[:, ::-1]
    keep = (grid * (nside ** np.arange(dim))).sum(axis=1)
    K = full[keep][:, keep].tocsr()
    K.sum_duplicates()
    return K, grid.astype(np.float64) * h


def h2_from_sparse(K, points: np.ndarray, leaf_size: int, eta: float, pad: float) -> H2Matrix:
    """The H^2 matrix of a sparse matrix whose admissible blocks vanish:
    rank-0 bases, empty couplings, nearfield leaves copied in tree order."""
    ct = ClusterTree(points, leaf_size, pad)
    bt = BlockTree(ct, ct, eta)
    Kp = K[ct.perm][:, ct.perm].tocsr()
    V, W = ClusterBasis(ct), ClusterBasis(ct)
    for cb in (V, W):
        for t in range(ct.n_clusters):
            if ct.is_leaf(t):
                cb.leaf[t] = np.zeros((ct.size[t], 0))
            if t != 0:
                cb.transfer[t] = np.zeros((0, 0))
    Z = H2Matrix(bt, V, W)
    for b in bt.admissible:
        t, s = bt.row[b], bt.col[b]
        blk = Kp[ct.offset[t]:ct.offset[t] + ct.size[t], ct.offset[s]:ct.offset[s] + ct.size[s]]
        if blk.nnz and np.any(blk.data != 0.0):
            raise ValueError("admissible block %d of the sparse matrix is not zero" % b)
        Z.S[b] = np.zeros((0, 0))
    for b in bt.inadmissible:
        t, s = bt.row[b], bt.col[b]
        Z.N[b] = Kp[ct.offset[t]:ct.offset[t] + ct.size[t], ct.offset[s]:ct.offset[s] + ct.size[s]].toarray()
    return Z
