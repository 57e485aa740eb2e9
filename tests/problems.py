"""Seeded H^2 test problems built on the oracle side (test helper).

The random draws come from ``synth`` in the canonical orders; the structure
comes from the oracle's own tree builder.  The library builds its own tree
and receives the same draws (see ``tests/libside.py``).
"""
from __future__ import annotations

import numpy as np

import synth
from oracle.h2 import ClusterBasis, H2Matrix
from oracle.tree import BlockTree, ClusterTree


def draw_matrix(tree_sizes, leaf_ids, sibling_pairs, n_clusters, adm_shapes, near_shapes, k, seed,
                coupling_scale=None, near_scale=1.0 / 16):
    """Random draws for an H^2 matrix of constant rank k (canonical layouts).

    Stream use: ``bases`` gives V then W; ``couplings`` gives the coupling
    matrices (N(0,1) * coupling_scale, default 1/k) and then the nearfield
    blocks (N(0,1) * near_scale).
    """
    st = synth.streams(seed)
    leaf_sizes = [(t, tree_sizes[t]) for t in leaf_ids]
    V = synth.nested_orthonormal_bases(st["bases"], leaf_sizes, sibling_pairs, n_clusters, k)
    W = synth.nested_orthonormal_bases(st["bases"], leaf_sizes, sibling_pairs, n_clusters, k)
    scale = 1.0 / k if coupling_scale is None else coupling_scale
    S = synth.gaussian_couplings(st["couplings"], len(adm_shapes), k, scale)
    N = synth.gaussian_nearfield(st["couplings"], near_shapes, near_scale)
    return dict(V=V, W=W, S=S, N=N, streams=st)


def oracle_problem(N: int, k: int, seed: int, leaf: int = 32, eta: float = 2.0,
                   coupling_scale=None, points=None):
    """Oracle H^2 matrix on the N x N grid of cell centres (or on ``points``)
    with rank k."""
    pts = synth.grid_points_2d(N) if points is None else np.ascontiguousarray(points, dtype=np.float64)
    ct = ClusterTree(pts, leaf)
    bt = BlockTree(ct, ct, eta)
    leaf_ids = [t for t in range(ct.n_clusters) if ct.is_leaf(t)]
    pairs = [tuple(ct.sons[t]) for t in range(ct.n_clusters) if ct.sons[t]]
    adm_shapes = [(k, k)] * len(bt.admissible)
    near_shapes = [(ct.size[bt.row[b]], ct.size[bt.col[b]]) for b in bt.inadmissible]
    d = draw_matrix(ct.size, leaf_ids, pairs, ct.n_clusters, adm_shapes, near_shapes, k, seed,
                    coupling_scale)
    V = ClusterBasis.from_canonical(ct, *d["V"])
    W = ClusterBasis.from_canonical(ct, *d["W"])
    Z = H2Matrix(bt, V, W)
    Z.set_couplings(d["S"])
    Z.set_nearfield(d["N"])
    return Z, d["streams"], pts


def draw_updates(Z: H2Matrix, st, count: int, u: int, candidates=None):
    """Update blocks (uniform over ``candidates``, default the admissible
    leaves) and their factors A_j, B_j ~ N(0,1)."""
    bt = Z.blocks
    cand = bt.admissible if candidates is None else candidates
    blocks = synth.choose_blocks(st["blocks"], cand, count)
    rows = [Z.V.tree.size[bt.row[b]] for b in blocks]
    cols = [Z.W.tree.size[bt.col[b]] for b in blocks]
    A, B = synth.update_factors(st["ab"], rows, cols, u)
    return [int(b) for b in blocks], A, B


def embed(Z: H2Matrix, b0: int, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Dense n x n matrix (tree order) that is A B^* on the block b0, 0 elsewhere."""
    bt = Z.blocks
    t0, s0 = bt.row[b0], bt.col[b0]
    out = np.zeros((Z.V.tree.n, Z.W.tree.n))
    r0, c0 = Z.V.tree.offset[t0], Z.W.tree.offset[s0]
    out[r0:r0 + A.shape[0], c0:c0 + B.shape[0]] = A @ B.T
    return out


def draw_matrix_general(sizes, sons, adm_rc, near_shapes, k, seed, coupling_scale=None, near_scale=1.0 / 16):
    """Like ``draw_matrix`` with ranks capped by the cluster sizes
    (``synth.nested_orthonormal_bases_general``); adm_rc = (row, col)
    cluster of every admissible block in block order."""
    st = synth.streams(seed)
    V = synth.nested_orthonormal_bases_general(st["bases"], sizes, sons, k)
    W = synth.nested_orthonormal_bases_general(st["bases"], sizes, sons, k)
    scale = 1.0 / max(k, 1) if coupling_scale is None else coupling_scale
    shapes = [(int(V[0][t]), int(W[0][s])) for t, s in adm_rc]
    S = synth.gaussian_blocks(st["couplings"], shapes, scale)
    N = synth.gaussian_nearfield(st["couplings"], near_shapes, near_scale)
    return dict(V=V, W=W, S=S, N=N, streams=st)


def oracle_problem_general(points, k, seed, leaf, eta=2.0):
    """Oracle H^2 matrix on arbitrary points with ranks capped by the sizes."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    ct = ClusterTree(pts, leaf)
    bt = BlockTree(ct, ct, eta)
    sons = [tuple(ct.sons[t]) if ct.sons[t] else None for t in range(ct.n_clusters)]
    adm_rc = [(bt.row[b], bt.col[b]) for b in bt.admissible]
    near_shapes = [(ct.size[bt.row[b]], ct.size[bt.col[b]]) for b in bt.inadmissible]
    d = draw_matrix_general(ct.size, sons, adm_rc, near_shapes, k, seed)
    V = ClusterBasis.from_canonical(ct, *d["V"])
    W = ClusterBasis.from_canonical(ct, *d["W"])
    Z = H2Matrix(bt, V, W)
    Z.set_couplings(d["S"])
    Z.set_nearfield(d["N"])
    return Z, d["streams"], pts


def block_triples(bt, ct):
    """(x, y, z) = ((t,s), (s,r), (t,r)) all blocks of the tree, one per
    combination of kinds."""
    where = {(bt.row[b], bt.col[b]): b for b in range(bt.n_blocks)}
    seen = {}
    for x in range(bt.n_blocks):
        t, s = bt.row[x], bt.col[x]
        for y in range(bt.n_blocks):
            if bt.row[y] != s:
                continue
            r = bt.col[y]
            z = where.get((t, r))
            if z is None:
                continue
            key = (bt.kind[x], bt.kind[y], bt.kind[z])
            if key not in seen and ct.size[t] <= 200 and ct.size[r] <= 200:
                seen[key] = (x, y, z)
    return seen
