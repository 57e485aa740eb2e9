"""Library-side construction of the seeded test problems (test helper).

The library builds its own trees; the random draws come from ``synth`` in
the canonical orders, with the counts taken from the library's trees.
"""
from __future__ import annotations

import numpy as np

import synth
from paper_1402_5056_gb300 import binding as b
from problems import draw_matrix, draw_matrix_general


def structure(Z):
    tc = b.h2_tree_clusters(Z)
    tb = b.h2_tree_blocks(Z)
    nc = len(tc["offset"])
    leaf_ids = [t for t in range(nc) if tc["son0"][t] < 0]
    pairs = [(int(tc["son0"][t]), int(tc["son1"][t])) for t in range(nc) if tc["son0"][t] >= 0]
    adm = [i for i in range(len(tb["kind"])) if tb["kind"][i] == 1]
    near = [i for i in range(len(tb["kind"])) if tb["kind"][i] == 2]
    return tc, tb, leaf_ids, pairs, adm, near


def lib_problem(ctx, N: int, k: int, seed: int, leaf: int = 32, eta: float = 2.0, kcap=None,
                coupling_scale=None, points=None):
    """Library H^2 matrix with the same draws as ``problems.oracle_problem``."""
    pts = synth.grid_points_2d(N) if points is None else np.ascontiguousarray(points, dtype=np.float64)
    Z = b.h2_matrix_create(ctx, pts, leaf, eta, 0.0, kcap or max(k, 1))
    tc, tb, leaf_ids, pairs, adm, near = structure(Z)
    near_shapes = [(int(tc["size"][tb["row"][i]]), int(tc["size"][tb["col"][i]])) for i in near]
    d = draw_matrix(tc["size"], leaf_ids, pairs, len(tc["offset"]), [(k, k)] * len(adm), near_shapes, k,
                    seed, coupling_scale)
    if ctx is not None:
        b.h2_set_basis(ctx, Z, 0, *d["V"])
        b.h2_set_basis(ctx, Z, 1, *d["W"])
        b.h2_set_couplings(ctx, Z, d["S"])
        b.h2_set_nearfield(ctx, Z, d["N"])
    return Z, d["streams"], pts


def to_oracle(ctx, Z, like):
    """Download the library matrix into the oracle's containers (for dense
    comparison); ``like`` is an oracle H2Matrix with the identical trees."""
    from oracle.h2 import ClusterBasis, H2Matrix
    V = ClusterBasis.from_canonical(like.V.tree, *b.h2_get_basis(ctx, Z, 0))
    W = ClusterBasis.from_canonical(like.W.tree, *b.h2_get_basis(ctx, Z, 1))
    out = H2Matrix(like.blocks, V, W)
    out.set_couplings(b.h2_get_couplings(ctx, Z))
    out.set_nearfield(b.h2_get_nearfield(ctx, Z))
    return out


def lib_problem_general(ctx, points, k, seed, leaf, eta=2.0, kcap=32):
    """Library H^2 matrix with the draws of ``problems.oracle_problem_general``."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    Z = b.h2_matrix_create(ctx, pts, leaf, eta, 0.0, kcap)
    tc, tb, leaf_ids, pairs, adm, near = structure(Z)
    nc = len(tc["offset"])
    sons = [(int(tc["son0"][t]), int(tc["son1"][t])) if tc["son0"][t] >= 0 else None for t in range(nc)]
    adm_rc = [(int(tb["row"][i]), int(tb["col"][i])) for i in adm]
    near_shapes = [(int(tc["size"][tb["row"][i]]), int(tc["size"][tb["col"][i]])) for i in near]
    d = draw_matrix_general([int(x) for x in tc["size"]], sons, adm_rc, near_shapes, k, seed)
    b.h2_set_basis(ctx, Z, 0, *d["V"])
    b.h2_set_basis(ctx, Z, 1, *d["W"])
    b.h2_set_couplings(ctx, Z, d["S"])
    b.h2_set_nearfield(ctx, Z, d["N"])
    return Z, d["streams"], pts
