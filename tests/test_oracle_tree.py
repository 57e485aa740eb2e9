"""Pins of the oracle's cluster and block trees (Section 2 definitions).

Checked against facts fixed by the definitions and brute force, never by
re-running the oracle's own construction.
"""
import itertools
import math

import numpy as np
import pytest

import synth
from oracle.tree import BlockTree, ClusterTree


def _box(points):
    return points.min(axis=0), points.max(axis=0)


@pytest.mark.parametrize("N,leaf", [(16, 8), (24, 32), (32, 32), (13, 5), (-1, 10)])
def test_leaf_labels_partition_index_set(N, leaf):
    if N > 0:
        pts = synth.grid_points_2d(N)
    else:
        N = 30
        pts = np.random.default_rng(4).uniform(size=(N * N, 2))
    ct = ClusterTree(pts, leaf)
    # Def. "Cluster tree": root labelled by I, sons partition the father
    assert sorted(ct.idx[0].tolist()) == list(range(N * N))
    for t in range(ct.n_clusters):
        if ct.sons[t]:
            a, b = ct.sons[t]
            assert len(ct.idx[a]) + len(ct.idx[b]) == len(ct.idx[t])
            assert set(ct.idx[a].tolist()) | set(ct.idx[b].tolist()) == set(ct.idx[t].tolist())
            assert not set(ct.idx[a].tolist()) & set(ct.idx[b].tolist())
            assert ct.father[a] == t and ct.father[b] == t
            assert ct.level[a] == ct.level[t] + 1
            # labels are contiguous in tree order and the sons follow each other
            assert ct.offset[a] == ct.offset[t]
            assert ct.offset[b] == ct.offset[t] + ct.size[a]
        else:
            assert ct.size[t] <= leaf
    # leaves partition I; perm is a permutation; labels are contiguous in it
    assert sorted(ct.perm.tolist()) == list(range(N * N))
    for t in range(ct.n_clusters):
        seg = ct.perm[ct.offset[t]:ct.offset[t] + ct.size[t]]
        assert sorted(seg.tolist()) == sorted(ct.idx[t].tolist())
    # depth-first preorder numbering: every son has a larger id than its father
    assert all(ct.father[t] < t for t in range(1, ct.n_clusters))


def _integer_grid(n):
    """n x n integer points: box midpoints fall exactly on points."""
    i, j = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64))
    return np.stack([j.ravel(), i.ravel()], axis=1)


@pytest.mark.parametrize("case", ["grid24", "integer13", "random3d"])
def test_bisection_geometry_brute_force(case):
    if case == "grid24":
        pts, leaf = synth.grid_points_2d(24), 32
    elif case == "integer13":
        pts, leaf = _integer_grid(13), 8
    else:
        pts, leaf = np.random.default_rng(8).uniform(size=(700, 3)), 16
    ct = ClusterTree(pts, leaf)
    on_mid = 0
    for t in range(ct.n_clusters):
        P = pts[ct.idx[t]]
        lo, hi = _box(P)
        if not ct.sons[t]:
            continue
        ext = hi - lo
        axis = int(np.flatnonzero(ext == ext.max())[0])   # lowest longest axis
        mid = 0.5 * (lo[axis] + hi[axis])
        a, b = ct.sons[t]
        assert np.all(pts[ct.idx[a]][:, axis] < mid)
        assert np.all(pts[ct.idx[b]][:, axis] >= mid)
        on_mid += int(np.sum(pts[ct.idx[t]][:, axis] == mid))
        # stable order inside the sons
        assert np.all(np.diff(np.searchsorted(ct.idx[t], ct.idx[a])) > 0) or len(ct.idx[a]) < 2
    if case == "integer13":
        assert on_mid > 0          # the rule for points on the midpoint was exercised


def test_power_of_two_grid_is_perfect():
    # 256 x 256 cell centres, leaf 32: midpoints split every box exactly in
    # half, so the tree is perfect: 2^11 leaves of 32, 2^12 - 1 clusters.
    pts = synth.grid_points_2d(256)
    ct = ClusterTree(pts, 32)
    assert ct.n_clusters == 4095
    leaves = [t for t in range(ct.n_clusters) if not ct.sons[t]]
    assert len(leaves) == 2048
    assert all(ct.size[t] == 32 and ct.level[t] == 11 for t in leaves)
    assert ct.subtree_count[0] == 4095


def _brute_adm(P1, P2, eta):
    lo1, hi1 = _box(P1)
    lo2, hi2 = _box(P2)
    d1 = math.dist(lo1, hi1)
    d2 = math.dist(lo2, hi2)
    gap = [max(0.0, lo2[i] - hi1[i], lo1[i] - hi2[i]) for i in range(len(lo1))]
    dist = math.sqrt(sum(g * g for g in gap))
    return dist > 0 and max(d1, d2) <= eta * dist


@pytest.mark.parametrize("N,leaf,eta", [(16, 8, 2.0), (24, 16, 2.0), (32, 32, 1.0),
                                         (-1, 12, 2.0), (-2, 10, 1.5)])
def test_block_tree_partition_and_admissibility(N, leaf, eta):
    if N > 0:
        pts = synth.grid_points_2d(N)
    else:   # ragged trees: leaves at several levels pair with larger clusters
        pts = np.random.default_rng(-N).uniform(size=(600, -N + 1)) ** 2
    ct = ClusterTree(pts, leaf)
    bt = BlockTree(ct, ct, eta)
    n = len(pts)
    if N < 0:
        assert any(bt.kind[b] == BlockTree.NEAR and bool(ct.sons[bt.row[b]]) != bool(ct.sons[bt.col[b]])
                   for b in range(bt.n_blocks))
    cover = np.zeros((n, n), dtype=np.int32)
    for b in range(bt.n_blocks):
        t, s = bt.row[b], bt.col[b]
        adm = _brute_adm(pts[ct.idx[t]], pts[ct.idx[s]], eta)
        if bt.kind[b] == BlockTree.ADM:
            assert adm
        elif bt.kind[b] == BlockTree.NEAR:
            assert not adm and (not ct.sons[t] or not ct.sons[s])
        else:
            assert not adm and ct.sons[t] and ct.sons[s]
            # sons(b) = sons(t) x sons(s) in the stated order
            assert [(bt.row[c], bt.col[c]) for c in bt.sons[b]] == \
                list(itertools.product(ct.sons[t], ct.sons[s]))
        if bt.kind[b] != BlockTree.SUB:
            r0, c0 = ct.offset[t], ct.offset[s]
            cover[r0:r0 + ct.size[t], c0:c0 + ct.size[s]] += 1
    # the leaves partition I x I
    assert np.all(cover == 1)
    assert bt.row[0] == 0 and bt.col[0] == 0
    assert len(bt.admissible) > 0


def test_row_lists_match_definition():
    pts = synth.grid_points_2d(16)
    ct = ClusterTree(pts, 8)
    bt = BlockTree(ct, ct, 2.0)
    for t in range(ct.n_clusters):
        want = sorted(b for b in range(bt.n_blocks) if bt.kind[b] == BlockTree.ADM and bt.row[b] == t)
        assert sorted(bt.row_blocks[t]) == want
        want = sorted(b for b in range(bt.n_blocks) if bt.kind[b] == BlockTree.ADM and bt.col[b] == t)
        assert sorted(bt.col_blocks[t]) == want
