"""Pins of the oracle's H^2 representation (oracle/h2.py): the canonical
host layouts (column-major matrices concatenated in cluster or block order,
as the C header states) and the dense assembly of Eq. (vsw) through the
nested bases of Eq. (nested), checked with unit entries whose dense image is
known in closed form.
"""
import numpy as np
import pytest

import synth
from oracle.h2 import ClusterBasis, H2Matrix
from oracle.tree import BlockTree, ClusterTree

K = 3


def _setup():
    pts = synth.grid_points_2d(16)
    ct = ClusterTree(pts, 8)
    bt = BlockTree(ct, ct, 2.0)
    return ct, bt


def _basis(ct, leaf_data=None, transfer_data=None, k=K):
    ranks = [k] * ct.n_clusters
    n_leaf = sum(ct.size[t] * k for t in range(ct.n_clusters) if not ct.sons[t])
    n_tr = (ct.n_clusters - 1) * k * k
    if leaf_data is None:
        leaf_data = np.zeros(n_leaf)
    if transfer_data is None:
        transfer_data = np.tile(np.eye(k).ravel(order="F"), ct.n_clusters - 1)
    return ClusterBasis.from_canonical(ct, ranks, leaf_data, transfer_data)


def _leaf_offsets(ct, k=K):
    off, pos = {}, 0
    for t in range(ct.n_clusters):
        if not ct.sons[t]:
            off[t] = pos
            pos += ct.size[t] * k
    return off, pos


def test_leaf_layout_unit_entry():
    """Leaf data entry off(t) + r + c #t is V_t[r, c]."""
    ct, _ = _setup()
    off, n = _leaf_offsets(ct)
    leaves = [t for t in range(ct.n_clusters) if not ct.sons[t]]
    t = leaves[5]
    r, c = 3, 2
    data = np.zeros(n)
    data[off[t] + r + c * ct.size[t]] = 1.0
    V = _basis(ct, data)
    want = np.zeros((ct.size[t], K))
    want[r, c] = 1.0
    np.testing.assert_array_equal(V.dense(t), want)


def test_transfer_layout_and_nesting():
    """Transfer data entry K*K*(t-1) + i + j K is E_t[i, j]; V_root
    restricted to t's rows is V_t E_t E_{t+} ... (Eq. (nested))."""
    ct, _ = _setup()
    off, n = _leaf_offsets(ct)
    leaves = [t for t in range(ct.n_clusters) if not ct.sons[t]]
    t = leaves[2]
    data = np.zeros(n)
    data[off[t] + 0 + 0 * ct.size[t]] = 1.0          # V_t = e_0 e_0^*
    tr = np.tile(np.eye(K).ravel(order="F"), ct.n_clusters - 1)
    i, j = 0, 2                                      # E_t = e_0 e_2^* (not symmetric)
    tr[K * K * (t - 1):K * K * t] = 0.0
    tr[K * K * (t - 1) + i + j * K] = 1.0
    V = _basis(ct, data, tr)
    # ancestors keep identity transfers: the root basis has a single 1 in
    # row (tree position of t's first index), column j
    want = np.zeros((ct.size[0], K))
    want[ct.offset[t], j] = 1.0
    np.testing.assert_array_equal(V.dense(0), want)


@pytest.mark.parametrize("which", [0, 7, -1])
def test_coupling_layout_and_block_assembly(which):
    """Coupling data entry pos(b) + i + j k_t is S_b[i, j]; the dense matrix
    is V_t S_b W_s^* on that block only (Eq. (vsw))."""
    ct, bt = _setup()
    off, n = _leaf_offsets(ct)
    rng = np.random.default_rng(3)
    V = _basis(ct, rng.standard_normal(n))
    W = _basis(ct, rng.standard_normal(n))
    Z = H2Matrix(bt, V, W)
    b = bt.admissible[which]
    data = np.zeros(len(bt.admissible) * K * K)
    pos = bt.admissible.index(b) * K * K
    i, j = 1, 2
    data[pos + i + j * K] = 1.0
    Z.set_couplings(data)
    Z.set_nearfield(np.zeros(sum(ct.size[bt.row[c]] * ct.size[bt.col[c]] for c in bt.inadmissible)))
    t, s = bt.row[b], bt.col[b]
    want = np.zeros((ct.n, ct.n))
    want[ct.offset[t]:ct.offset[t] + ct.size[t], ct.offset[s]:ct.offset[s] + ct.size[s]] = \
        np.outer(V.dense(t)[:, i], W.dense(s)[:, j])
    np.testing.assert_allclose(Z.dense(), want, rtol=0, atol=1e-14)


def test_nearfield_layout_unit_entry():
    """Nearfield data entry pos(b) + r + c #t is G|_b[r, c], placed at the
    block's tree-order position."""
    ct, bt = _setup()
    off, n = _leaf_offsets(ct)
    V = _basis(ct)
    Z = H2Matrix(bt, V, _basis(ct))
    Z.set_couplings(np.zeros(len(bt.admissible) * K * K))
    b = bt.inadmissible[4]
    t, s = bt.row[b], bt.col[b]
    pos = sum(ct.size[bt.row[c]] * ct.size[bt.col[c]] for c in bt.inadmissible[:4])
    total = sum(ct.size[bt.row[c]] * ct.size[bt.col[c]] for c in bt.inadmissible)
    r, c = 2, 5
    data = np.zeros(total)
    data[pos + r + c * ct.size[t]] = 1.0
    Z.set_nearfield(data)
    want = np.zeros((ct.n, ct.n))
    want[ct.offset[t] + r, ct.offset[s] + c] = 1.0
    np.testing.assert_array_equal(Z.dense(), want)
