"""Host-side checks of libh2gb (no GPU needed).

* the shared library loads and exports every entry point ``include/h2gb.h``
  declares;
* the library's trees are bit-identical to the oracle's independent ones;
* the batch planner's task counts and factor layout follow the definitions
  of Section 5 (subtrees T_t0, T_s0 and the blocks whose row lies in T_t0 or
  whose column lies in T_s0).
"""
import os
import re

import numpy as np
import pytest

import synth
from layout import check_result_layout
from oracle.tree import BlockTree, ClusterTree

b = pytest.importorskip("paper_1402_5056_gb300.binding")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "h2gb.h")).read()
    declared = set(re.findall(r"\b(h2_[a-z0-9_]+)\s*\(", hdr))
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(b._lib, n)]
    assert not missing, missing
    assert declared == set(b.EXPORTS)


def _compare_trees(pts, leaf, eta):
    Z = b.h2_matrix_create(None, pts, leaf, eta, 0.0, 8)
    try:
        tc = b.h2_tree_clusters(Z)
        tb = b.h2_tree_blocks(Z)
        perm = b.h2_tree_permutation(Z)
    finally:
        b.h2_matrix_free(Z)
    ct = ClusterTree(pts, leaf)
    bt = BlockTree(ct, ct, eta)
    nc = ct.n_clusters
    assert len(tc["offset"]) == nc
    np.testing.assert_array_equal(tc["offset"], ct.offset)
    np.testing.assert_array_equal(tc["size"], ct.size)
    np.testing.assert_array_equal(tc["father"], ct.father)
    np.testing.assert_array_equal(tc["level"], ct.level)
    np.testing.assert_array_equal(tc["subtree"], ct.subtree_count)
    np.testing.assert_array_equal(tc["son0"], [s[0] if s else -1 for s in ct.sons])
    np.testing.assert_array_equal(tc["son1"], [s[1] if s else -1 for s in ct.sons])
    np.testing.assert_array_equal(perm, ct.perm)
    assert len(tb["row"]) == bt.n_blocks
    np.testing.assert_array_equal(tb["row"], bt.row)
    np.testing.assert_array_equal(tb["col"], bt.col)
    np.testing.assert_array_equal(tb["kind"], bt.kind)
    np.testing.assert_array_equal(tb["father"], bt.father)


@pytest.mark.parametrize("N,leaf,eta", [(16, 8, 2.0), (24, 32, 2.0), (32, 32, 2.0), (37, 20, 1.5)])
def test_trees_bit_identical_on_grids(N, leaf, eta):
    _compare_trees(synth.grid_points_2d(N), leaf, eta)


@pytest.mark.parametrize("seed,dim", [(0, 2), (1, 3), (2, 1)])
def test_trees_bit_identical_on_random_points(seed, dim):
    pts = np.random.default_rng(seed).uniform(size=(1500, dim))
    _compare_trees(pts, 24, 2.0)


def test_trees_bit_identical_isolated_update_workload():
    # 256 x 256 grid, leaf 32, eta 2 (the isolated-update benchmark structure)
    _compare_trees(synth.grid_points_2d(256), 32, 2.0)


def test_host_plan_counts_and_layout():
    N, leaf, u = 32, 16, 3
    pts = synth.grid_points_2d(N)
    Z = b.h2_matrix_create(None, pts, leaf, 2.0, 0.0, 8)
    ct = ClusterTree(pts, leaf)
    bt = BlockTree(ct, ct, 2.0)
    rng = np.random.default_rng(3)
    blocks = list(rng.choice(bt.admissible, 7)) + [0, bt.inadmissible[3]]
    P = b.h2_batch_create(None, Z, blocks, u)
    try:
        st = b.h2_batch_stats(None, P, flops=False)
        items = 0
        tasks = 0
        offA = offB = 0
        for j, blk in enumerate(blocks):
            t0, s0 = bt.row[blk], bt.col[blk]
            Tt, Ts = set(ct.descendants(t0)), set(ct.descendants(s0))
            items += len(Tt) + len(Ts)
            tasks += sum(1 for c in bt.admissible if bt.row[c] in Tt or bt.col[c] in Ts)
            lay = b.h2_batch_factor_layout(P, j)
            assert lay == (ct.size[t0], offA, ct.size[s0], offB)
            offA += ct.size[t0] * u
            offB += ct.size[s0] * u
        assert st["cluster_tasks"] == items
        assert st["block_tasks"] == tasks
        assert b.h2_batch_factor_sizes(P) == (offA, offB)
    finally:
        b.h2_batch_free(P)
        b.h2_matrix_free(Z)


def test_invalid_arguments_rejected():
    pts = synth.grid_points_2d(8)
    with pytest.raises(b.H2Error) as e:
        b.h2_matrix_create(None, pts, 0, 2.0)
    assert e.value.status == 1
    Z = b.h2_matrix_create(None, pts, 8, 2.0, 0.0, 4)
    try:
        with pytest.raises(b.H2Error):
            b.h2_batch_create(None, Z, [10 ** 6], 2)
        with pytest.raises(b.H2Error):
            b.h2_batch_create(None, Z, [0], 0)
        with pytest.raises(b.H2Error):
            b.h2_batch_create(None, Z, [0], 32)
    finally:
        b.h2_matrix_free(Z)



@pytest.mark.parametrize("ragged", [False, True])
def test_host_result_layout_tiles_the_buffer(ragged):
    """The host result's layout on a planned batch (no GPU: every rank is 0,
    so one-sided couplings have empty pieces; the GPU host-result test runs
    the same check with ranks), the compact entry point's argument check,
    and the byte counts before any host execution."""
    pts = np.random.default_rng(2).uniform(size=(900, 3)) ** 2 if ragged else synth.grid_points_2d(32)
    Z = b.h2_matrix_create(None, pts, 16, 2.0, 0.0, 8)
    tb = b.h2_tree_blocks(Z)
    rng = np.random.default_rng(5)
    blocks = [int(x) for x in rng.choice(np.flatnonzero(np.asarray(tb["kind"]) == 1), 6)] + [0]
    P = b.h2_batch_create(None, Z, blocks, 3)
    try:
        regions = check_result_layout(b, P, Z, 3)
        assert {1, 2} <= regions
        with pytest.raises(b.H2Error):   # no context
            b.h2_batch_execute_host_compact(None, P, np.zeros(1), np.zeros(1), 1e-8)
        assert b.h2_batch_host_bytes(P) == (0, 0)
    finally:
        b.h2_batch_free(P)
        b.h2_matrix_free(Z)


def test_update_work_is_linear_in_the_subtrees():
    """Section 5: an update touches the clusters of T_t0 and T_s0 and the
    couplings of their block rows and columns, at most C_sp (#T_t0 + #T_s0)
    of them (C_sp = the most admissible blocks in one block row or column):
    the planner's task counts for single updates at every level, with
    equality for the cluster tasks."""
    pts = synth.grid_points_2d(64)
    Z = b.h2_matrix_create(None, pts, 16, 2.0, 0.0, 8)
    ct = ClusterTree(pts, 16)
    bt = BlockTree(ct, ct, 2.0)
    c_sp = max(max(len(r) for r in bt.row_blocks), max(len(c) for c in bt.col_blocks))
    by_level = {}
    for blk in bt.admissible + bt.inadmissible + [0]:
        by_level.setdefault(ct.level[bt.row[blk]], []).append(blk)
    rng = np.random.default_rng(11)
    ratios = []
    try:
        for lev, blks in sorted(by_level.items()):
            for blk in rng.choice(blks, min(4, len(blks)), replace=False):
                blk = int(blk)
                nt = len(ct.descendants(bt.row[blk])) + len(ct.descendants(bt.col[blk]))
                P = b.h2_batch_create(None, Z, [blk], 2)
                try:
                    st = b.h2_batch_stats(None, P, flops=False)
                finally:
                    b.h2_batch_free(P)
                assert st["cluster_tasks"] == nt
                assert st["block_tasks"] <= c_sp * nt
                ratios.append(st["block_tasks"] / nt)
        assert len(by_level) > 5 and max(ratios) <= c_sp
    finally:
        b.h2_matrix_free(Z)


def test_binding_rejects_short_host_buffers():
    """The binding checks a caller's output arrays before the library
    writes them (dtype, contiguity, length)."""
    pts = synth.grid_points_2d(16)
    Z = b.h2_matrix_create(None, pts, 8, 2.0, 0.0, 4)
    tb = b.h2_tree_blocks(Z)
    P = b.h2_batch_create(None, Z, [int(np.flatnonzero(np.asarray(tb["kind"]) == 1)[0])], 2)
    try:
        n = b.h2_batch_result_size(P)
        nt = b.h2_batch_stats(None, P, flops=False)["block_tasks"]
        for bad in (np.zeros(n - 1), np.zeros(n, np.float32), np.zeros((n, 2))[:, 0]):
            with pytest.raises(ValueError):
                b.h2_batch_execute_host(None, P, np.zeros(1), np.zeros(1), 1e-8, bad)
        with pytest.raises(ValueError):
            b.h2_batch_execute_host_compact(None, P, np.zeros(1), np.zeros(1), 1e-8, np.zeros(n),
                                            np.zeros(max(nt - 1, 0), np.int8))
        with pytest.raises(ValueError):
            b.h2_batch_execute_host_compact(None, P, np.zeros(1), np.zeros(1), 1e-8, np.zeros(n),
                                            np.zeros(nt, np.int32))
    finally:
        b.h2_batch_free(P)
        b.h2_matrix_free(Z)


def test_stats_of_the_structure():
    """h2_stats on a structure-only matrix: the counts of the oracle's trees,
    rank 0 everywhere, device bytes of the empty storage, value bytes of the
    nearfield alone."""
    pts = synth.grid_points_2d(24)
    Z = b.h2_matrix_create(None, pts, 16, 2.0, 0.0, 8)
    try:
        st = b.h2_stats(Z)
    finally:
        b.h2_matrix_free(Z)
    ct = ClusterTree(pts, 16)
    bt = BlockTree(ct, ct, 2.0)
    assert st["n"] == len(pts) and st["n_clusters"] == ct.n_clusters and st["n_blocks"] == bt.n_blocks
    assert st["n_admissible"] == len(bt.admissible) and st["n_inadmissible"] == len(bt.inadmissible)
    assert st["depth"] == max(ct.level)
    assert st["max_rank_rows"] == 0 and st["max_rank_cols"] == 0 and st["rank_sum_rows"] == 0
    assert st["max_rank_per_level"] == [0] * (st["depth"] + 1)
    near = sum(ct.size[bt.row[c]] * ct.size[bt.col[c]] for c in bt.inadmissible)
    assert st["value_bytes"] == 8 * near
    assert st["device_bytes"] == 0   # structure only: no device storage


def test_factorisation_entry_points_reject_missing_arguments():
    """The factorisations, solves and preconditioned CG refuse a missing
    context, matrix or vector with H2_EINVAL before any device work (no GPU
    is touched)."""
    import ctypes as C
    lib = b._lib
    pts = synth.grid_points_2d(8)
    Z = b.h2_matrix_create(None, pts, 8, 2.0, 0.0, 4)
    opt = b.options(eps=1e-4, leaf_size=8)
    x = np.zeros(64)
    try:
        for name in ("h2_lr_factor", "h2_chol_factor"):
            f = getattr(lib, name)
            assert f(None, Z, C.byref(opt), None) == 1
        arr = (C.c_void_p * 1)(Z)
        for name in ("h2_lr_factor_many", "h2_chol_factor_many"):
            f = getattr(lib, name)
            assert f(None, arr, 1, C.byref(opt), 0, None) == 1
        for name in ("h2_lr_solve", "h2_chol_solve"):
            assert getattr(lib, name)(None, Z, 1, x.ctypes.data, 64) == 1
        it, rr = C.c_int(), C.c_double()
        for name in ("h2_pcg", "h2_pcg_chol", "h2_pcg_inverse"):
            assert getattr(lib, name)(None, Z, Z, x.ctypes.data, x.ctypes.data, 1e-10, 10, C.byref(it),
                                      C.byref(rr)) == 1
        err = C.c_double()
        for name in ("h2_lr_error", "h2_chol_error"):
            assert getattr(lib, name)(None, Z, Z, x.ctypes.data, 5, C.byref(err)) == 1
    finally:
        b.h2_matrix_free(Z)
