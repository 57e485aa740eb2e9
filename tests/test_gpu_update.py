"""Parity of the CUDA local low-rank update with the CPU oracle (Section 5).

The library and the oracle build their own trees and receive the same
seeded draws; results are compared on the assembled matrices:

* small problems (n <= 1024): the whole updated matrix densely, relative
  Frobenius error <= 1e-10, and the new ranks;
* the isolated-update workload at full size (256 x 256 points, k = 16,
  rank-8 updates, eps = 1e-8): sampled updates, compared entry by entry on
  rows of T_t0 and columns of T_s0 (where the update acts) plus random
  entries elsewhere, and properties of the whole 4096-update batch.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

import synth  # noqa: E402
from blockwise import assert_blockwise_dense  # noqa: E402
from blockwise import blockwise_h2, leaf_blocks  # noqa: E402
from dense_ref import entries  # noqa: E402
from gpu_util import applied_delta, concat_factors, run_isolated  # noqa: E402
from libside import lib_problem, to_oracle  # noqa: E402
from oracle.tree import BlockTree  # noqa: E402
from oracle.update import apply_delta, local_update, sequential_batch  # noqa: E402
from problems import draw_updates, oracle_problem  # noqa: E402

TOL = 1e-10   # relative Frobenius error on assembled matrices


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_ctx_destroy(c)


def _extra(Zo, u, rng):
    bt = Zo.blocks
    sub = [c for c in range(1, bt.n_blocks) if bt.kind[c] == BlockTree.SUB]
    extra = [0, sub[len(sub) // 2], bt.inadmissible[len(bt.inadmissible) // 3]]
    A = [rng.standard_normal((Zo.V.tree.size[bt.row[c]], u)) for c in extra]
    B = [rng.standard_normal((Zo.W.tree.size[bt.col[c]], u)) for c in extra]
    return extra, A, B


def _rank_check(Zo, d, rV, rW):
    """Compare the new ranks unless the oracle's rank decision lies within
    1e-6 (relative, in the threshold) of flipping; returns 1 if compared."""
    if d["margin"] < 1e-6:
        return 0
    for t, r in d["V"]["rank"].items():
        assert rV[t] == r, ("row rank", t)
    for t, r in d["W"]["rank"].items():
        assert rW[t] == r, ("column rank", t)
    return 1


def _BW(got, ref, Zo, what):
    assert_blockwise_dense(got, ref, Zo.blocks, Zo.V.tree, Zo.W.tree, TOL, what)


@pytest.mark.parametrize("N,leaf,k,u,eps", [
    (24, 16, 6, 3, 1e-8),
    (24, 16, 6, 3, 0.5),
    (24, 16, 6, 3, 2.0),
    (32, 32, 8, 4, 1e-8),
    (32, 32, 8, 4, 1.0),
    (20, 10, 4, 5, 0.3),
])
def test_isolated_batch_matches_oracle_dense(ctx, N, leaf, k, u, eps):
    seed = 100 + N + k
    Zo, st, _ = oracle_problem(N, k, seed, leaf)
    blocks, A, B = draw_updates(Zo, st, 6, u)
    eb, eA, eB = _extra(Zo, u, np.random.default_rng(seed))
    blocks += eb
    A += eA
    B += eB
    Zl, _, _ = lib_problem(ctx, N, k, seed, leaf)
    P, dA, dB = run_isolated(torch, ctx, Zl, blocks, A, B, u, eps)
    checked = 0
    try:
        for j, b0 in enumerate(blocks):
            d = local_update(Zo, b0, A[j], B[j], eps)
            ref = apply_delta(Zo, d).dense()
            C = b.h2_matrix_clone(ctx, Zl)
            try:
                b.h2_batch_apply(ctx, P, j, dA.data_ptr(), dB.data_ptr(), C)
                got = to_oracle(ctx, C, Zo).dense()
                rV, rW = b.h2_get_ranks(C, 0), b.h2_get_ranks(C, 1)
            finally:
                b.h2_matrix_free(C)
            _BW(got, ref, Zo, (j, b0))
            checked += _rank_check(Zo, d, rV, rW)
        # the margin gate must leave most rank comparisons in place
        assert checked == len(blocks), (checked, len(blocks))
    finally:
        b.h2_batch_free(P)
        b.h2_matrix_free(Zl)


def test_execute_host_path_matches(ctx):
    N, leaf, k, u, eps = 24, 16, 6, 3, 0.5
    Zo, st, _ = oracle_problem(N, k, 7, leaf)
    blocks, A, B = draw_updates(Zo, st, 5, u)
    Zl, _, _ = lib_problem(ctx, N, k, 7, leaf)
    P = b.h2_batch_create(ctx, Zl, blocks, u)
    try:
        Acat, Bcat = concat_factors(P, A, B, u)
        res = b.h2_batch_execute_host(ctx, P, Acat, Bcat, eps)
        n_items = b.h2_batch_stats(ctx, P, flops=False)["cluster_tasks"]
        rk = res[:n_items]
        assert np.all(rk == np.round(rk)) and rk.max() <= k + u and rk.min() >= 0
        res2 = b.h2_batch_execute_host(ctx, P, Acat, Bcat, eps)
        np.testing.assert_array_equal(res, res2)   # deterministic
        dA = torch.from_numpy(Acat).cuda()
        dB = torch.from_numpy(Bcat).cuda()
        for j, b0 in enumerate(blocks):
            d = local_update(Zo, b0, A[j], B[j], eps)
            ref = apply_delta(Zo, d).dense()
            C = b.h2_matrix_clone(ctx, Zl)
            try:
                b.h2_batch_apply(ctx, P, j, dA.data_ptr(), dB.data_ptr(), C)
                got = to_oracle(ctx, C, Zo).dense()
            finally:
                b.h2_matrix_free(C)
            _BW(got, ref, Zo, (j, b0))
    finally:
        b.h2_batch_free(P)
        b.h2_matrix_free(Zl)


@pytest.mark.parametrize("eps", [1e-8, 0.5])
def test_sequential_updates_in_place(ctx, eps):
    """Updates applied one after the other in place (ranks grow or shrink,
    storage capacity grows).  Each step is compared with the oracle applied
    to the library's own state before that step: chained truncations make
    the end state depend on rounding through near-degenerate singular values
    at the cut, so per-step parity is the meaningful check."""
    N, leaf, k, u = 24, 16, 5, 3
    Zo, st, _ = oracle_problem(N, k, 21, leaf)
    blocks, A, B = draw_updates(Zo, st, 4, u)
    # a repeated block
    blocks = blocks + [blocks[0]]
    A = A + [A[0] * 0.5]
    B = B + [B[0]]
    Zl, _, _ = lib_problem(ctx, N, k, 21, leaf)
    checked = 0
    try:
        for j, b0 in enumerate(blocks):
            before = to_oracle(ctx, Zl, Zo)
            d = local_update(before, b0, A[j], B[j], eps)
            ref = apply_delta(before, d).dense()
            dA = torch.from_numpy(np.asfortranarray(A[j]).ravel(order="F")).cuda()
            dB = torch.from_numpy(np.asfortranarray(B[j]).ravel(order="F")).cuda()
            b.h2_lowrank_update(ctx, Zl, b0, u, dA.data_ptr(), A[j].shape[0], dB.data_ptr(), B[j].shape[0], eps)
            b.h2_ctx_synchronize(ctx)
            got = to_oracle(ctx, Zl, Zo)
            _BW(got.dense(), ref, Zo, j)
            if d["margin"] >= 1e-6:
                checked += 1
                assert list(got.V.rank) == list(apply_delta(before, d).V.rank)
                assert list(got.W.rank) == list(apply_delta(before, d).W.rank)
        if eps < 1e-6:
            # no truncation happens: the chain equals the oracle's chain
            ref = sequential_batch(Zo, blocks, A, B, eps).dense()
            _BW(to_oracle(ctx, Zl, Zo).dense(), ref, Zo, "chain")
        assert checked == len(blocks), checked
    finally:
        b.h2_matrix_free(Zl)


# ---------------------------------------------------------------- full size
FULL_N, FULL_K, FULL_U, FULL_EPS, FULL_COUNT = 256, 16, 8, 1e-8, 4096
FULL_SEED = synth.SEED_BASE + 1


@pytest.fixture(scope="module")
def full(ctx):
    Zo, st, _ = oracle_problem(FULL_N, FULL_K, FULL_SEED, 32)
    blocks, A, B = draw_updates(Zo, st, FULL_COUNT, FULL_U)
    Zl, _, _ = lib_problem(ctx, FULL_N, FULL_K, FULL_SEED, 32)
    yield Zo, Zl, blocks, A, B
    b.h2_matrix_free(Zl)


def _sample_positions(Zo, b0, rng, m=40):
    bt = Zo.blocks
    t0, s0 = bt.row[b0], bt.col[b0]
    rt, ct = Zo.V.tree, Zo.W.tree
    n = rt.n
    I1 = rng.integers(rt.offset[t0], rt.offset[t0] + rt.size[t0], m)
    J1 = rng.integers(0, n, m)
    I2 = rng.integers(0, n, m)
    J2 = rng.integers(ct.offset[s0], ct.offset[s0] + ct.size[s0], m)
    I3 = rng.integers(rt.offset[t0], rt.offset[t0] + rt.size[t0], m)
    J3 = rng.integers(ct.offset[s0], ct.offset[s0] + ct.size[s0], m)
    I4 = rng.integers(0, n, m // 2)
    J4 = rng.integers(0, n, m // 2)
    return np.concatenate([I1, I2, I3, I4]), np.concatenate([J1, J2, J3, J4])


def test_full_size_sampled_updates_match_oracle(ctx, full):
    Zo, Zl, blocks, A, B = full
    # the first 48 updates of the benchmark batch, in one isolated launch set
    nb = 48
    P, dA, dB = run_isolated(torch, ctx, Zl, blocks[:nb], A[:nb], B[:nb], FULL_U, FULL_EPS)
    rng = np.random.default_rng(0)
    levels = [Zo.V.tree.level[Zo.blocks.row[c]] for c in blocks[:nb]]
    # every level present among the first updates, plus a few more
    pick = sorted({levels.index(l) for l in set(levels)} | {0, 1, 2})
    checked = 0
    try:
        for j in pick:
            b0 = blocks[j]
            c, d = _full_size_blockwise(ctx, Zo, Zl, P, j, b0, A[j], B[j], dA, dB, FULL_EPS, rng)
            checked += c
            # entries anywhere, one by one (unchanged blocks included)
            ref_m = apply_delta(Zo, d)
            got_m, _, _ = applied_delta(ctx, Zl, P, j, dA, dB, Zo, b0)
            I, J = _sample_positions(Zo, b0, rng)
            ref = entries(ref_m, I, J)
            got = entries(got_m, I, J)
            np.testing.assert_allclose(got, ref, rtol=0, atol=TOL * np.abs(ref).max())
        assert checked == len(pick), checked
    finally:
        b.h2_batch_free(P)


def _full_size_blockwise(ctx, Zo, Zl, P, j, b0, A, B, dA, dB, eps, rng, cap=40):
    """Per-block parity of update j of an executed batch at full size: the
    changed blocks (row in T_t0 or column in T_s0; the block rows of t0 and
    s0 always, a sample of the rest) in compressed form and the nearfield
    leaves inside b0.  Returns whether the ranks were compared."""
    d = local_update(Zo, b0, A, B, eps)
    ref_m = apply_delta(Zo, d)
    got_m, rV, rW = applied_delta(ctx, Zl, P, j, dA, dB, Zo, b0)
    checked = _rank_check(Zo, d, rV, rW)
    bt = Zo.blocks
    Tt = set(Zo.V.tree.descendants(bt.row[b0]))
    Ts = set(Zo.W.tree.descendants(bt.col[b0]))
    aff = [c for c in bt.admissible if bt.row[c] in Tt or bt.col[c] in Ts]
    must = [c for c in aff if bt.row[c] == bt.row[b0] or bt.col[c] == bt.col[b0]]
    rest = [c for c in aff if c not in set(must)]
    if len(rest) > cap:
        rest = [int(x) for x in rng.choice(rest, cap, replace=False)]
    near = [c for c in bt.descendants(b0) if bt.kind[c] == BlockTree.NEAR]
    worst, where = blockwise_h2(got_m, ref_m, must + rest + near)
    assert worst <= TOL, (j, b0, where, worst)
    return checked, d


def test_full_size_exact_path_truncating(ctx, full):
    """The exact (truncating) path at the benchmark's structure: 256^2
    points, k = 16, rank-8 updates, H2_MODE_EXACT, eps = 0.3 (every level
    truncates: new ranks 21-24 of 24), on the first update of every level
    and the first 16 of the batch, in one isolated launch set.  Per-block
    parity with the oracle and equal ranks."""
    Zo, Zl, blocks, A, B = full
    eps = 0.3
    bt = Zo.blocks
    levels = [Zo.V.tree.level[bt.row[c]] for c in blocks]
    first = {}
    for j, l in enumerate(levels):
        first.setdefault(l, j)
    pick = sorted(set(first.values()) | set(range(16)))
    sb, sA, sB = [blocks[j] for j in pick], [A[j] for j in pick], [B[j] for j in pick]
    P = b.h2_batch_create(ctx, Zl, sb, FULL_U)
    b.h2_batch_set_mode(P, b.MODE_EXACT)
    try:
        Acat, Bcat = concat_factors(P, sA, sB, FULL_U)
        dA = torch.from_numpy(Acat).cuda()
        dB = torch.from_numpy(Bcat).cuda()
        b.h2_batch_execute(ctx, P, dA.data_ptr(), dB.data_ptr(), eps)
        b.h2_ctx_synchronize(ctx)
        assert b.h2_batch_paths(ctx, P, len(sb)).sum() == len(sb)
        rng = np.random.default_rng(3)
        checked, truncated = 0, 0
        for i, b0 in enumerate(sb):
            c, d = _full_size_blockwise(ctx, Zo, Zl, P, i, b0, sA[i], sB[i], dA, dB, eps, rng)
            checked += c
            truncated += any(r < FULL_K + FULL_U for r in d["V"]["rank"].values())
        assert checked == len(sb), checked
        assert truncated >= len(sb) // 2, truncated
        assert len({levels[j] for j in pick}) == len(first)
    finally:
        b.h2_batch_free(P)


def test_full_batch_properties(ctx, full):
    """All 4096 updates in the benchmark's launch configuration: no device
    error, ranks within k + u, orthonormal new leaf bases (sampled)."""
    Zo, Zl, blocks, A, B = full
    P = b.h2_batch_create(ctx, Zl, blocks, FULL_U)
    try:
        Acat, Bcat = concat_factors(P, A, B, FULL_U)
        res = b.h2_batch_execute_host(ctx, P, Acat, Bcat, FULL_EPS)
        st = b.h2_batch_stats(ctx, P)
        rk = res[:st["cluster_tasks"]]
        assert rk.min() >= 0 and rk.max() <= FULL_K + FULL_U
        assert np.all(np.isfinite(res))
        assert st["flops"] > 0
        dA = torch.from_numpy(Acat).cuda()
        dB = torch.from_numpy(Bcat).cuda()
        rng = np.random.default_rng(1)
        for j in rng.choice(len(blocks), 4, replace=False):
            b0 = blocks[j]
            got_m, _, _ = applied_delta(ctx, Zl, P, int(j), dA, dB, Zo, b0)
            t0 = Zo.blocks.row[b0]
            for t in got_m.V.tree.descendants(t0):
                if got_m.V.tree.is_leaf(t):
                    Q = got_m.V.leaf[t]
                    np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-13)
    finally:
        b.h2_batch_free(P)


@pytest.mark.parametrize("mode", ["auto", "exact"])
def test_update_independent_of_its_batch(ctx, full, mode):
    """An update computes the same bits whether it runs inside the 4096-update
    batch or alone: the Gram matrices of steps 2 and 3, R_t of step 4, the
    ranks, and the committed couplings and bases.  Certified path: the upper
    levels of the batch run on k_fweights_wide, the others on k_fweights,
    the update alone on k_fweights_wide throughout.  Exact path: the levels
    of the batch with many cluster tasks run one warp per task, the update
    alone runs a block of four warps per task."""
    Zo, Zl, blocks, A, B = full
    exact = mode == "exact"
    P = b.h2_batch_create(ctx, Zl, blocks, FULL_U)
    if exact:
        b.h2_batch_set_mode(P, b.MODE_EXACT)
    try:
        Acat, Bcat = concat_factors(P, A, B, FULL_U)
        dA = torch.from_numpy(Acat).cuda()
        dB = torch.from_numpy(Bcat).cuda()
        b.h2_batch_execute(ctx, P, dA.data_ptr(), dB.data_ptr(), FULL_EPS)
        b.h2_ctx_synchronize(ctx)
        bt = Zo.blocks
        rng = np.random.default_rng(11)
        # updates with large subtrees reach the levels that run one warp per task
        big = sorted(range(len(blocks)), key=lambda j: -Zo.V.tree.size[bt.row[blocks[j]]])[:2]
        for j in big + [int(x) for x in rng.choice(len(blocks), 2, replace=False)]:
            first, last = b.h2_batch_update_items(P, j)
            Q = b.h2_batch_create(ctx, Zl, [blocks[j]], FULL_U)
            if exact:
                b.h2_batch_set_mode(Q, b.MODE_EXACT)
            try:
                a1, b1 = concat_factors(Q, [A[j]], [B[j]], FULL_U)
                qa = torch.from_numpy(a1).cuda()
                qb = torch.from_numpy(b1).cuda()
                b.h2_batch_execute(ctx, Q, qa.data_ptr(), qb.data_ptr(), FULL_EPS)
                b.h2_ctx_synchronize(ctx)
                f1, l1 = b.h2_batch_update_items(Q, 0)
                assert l1 - f1 == last - first
                for i in range(last - first):
                    ia, ib = b.h2_batch_item_info(P, first + i), b.h2_batch_item_info(Q, f1 + i)
                    assert (ia["side"], ia["cluster"], ia["rank"]) == (ib["side"], ib["cluster"], ib["rank"])
                    for which in (0, 1, 2):
                        np.testing.assert_array_equal(b.h2_batch_item_tile(ctx, P, first + i, which),
                                                      b.h2_batch_item_tile(ctx, Q, f1 + i, which))
                C1 = b.h2_matrix_clone(ctx, Zl)
                C2 = b.h2_matrix_clone(ctx, Zl)
                try:
                    b.h2_batch_apply(ctx, P, j, dA.data_ptr(), dB.data_ptr(), C1)
                    b.h2_batch_apply(ctx, Q, 0, qa.data_ptr(), qb.data_ptr(), C2)
                    np.testing.assert_array_equal(b.h2_get_couplings(ctx, C1), b.h2_get_couplings(ctx, C2))
                    for sd in (0, 1):
                        for x, y in zip(b.h2_get_basis(ctx, C1, sd), b.h2_get_basis(ctx, C2, sd)):
                            np.testing.assert_array_equal(x, y)
                finally:
                    b.h2_matrix_free(C1)
                    b.h2_matrix_free(C2)
            finally:
                b.h2_batch_free(Q)
    finally:
        b.h2_batch_free(P)
