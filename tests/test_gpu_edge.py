"""Edge cases of the CUDA update against the oracle (dense, n <= 1024).

Update rank 1, zero factors, rank-0 bases, the widest extended rank k+u = 32,
leaves of 64 indices (the 64-row kernels), eps = 0, ragged 1-D and 3-D point
sets with ranks capped by the cluster sizes, duplicate targets in one batch
and an empty batch.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

from blockwise import assert_blockwise_dense  # noqa: E402
from gpu_util import run_isolated  # noqa: E402
from libside import lib_problem, lib_problem_general, to_oracle  # noqa: E402
from oracle.tree import BlockTree  # noqa: E402
from oracle.update import apply_delta, local_update  # noqa: E402
from problems import draw_updates, oracle_problem, oracle_problem_general  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_ctx_destroy(c)


def _check(ctx, Zo, Zl, blocks, A, B, u, eps):
    P, dA, dB = run_isolated(torch, ctx, Zl, blocks, A, B, u, eps)
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
            assert_blockwise_dense(got, ref, Zo.blocks, Zo.V.tree, Zo.W.tree, TOL, (j, b0))
            if d["margin"] >= 1e-6:
                for t, r in d["V"]["rank"].items():
                    assert rV[t] == r
                for t, r in d["W"]["rank"].items():
                    assert rW[t] == r
    finally:
        b.h2_batch_free(P)


def _mixed_blocks(Zo, st, count, u):
    blocks, A, B = draw_updates(Zo, st, count, u)
    bt = Zo.blocks
    rng = np.random.default_rng(17)
    sub = [c for c in range(1, bt.n_blocks) if bt.kind[c] == BlockTree.SUB]
    extra = [bt.inadmissible[len(bt.inadmissible) // 2]] + ([sub[len(sub) // 3]] if sub else [])
    for c in extra:
        blocks.append(c)
        A.append(rng.standard_normal((Zo.V.tree.size[bt.row[c]], u)))
        B.append(rng.standard_normal((Zo.W.tree.size[bt.col[c]], u)))
    return blocks, A, B


@pytest.mark.parametrize("eps", [1e-8, 0.5])
def test_update_rank_one(ctx, eps):
    Zo, st, _ = oracle_problem(24, 6, 41, 16)
    Zl, _, _ = lib_problem(ctx, 24, 6, 41, 16)
    try:
        blocks, A, B = _mixed_blocks(Zo, st, 4, 1)
        _check(ctx, Zo, Zl, blocks, A, B, 1, eps)
    finally:
        b.h2_matrix_free(Zl)


def test_zero_factors_reproject_only(ctx):
    Zo, st, _ = oracle_problem(24, 6, 43, 16)
    Zl, _, _ = lib_problem(ctx, 24, 6, 43, 16)
    try:
        blocks, A, B = _mixed_blocks(Zo, st, 4, 3)
        A = [np.zeros_like(a) for a in A]
        B = [np.zeros_like(x) for x in B]
        _check(ctx, Zo, Zl, blocks, A, B, 3, 1e-8)
    finally:
        b.h2_matrix_free(Zl)


@pytest.mark.parametrize("eps", [1e-8, 0.0])
def test_rank_zero_bases(ctx, eps):
    pts = np.random.default_rng(3).uniform(size=(500, 2))
    Zo, st, _ = oracle_problem_general(pts, 0, 47, 16)
    Zl, _, _ = lib_problem_general(ctx, pts, 0, 47, 16)
    try:
        assert max(Zo.V.rank) == 0
        blocks, A, B = _mixed_blocks(Zo, st, 4, 3)
        _check(ctx, Zo, Zl, blocks, A, B, 3, eps)
    finally:
        b.h2_matrix_free(Zl)


@pytest.mark.parametrize("leaf", [32, 64])
def test_widest_extended_rank(ctx, leaf):
    # k + u = 32 (all lanes), leaves of 32 and of 64 indices (64-row kernels)
    Zo, st, _ = oracle_problem(32, 24, 53, leaf)
    Zl, _, _ = lib_problem(ctx, 32, 24, 53, leaf, kcap=32)
    try:
        blocks, A, B = _mixed_blocks(Zo, st, 4, 8)
        _check(ctx, Zo, Zl, blocks, A, B, 8, 1e-8)
    finally:
        b.h2_matrix_free(Zl)


def test_eps_zero_is_exact(ctx):
    Zo, st, _ = oracle_problem(24, 5, 59, 16)
    Zl, _, _ = lib_problem(ctx, 24, 5, 59, 16)
    try:
        blocks, A, B = _mixed_blocks(Zo, st, 4, 3)
        _check(ctx, Zo, Zl, blocks, A, B, 3, 0.0)
    finally:
        b.h2_matrix_free(Zl)


@pytest.mark.parametrize("dim,eps", [(1, 1e-8), (1, 0.3), (3, 1e-8), (3, 0.3)])
def test_ragged_point_sets(ctx, dim, eps):
    pts = np.random.default_rng(dim).uniform(size=(600, dim))
    Zo, st, _ = oracle_problem_general(pts, 5, 61 + dim, 12)
    Zl, _, _ = lib_problem_general(ctx, pts, 5, 61 + dim, 12)
    try:
        blocks, A, B = _mixed_blocks(Zo, st, 5, 2)
        _check(ctx, Zo, Zl, blocks, A, B, 2, eps)
    finally:
        b.h2_matrix_free(Zl)


def test_duplicate_targets_and_empty_batch(ctx):
    Zo, st, _ = oracle_problem(24, 6, 67, 16)
    Zl, _, _ = lib_problem(ctx, 24, 6, 67, 16)
    try:
        blocks, A, B = draw_updates(Zo, st, 3, 3)
        blocks = blocks + blocks[:2]
        A = A + [2.0 * a for a in A[:2]]
        B = B + B[:2]
        _check(ctx, Zo, Zl, blocks, A, B, 3, 1e-8)
        P = b.h2_batch_create(ctx, Zl, [], 3)
        try:
            b.h2_batch_execute(ctx, P, 0, 0, 1e-8)
            b.h2_ctx_synchronize(ctx)
            assert b.h2_batch_stats(ctx, P)["cluster_tasks"] == 0
        finally:
            b.h2_batch_free(P)
    finally:
        b.h2_matrix_free(Zl)
