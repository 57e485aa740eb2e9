"""The allocation-free update entry point.

Some callers cannot allocate device memory while they run: code confined
to a device-memory budget reserved at start-up (an allocation mid-run could
fail or take memory another part of the program counts on), and hosts whose
device allocator belongs to another runtime (a framework's caching allocator
that already holds the free memory).  For them h2_lowrank_update_noalloc
performs the in-place update with fixed scratch inside the library.  Here it
is called through the C ABI twice in a row and must give the same matrix as
h2_lowrank_update, within the per-block 1e-10 relative Frobenius tolerance of
the other parity tests, on admissible leaves, on a subdivided block with
padded factors (leading dimensions above the row counts), and on an update
that the certificate sends to the exact path; the second call must leave the
device's free memory unchanged; requests beyond its fixed limits must be
refused with H2_EINVAL.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

import synth  # noqa: E402
from blockwise import assert_blockwise_dense  # noqa: E402
from gpu_util import run_isolated  # noqa: E402
from libside import lib_problem, to_oracle  # noqa: E402
from oracle.tree import BlockTree  # noqa: E402
from problems import draw_updates, oracle_problem  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_ctx_destroy(c)


@pytest.mark.parametrize("eps", [1e-8, 0.5])
def test_noalloc_update_matches_allocating_update(ctx, eps):
    N, leaf, k, u, seed = 24, 16, 5, 3, 31
    Zo, st, _ = oracle_problem(N, k, seed, leaf)
    blocks, A, B = draw_updates(Zo, st, 2, u)
    Z1, _, _ = lib_problem(ctx, N, k, seed, leaf, kcap=16)
    Z2, _, _ = lib_problem(ctx, N, k, seed, leaf, kcap=16)
    try:
        for j in range(2):   # two calls in a row on the same matrix
            dA = torch.from_numpy(np.asfortranarray(A[j]).ravel(order="F")).cuda()
            dB = torch.from_numpy(np.asfortranarray(B[j]).ravel(order="F")).cuda()
            rows_a, rows_b = A[j].shape[0], B[j].shape[0]
            b.h2_lowrank_update(ctx, Z1, blocks[j], u, dA.data_ptr(), rows_a, dB.data_ptr(), rows_b, eps)
            b.h2_lowrank_update_noalloc(ctx, Z2, blocks[j], u, dA.data_ptr(), rows_a, dB.data_ptr(), rows_b, eps)
            b.h2_ctx_synchronize(ctx)
            want = to_oracle(ctx, Z1, Zo).dense()
            got = to_oracle(ctx, Z2, Zo).dense()
            assert_blockwise_dense(got, want, Zo.blocks, Zo.V.tree, Zo.W.tree, 1e-10, j)
            np.testing.assert_array_equal(b.h2_get_ranks(Z1, 0), b.h2_get_ranks(Z2, 0))
            np.testing.assert_array_equal(b.h2_get_ranks(Z1, 1), b.h2_get_ranks(Z2, 1))
    finally:
        b.h2_matrix_free(Z1)
        b.h2_matrix_free(Z2)


def _padded(M, extra):
    """Column-major device copy of M with `extra` unused rows per column."""
    P = np.zeros((M.shape[0] + extra, M.shape[1]))
    P[:M.shape[0]] = M
    P[M.shape[0]:] = np.nan    # never read
    return torch.from_numpy(P.ravel(order="F")).cuda(), P.shape[0]


def test_noalloc_subdivided_block_and_exact_path(ctx):
    N, leaf, k, u, seed = 24, 16, 5, 3, 37
    Zo, st, _ = oracle_problem(N, k, seed, leaf)
    bt = Zo.blocks
    sub = [c for c in range(1, bt.n_blocks) if bt.kind[c] == BlockTree.SUB]
    blocks, A, B = draw_updates(Zo, st, 1, u)
    rng = np.random.default_rng(seed)
    # a subdivided block with admissible and nearfield leaves below it
    def count(c, kind):
        return sum(bt.kind[x] == kind for x in bt.descendants(c))
    c = next(c for c in sub if count(c, BlockTree.NEAR) >= 4 and count(c, BlockTree.ADM) >= 4
             and Zo.V.tree.size[bt.row[c]] <= 72)
    cases = [(c, rng.standard_normal((Zo.V.tree.size[bt.row[c]], u)),
              rng.standard_normal((Zo.W.tree.size[bt.col[c]], u)), 1e-8),
             (blocks[0], A[0], B[0], 0.5)]
    # the second case truncates: the batch API reports the exact path for it
    Zp, _, _ = lib_problem(ctx, N, k, seed, leaf, kcap=16)
    try:
        P, _, _ = run_isolated(torch, ctx, Zp, [cases[1][0]], [cases[1][1]], [cases[1][2]], u, 0.5)
        try:
            assert b.h2_batch_paths(ctx, P, 1)[0] == 1
        finally:
            b.h2_batch_free(P)
    finally:
        b.h2_matrix_free(Zp)
    Z1, _, _ = lib_problem(ctx, N, k, seed, leaf, kcap=16)
    Z2, _, _ = lib_problem(ctx, N, k, seed, leaf, kcap=16)
    try:
        for j, (blk, Aj, Bj, eps) in enumerate(cases):
            dA, lda = _padded(Aj, 5)
            dB, ldb = _padded(Bj, 3)
            b.h2_lowrank_update(ctx, Z1, blk, u, dA.data_ptr(), lda, dB.data_ptr(), ldb, eps)
            b.h2_ctx_synchronize(ctx)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            b.h2_lowrank_update_noalloc(ctx, Z2, blk, u, dA.data_ptr(), lda, dB.data_ptr(), ldb, eps)
            b.h2_ctx_synchronize(ctx)
            if j == 1:
                # kernels and the scratch array are resident since the
                # first call: nothing may be allocated now
                assert torch.cuda.mem_get_info()[0] == free0
            want = to_oracle(ctx, Z1, Zo).dense()
            got = to_oracle(ctx, Z2, Zo).dense()
            assert_blockwise_dense(got, want, Zo.blocks, Zo.V.tree, Zo.W.tree, 1e-10, (j, blk))
            np.testing.assert_array_equal(b.h2_get_ranks(Z1, 0), b.h2_get_ranks(Z2, 0))
            np.testing.assert_array_equal(b.h2_get_ranks(Z1, 1), b.h2_get_ranks(Z2, 1))
    finally:
        b.h2_matrix_free(Z1)
        b.h2_matrix_free(Z2)


def test_noalloc_refuses_requests_beyond_its_limits(ctx):
    # 4095 clusters per side: above the fixed 512
    Z = b.h2_matrix_create(ctx, synth.grid_points_2d(256), 32, 2.0, 0.0, 16)
    try:
        tb = b.h2_tree_blocks(Z)
        blk = int(np.flatnonzero(tb["kind"] == 1)[0])
        dA = torch.zeros(65536 * 2, dtype=torch.float64, device="cuda")
        with pytest.raises(b.H2Error) as e:
            b.h2_lowrank_update_noalloc(ctx, Z, blk, 2, dA.data_ptr(), 65536, dA.data_ptr(), 65536, 1e-8)
        assert e.value.status == 1 and "512" in str(e.value)
    finally:
        b.h2_matrix_free(Z)
    # rank capacity that the update would have to grow
    Zs, _, _ = lib_problem(ctx, 24, 5, 3, 16, kcap=5)
    try:
        tb = b.h2_tree_blocks(Zs)
        blk = int(np.flatnonzero(tb["kind"] == 1)[0])
        dA = torch.zeros(576 * 3, dtype=torch.float64, device="cuda")
        with pytest.raises(b.H2Error) as e:
            b.h2_lowrank_update_noalloc(ctx, Zs, blk, 3, dA.data_ptr(), 576, dA.data_ptr(), 576, 1e-8)
        assert e.value.status == 1 and "capacity" in str(e.value)
    finally:
        b.h2_matrix_free(Zs)
