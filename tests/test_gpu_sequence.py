"""Updates applied in order through h2_lowrank_update_sequence (waves of
updates whose footprints do not meet, each wave one isolated batch).

The result must be the bits of h2_lowrank_update called for each update in
turn: ranks, bases, couplings and nearfield of the whole matrix.  Without
truncation it must also match the oracle's chain (the exact sum of all
updates, Section 5 applied repeatedly) to 1e-10.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

from blockwise import assert_blockwise_dense  # noqa: E402
from libside import lib_problem, to_oracle  # noqa: E402
from oracle.tree import BlockTree  # noqa: E402
from oracle.update import sequential_batch  # noqa: E402
from problems import draw_updates, oracle_problem  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_ctx_destroy(c)


def _state(ctx, Z):
    out = [b.h2_get_couplings(ctx, Z), b.h2_get_nearfield(ctx, Z)]
    for sd in (0, 1):
        out.extend(b.h2_get_basis(ctx, Z, sd))
    return out


def _col(M):
    # u x rows row-major = rows x u column-major
    return torch.from_numpy(np.ascontiguousarray(np.asarray(M).T)).cuda()


def _run_both(ctx, N, k, seed, leaf, blocks, A, B, u, eps):
    Z1, _, _ = lib_problem(ctx, N, k, seed, leaf)
    Z2, _, _ = lib_problem(ctx, N, k, seed, leaf)
    try:
        for j, b0 in enumerate(blocks):
            a, bb = _col(A[j]), _col(B[j])
            b.h2_lowrank_update(ctx, Z1, b0, u, a.data_ptr(), A[j].shape[0], bb.data_ptr(), B[j].shape[0], eps)
        b.h2_ctx_synchronize(ctx)
        Acat = torch.from_numpy(np.concatenate([np.asarray(x).ravel(order="F") for x in A])).cuda()
        Bcat = torch.from_numpy(np.concatenate([np.asarray(x).ravel(order="F") for x in B])).cuda()
        waves = b.h2_lowrank_update_sequence(ctx, Z2, blocks, u, Acat.data_ptr(), Bcat.data_ptr(), eps)
        s1, s2 = _state(ctx, Z1), _state(ctx, Z2)
        assert len(s1) == len(s2)
        for x, y in zip(s1, s2):
            np.testing.assert_array_equal(x, y)
        return waves, Z2
    except Exception:
        b.h2_matrix_free(Z2)
        raise
    finally:
        b.h2_matrix_free(Z1)


@pytest.mark.parametrize("eps", [1e-8, 0.5])
def test_sequence_equals_one_by_one(ctx, eps):
    N, leaf, k, u = 32, 16, 6, 3
    Zo, st, _ = oracle_problem(N, k, 431, leaf)
    blocks, A, B = draw_updates(Zo, st, 24, u)
    bt = Zo.blocks
    rng = np.random.default_rng(5)
    # a repeated block, a subdivided and an inadmissible block
    sub = [c for c in range(1, bt.n_blocks) if bt.kind[c] == BlockTree.SUB]
    for c in (blocks[3], sub[len(sub) // 2], bt.inadmissible[len(bt.inadmissible) // 2]):
        blocks.append(c)
        A.append(rng.standard_normal((Zo.V.tree.size[bt.row[c]], u)))
        B.append(rng.standard_normal((Zo.W.tree.size[bt.col[c]], u)))
    waves, Z2 = _run_both(ctx, N, k, 431, leaf, blocks, A, B, u, eps)
    try:
        assert 1 <= waves < len(blocks)   # some updates ran together
        if eps < 1e-6:
            ref = sequential_batch(Zo, blocks, A, B, eps).dense()
            got = to_oracle(ctx, Z2, Zo).dense()
            assert_blockwise_dense(got, ref, Zo.blocks, Zo.V.tree, Zo.W.tree, TOL, "chain")
    finally:
        b.h2_matrix_free(Z2)


def test_sequence_of_leaf_blocks_runs_in_waves(ctx):
    N, leaf, k, u = 64, 16, 6, 2
    Zo, st, _ = oracle_problem(N, k, 433, leaf)
    blocks, A, B = draw_updates(Zo, st, 64, u)
    waves, Z2 = _run_both(ctx, N, k, 433, leaf, blocks, A, B, u, 1e-8)
    try:
        assert waves <= len(blocks) // 2   # 17 waves for these 64 updates
    finally:
        b.h2_matrix_free(Z2)


def test_empty_sequence(ctx):
    Zl, _, _ = lib_problem(ctx, 24, 6, 435, 16)
    try:
        before = _state(ctx, Zl)
        assert b.h2_lowrank_update_sequence(ctx, Zl, [], 3, 0, 0, 1e-8) == 0
        for x, y in zip(before, _state(ctx, Zl)):
            np.testing.assert_array_equal(x, y)
    finally:
        b.h2_matrix_free(Zl)
