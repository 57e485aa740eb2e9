"""Repeated executions of one batch: the first runs eagerly, a repeat with the
same arguments is captured into a CUDA graph and replayed.  Results must be
bit-identical across the eager run and the replays, and changing an argument
(eps, path mode, factors) must give a fresh, correct execution."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

from gpu_util import concat_factors  # noqa: E402
from libside import lib_problem, to_oracle  # noqa: E402
from oracle.update import apply_delta, local_update  # noqa: E402
from problems import draw_updates, oracle_problem  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_ctx_destroy(c)


def _dense_of(ctx, Zl, Zo, P, j, dA, dB):
    C = b.h2_matrix_clone(ctx, Zl)
    try:
        b.h2_batch_apply(ctx, P, j, dA.data_ptr(), dB.data_ptr(), C)
        return to_oracle(ctx, C, Zo).dense()
    finally:
        b.h2_matrix_free(C)


def test_replays_match_eager_and_oracle(ctx):
    N, leaf, k, u = 24, 16, 6, 3
    Zo, st, _ = oracle_problem(N, k, 361, leaf)
    blocks, A, B = draw_updates(Zo, st, 6, u)
    Zl, _, _ = lib_problem(ctx, N, k, 361, leaf)
    P = b.h2_batch_create(ctx, Zl, blocks, u)
    try:
        Acat, Bcat = concat_factors(P, A, B, u)
        b.h2_batch_set_timing(P, True)
        for eps, mode in ((1e-8, b.MODE_AUTO), (0.5, b.MODE_AUTO), (1e-8, b.MODE_EXACT)):
            b.h2_batch_set_mode(P, mode)
            runs = [b.h2_batch_execute_host(ctx, P, Acat, Bcat, eps) for _ in range(3)]
            for r in runs[1:]:
                np.testing.assert_array_equal(r, runs[0])
            # phase timing works in the replays too
            assert b.h2_batch_phase_stats(ctx, P, b.PHASES.index("reproject"), flops=False)["ms"] >= 0.0
            dA = torch.from_numpy(Acat).cuda()
            dB = torch.from_numpy(Bcat).cuda()
            b.h2_batch_execute(ctx, P, dA.data_ptr(), dB.data_ptr(), eps)   # new factor pointers
            b.h2_ctx_synchronize(ctx)
            for j in (0, len(blocks) - 1):
                ref = apply_delta(Zo, local_update(Zo, blocks[j], A[j], B[j], eps)).dense()
                got = _dense_of(ctx, Zl, Zo, P, j, dA, dB)
                assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref), (eps, mode, j)
    finally:
        b.h2_batch_free(P)
        b.h2_matrix_free(Zl)


def test_replay_follows_matrix_storage(ctx):
    """Committing an update that grows the matrix's rank capacity moves its
    storage; the next execution of another batch on the grown matrix must not
    replay a graph that reads the old storage."""
    N, leaf, k, u = 24, 16, 6, 3
    Zo, st, _ = oracle_problem(N, k, 363, leaf)
    blocks, A, B = draw_updates(Zo, st, 2, u)
    Zl, _, _ = lib_problem(ctx, N, k, 363, leaf, kcap=k)
    try:
        dA = torch.from_numpy(np.asfortranarray(A[0]).ravel(order="F")).cuda()
        dB = torch.from_numpy(np.asfortranarray(B[0]).ravel(order="F")).cuda()
        Q = b.h2_batch_create(ctx, Zl, [blocks[1]], u)
        try:
            A1 = torch.from_numpy(np.asfortranarray(A[1]).ravel(order="F")).cuda()
            B1 = torch.from_numpy(np.asfortranarray(B[1]).ravel(order="F")).cuda()
            for _ in range(2):
                b.h2_batch_execute(ctx, Q, A1.data_ptr(), B1.data_ptr(), 1e-8)   # eager, then captured
            b.h2_ctx_synchronize(ctx)
            before = to_oracle(ctx, Zl, Zo)
            # grow the capacity of Zl in place (ranks k + u > kcap)
            b.h2_lowrank_update(ctx, Zl, blocks[0], u, dA.data_ptr(), A[0].shape[0], dB.data_ptr(),
                                B[0].shape[0], 1e-8)
            b.h2_ctx_synchronize(ctx)
            assert b.h2_get_ranks(Zl, 0).max() == k + u
        finally:
            b.h2_batch_free(Q)
        after = to_oracle(ctx, Zl, Zo)
        ref = apply_delta(before, local_update(before, blocks[0], A[0], B[0], 1e-8)).dense()
        assert np.linalg.norm(after.dense() - ref) <= TOL * np.linalg.norm(ref)
    finally:
        b.h2_matrix_free(Zl)
