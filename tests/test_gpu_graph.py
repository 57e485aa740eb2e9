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

from blockwise import assert_blockwise_dense  # noqa: E402
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
                assert_blockwise_dense(got, ref, Zo.blocks, Zo.V.tree, Zo.W.tree, TOL, (eps, mode, j))
    finally:
        b.h2_batch_free(P)
        b.h2_matrix_free(Zl)
