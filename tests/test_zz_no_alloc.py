"""The allocation-free update entry point.

Some callers cannot allocate device memory while they run (work recorded
into CUDA graphs, code confined to a device-memory budget reserved at
start-up, hosts whose allocator belongs to another runtime).  For them
h2_lowrank_update_noalloc performs the in-place update with fixed scratch
inside the library.  Here it is called through the C ABI twice in a row and
must give the same matrix as h2_lowrank_update, within the 1e-10 relative
Frobenius tolerance of the other parity tests; requests beyond its fixed
limits must be refused with H2_EINVAL.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

import synth  # noqa: E402
from libside import lib_problem, to_oracle  # noqa: E402
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
            assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want), j
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
