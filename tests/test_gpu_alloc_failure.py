"""Device allocation failures in the update calls (error behaviour of the C
ABI; the paper has no counterpart).

The library's failure hook makes the n-th device allocation fail.  For every
n up to the number of allocations one update makes, h2_lowrank_update and
h2_batch_apply must return H2_ENOMEM and leave the matrix as it was (every
basis, coupling and nearfield entry; the rank capacity may have grown), and
the next call without the hook must give the bits of an update that never
met a failure.  The update is chosen to reach every allocation site of the
commit: its block is subdivided (nearfield leaves inside it) and the new
ranks exceed the matrix's rank capacity (the storage is re-laid out).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

from libside import lib_problem, structure  # noqa: E402

N, K, LEAF, U, EPS = 32, 6, 16, 3, 1e-12
ENOMEM = 2


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_debug_fail_allocation(0)
    b.h2_ctx_destroy(c)


def _state(ctx, Z):
    out = [b.h2_get_couplings(ctx, Z), b.h2_get_nearfield(ctx, Z)]
    for sd in (0, 1):
        out.extend(b.h2_get_basis(ctx, Z, sd))
        out.append(b.h2_get_ranks(Z, sd))
    return out


def _assert_same(s1, s2, what):
    assert len(s1) == len(s2), what
    for x, y in zip(s1, s2):
        np.testing.assert_array_equal(x, y, err_msg=str(what))


@pytest.fixture(scope="module")
def problem(ctx):
    Z, _, _ = lib_problem(ctx, N, K, 611, LEAF, kcap=K)
    tc, tb, _, _, _, _ = structure(Z)
    size = tc["size"]
    # a subdivided block of 64 x 64 points: nearfield leaves inside, and
    # extended ranks K + U above the capacity K
    sub = [i for i in range(1, len(tb["kind"])) if tb["kind"][i] == 0 and size[tb["row"][i]] == 64]
    assert sub
    b0 = sub[len(sub) // 2]
    rows, cols = int(size[tb["row"][b0]]), int(size[tb["col"][b0]])
    rng = np.random.default_rng(7)
    A = torch.from_numpy(np.asfortranarray(rng.standard_normal((rows, U)))).T.contiguous().cuda()
    B = torch.from_numpy(np.asfortranarray(rng.standard_normal((cols, U)))).T.contiguous().cuda()
    yield Z, b0, rows, cols, A, B
    b.h2_matrix_free(Z)


def _update(ctx, Z, b0, rows, cols, A, B):
    # A, B: u x rows row-major tensors = rows x u column-major
    b.h2_lowrank_update(ctx, Z, b0, U, A.data_ptr(), rows, B.data_ptr(), cols, EPS)


def test_update_is_all_or_nothing_under_allocation_failure(ctx, problem):
    Z, b0, rows, cols, A, B = problem
    before = _state(ctx, Z)
    Zref = b.h2_matrix_clone(ctx, Z)
    try:
        _update(ctx, Zref, b0, rows, cols, A, B)
        want = _state(ctx, Zref)
    finally:
        b.h2_matrix_free(Zref)
    assert max(want[-1]) > K and max(want[-1]) <= K + U   # the capacity has to grow

    failed = 0
    for n in range(1, 400):
        Zn = b.h2_matrix_clone(ctx, Z)
        try:
            b.h2_debug_fail_allocation(n)
            try:
                _update(ctx, Zn, b0, rows, cols, A, B)
                ok = True
            except b.H2Error as e:
                assert e.status == ENOMEM, (n, e)
                ok = False
            b.h2_debug_fail_allocation(0)
            if not ok:
                failed += 1
                _assert_same(_state(ctx, Zn), before, ("unchanged after failed allocation", n))
                # the same matrix takes the update once the device has memory
                _update(ctx, Zn, b0, rows, cols, A, B)
            _assert_same(_state(ctx, Zn), want, ("update after failure", n))
        finally:
            b.h2_debug_fail_allocation(0)
            b.h2_matrix_free(Zn)
        if ok:
            break
    else:
        pytest.fail("the update never completed")
    # the plan, the factor copies, the new layout and the commit lists
    assert failed >= 20, failed


def test_batch_apply_is_all_or_nothing_under_allocation_failure(ctx, problem):
    Z, b0, rows, cols, A, B = problem
    P = b.h2_batch_create(ctx, Z, [b0], U)
    try:
        lenA, lenB = b.h2_batch_factor_sizes(P)
        assert lenA == rows * U and lenB == cols * U
        Af, Bf = A.reshape(-1).contiguous(), B.reshape(-1).contiguous()
        b.h2_batch_execute(ctx, P, Af.data_ptr(), Bf.data_ptr(), EPS)
        before = _state(ctx, Z)
        Zref = b.h2_matrix_clone(ctx, Z)
        try:
            b.h2_batch_apply(ctx, P, 0, Af.data_ptr(), Bf.data_ptr(), Zref)
            want = _state(ctx, Zref)
        finally:
            b.h2_matrix_free(Zref)
        failed = 0
        for n in range(1, 100):
            Zn = b.h2_matrix_clone(ctx, Z)
            try:
                b.h2_debug_fail_allocation(n)
                try:
                    b.h2_batch_apply(ctx, P, 0, Af.data_ptr(), Bf.data_ptr(), Zn)
                    ok = True
                except b.H2Error as e:
                    assert e.status == ENOMEM, (n, e)
                    ok = False
                b.h2_debug_fail_allocation(0)
                if not ok:
                    failed += 1
                    _assert_same(_state(ctx, Zn), before, ("unchanged after failed allocation", n))
                    b.h2_batch_apply(ctx, P, 0, Af.data_ptr(), Bf.data_ptr(), Zn)
                _assert_same(_state(ctx, Zn), want, ("apply after failure", n))
            finally:
                b.h2_debug_fail_allocation(0)
                b.h2_matrix_free(Zn)
            if ok:
                break
        else:
            pytest.fail("the commit never completed")
        assert failed >= 5, failed
    finally:
        b.h2_batch_free(P)


def test_matvec_reports_allocation_failure(ctx, problem):
    Z = problem[0]
    n = N * N
    X = torch.ones(n, dtype=torch.float64, device="cuda")
    Y = torch.full((n,), 3.0, dtype=torch.float64, device="cuda")
    b.h2_debug_fail_allocation(1)
    try:
        with pytest.raises(b.H2Error) as e:
            b.h2_matvec(ctx, Z, 1, 1.0, X.data_ptr(), n, 0.0, Y.data_ptr(), n)
        assert e.value.status == ENOMEM
    finally:
        b.h2_debug_fail_allocation(0)
    torch.cuda.synchronize()
    assert bool((Y == 3.0).all())
    b.h2_matvec(ctx, Z, 1, 1.0, X.data_ptr(), n, 0.0, Y.data_ptr(), n)
    torch.cuda.synchronize()
    assert not bool((Y == 3.0).all())


def test_hook_rejects_negative_counts():
    with pytest.raises(b.H2Error):
        b.h2_debug_fail_allocation(-1)
