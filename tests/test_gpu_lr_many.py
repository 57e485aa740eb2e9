"""h2_lr_factor_many and h2_chol_factor_many: independent factorisations
side by side (batches of problems of different sizes).  Each result must be
the bits of the factorisation of that matrix alone: bases, couplings,
nearfield and statistics."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

import synth  # noqa: E402

SIZES = [24, 32, 20, 28, 16]


def _state(ctx, Z):
    out = [b.h2_get_couplings(ctx, Z), b.h2_get_nearfield(ctx, Z)]
    for sd in (0, 1):
        out.extend(b.h2_get_basis(ctx, Z, sd))
    return out


def _problems(ctx, opt):
    out = []
    for i, cells in enumerate(SIZES):
        sigma = synth.checker_sigma(np.random.default_rng(700 + i), 4, 2)
        out.append(b.h2_build_fem(ctx, 2, cells, 4, sigma, opt))
    return out


def test_many_equals_one_by_one():
    ctx = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    opt = b.options(eps=1e-4, leaf_size=16)
    alone = _problems(ctx, opt)
    many = _problems(ctx, opt)
    try:
        want = [b.h2_lr_factor(ctx, Z, opt) for Z in alone]
        got = b.h2_lr_factor_many(ctx, many, opt, threads=3)
        for i in range(len(SIZES)):
            assert got[i]["updates"] == want[i]["updates"] > 0
            assert got[i]["products"] == want[i]["products"]
            assert got[i]["max_rank"] == want[i]["max_rank"]
            for x, y in zip(_state(ctx, many[i]), _state(ctx, alone[i])):
                np.testing.assert_array_equal(x, y)
        with pytest.raises(b.H2Error) as e:
            b.h2_lr_factor_many(ctx, [alone[0], alone[0]], opt)
        assert e.value.status == 1
    finally:
        for Z in alone + many:
            b.h2_matrix_free(Z)
        b.h2_ctx_destroy(ctx)


def test_chol_many_equals_one_by_one():
    """h2_chol_factor_many: the same rule for the Cholesky factorisation."""
    ctx = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    opt = b.options(eps=1e-4, leaf_size=16)
    alone = _problems(ctx, opt)
    many = _problems(ctx, opt)
    try:
        want = [b.h2_chol_factor(ctx, Z, opt) for Z in alone]
        got = b.h2_chol_factor_many(ctx, many, opt, threads=3)
        for i in range(len(SIZES)):
            assert got[i] == want[i] and want[i]["updates"] > 0
            for x, y in zip(_state(ctx, many[i]), _state(ctx, alone[i])):
                np.testing.assert_array_equal(x, y)
    finally:
        for Z in alone + many:
            b.h2_matrix_free(Z)
        b.h2_ctx_destroy(ctx)
