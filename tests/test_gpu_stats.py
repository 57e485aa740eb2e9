"""h2_stats of a matrix with device storage: ranks per level and the byte
counts against the definitions, computed from the trees and ranks in
Python."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

from libside import lib_problem, structure  # noqa: E402


def test_stats_match_the_definitions():
    ctx = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        Z, _, _ = lib_problem(ctx, 32, 6, 91, 16, kcap=8)
        try:
            st = b.h2_stats(Z)
            tc, tb, leaf_ids, pairs, adm, near = structure(Z)
            rv, rw = b.h2_get_ranks(Z, 0), b.h2_get_ranks(Z, 1)
            size, father, level = tc["size"], tc["father"], tc["level"]
            assert st["max_rank_rows"] == rv.max() == 6 and st["max_rank_cols"] == rw.max()
            assert st["rank_sum_rows"] == rv.sum()
            want_lv = [int(max([rv[c] for c in range(len(size)) if level[c] == l])) for l in range(st["depth"] + 1)]
            assert st["max_rank_per_level"] == want_lv
            nb = sum(int(size[tb["row"][c]]) * int(size[tb["col"][c]]) for c in near)
            val = nb + sum(int(rv[tb["row"][c]]) * int(rw[tb["col"][c]]) for c in adm)
            for r in (rv, rw):
                val += sum(int(size[t]) * int(r[t]) for t in leaf_ids)
                val += sum(int(r[t]) * int(r[father[t]]) for t in range(len(size)) if father[t] >= 0)
            assert st["value_bytes"] == 8 * val
            k = st["rank_capacity"]
            cap = 2 * (sum(int(size[t]) for t in leaf_ids) * k + len(size) * k * k) + len(adm) * k * k + nb
            assert st["device_bytes"] == 8 * cap
        finally:
            b.h2_matrix_free(Z)
    finally:
        b.h2_ctx_destroy(ctx)
