"""The host result of h2_batch_execute_host, decoded piece by piece.

Every piece (new rank, leaf basis, transfer matrix, coupling) must equal,
bit for bit, what h2_batch_apply commits into a copy of the matrix; a
page-locked destination (copies overlapping the update, the graph replays
included) and a pageable one give the same bytes.  Cases: certified updates
(one-sided couplings copied early), truncating updates (their early copies
are packed again and re-sent), the exact path for everything, and bases that
are not orthonormal (no early copies for their clusters).

The compact result (h2_batch_execute_host_compact) must flag exactly the
one-sided couplings that are the unchanged S_b padded with zeros and give
every other piece the same bytes as the full result.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

from gpu_util import concat_factors  # noqa: E402
from layout import ONE, check_result_layout  # noqa: E402
from libside import lib_problem  # noqa: E402
from problems import draw_updates, oracle_problem  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_ctx_destroy(c)


def _pinned(n):
    return torch.zeros(n, dtype=torch.float64).pin_memory().numpy()


def _decode_check(ctx, P, Zl, n_updates, res, dA, dB, u):
    io, to = b.h2_batch_result_offsets(P)
    st = b.h2_batch_stats(None, P, flops=False)
    tc = b.h2_tree_clusters(Zl)
    tb = b.h2_tree_blocks(Zl)
    tasks = [b.h2_batch_task_info(P, t) for t in range(st["block_tasks"])]
    pieces = 0
    for j in range(n_updates):
        C = b.h2_matrix_clone(ctx, Zl)
        try:
            b.h2_batch_apply(ctx, P, j, dA.data_ptr(), dB.data_ptr(), C)
            r = (b.h2_get_ranks(C, 0), b.h2_get_ranks(C, 1))
            first, last = b.h2_batch_update_items(P, j)
            for i in range(first, last):
                info = b.h2_batch_item_info(P, i)
                side, c = info["side"], info["cluster"]
                ri = int(res[i])
                assert ri == res[i] and ri == r[side][c], (j, i)
                off = int(io[i])
                size = int(tc["size"][c])
                if info["flags"] & 1:
                    V = res[off:off + size * ri].reshape((size, ri), order="F")
                    np.testing.assert_array_equal(V, b.h2_get_leaf(ctx, C, side, c, size, ri))
                    off += size * (info["k"] + u)
                    pieces += 1
                if not info["flags"] & 8:
                    rf = int(r[side][tc["father"][c]])
                    E = res[off:off + ri * rf].reshape((ri, rf), order="F")
                    np.testing.assert_array_equal(E, b.h2_get_transfer(ctx, C, side, c, ri, rf))
                    pieces += 1
            for t, ti in enumerate(tasks):
                if ti["update"] != j:
                    continue
                blk = ti["block"]
                rt, rs = int(r[0][tb["row"][blk]]), int(r[1][tb["col"][blk]])
                if ti["row_item"] < 0:
                    assert rt == ti["kt"]
                if ti["col_item"] < 0:
                    assert rs == ti["ls"]
                S = res[int(to[t]):int(to[t]) + rt * rs].reshape((rt, rs), order="F")
                np.testing.assert_array_equal(S, b.h2_get_coupling(ctx, C, blk, rt, rs))
                pieces += 1
        finally:
            b.h2_matrix_free(C)
    return pieces


def _check_compact(ctx, P, Zl, u, full, compact, copied):
    """Pieces outside the flagged couplings: the bytes of the full result;
    flagged couplings: one-sided, and in the full result the unchanged
    coupling padded with zeros."""
    _, to = b.h2_batch_result_offsets(P)
    keep = np.ones(len(full), bool)
    for t in np.flatnonzero(copied):
        ti = b.h2_batch_task_info(P, int(t))
        assert ti["row_item"] < 0 or ti["col_item"] < 0
        R = ti["kt"] + (u if ti["row_item"] >= 0 else 0)
        Cn = ti["ls"] + (u if ti["col_item"] >= 0 else 0)
        piece = full[int(to[t]):int(to[t]) + R * Cn].reshape((R, Cn), order="F")
        pad = np.zeros((R, Cn))
        pad[:ti["kt"], :ti["ls"]] = b.h2_get_coupling(ctx, Zl, ti["block"], ti["kt"], ti["ls"])
        np.testing.assert_array_equal(piece, pad)
        keep[int(to[t]):int(to[t]) + R * Cn] = False
    np.testing.assert_array_equal(compact[keep], full[keep])


def _run(ctx, Zl, blocks, A, B, u, eps, mode):
    P = b.h2_batch_create(ctx, Zl, blocks, u)
    try:
        assert ONE in check_result_layout(b, P, Zl, u)
        b.h2_batch_set_mode(P, mode)
        Acat, Bcat = concat_factors(P, A, B, u)
        n = b.h2_batch_result_size(P)
        pa = torch.from_numpy(Acat).pin_memory().numpy()
        pb = torch.from_numpy(Bcat).pin_memory().numpy()
        pinned = _pinned(n)
        runs = []
        for _ in range(3):            # eager, captured, replayed
            pinned[:] = np.nan
            b.h2_batch_execute_host(ctx, P, pa, pb, eps, pinned)
            runs.append(pinned.copy())
        pageable = b.h2_batch_execute_host(ctx, P, Acat, Bcat, eps)
        for r in runs:
            np.testing.assert_array_equal(r, pageable)
        flags = []
        for _ in range(3):            # compact: eager, captured, replayed
            pinned[:] = np.nan
            _, copied = b.h2_batch_execute_host_compact(ctx, P, pa, pb, eps, pinned)
            _check_compact(ctx, P, Zl, u, pageable, pinned, copied)
            flags.append(copied)
        res_pg, copied_pg = b.h2_batch_execute_host_compact(ctx, P, Acat, Bcat, eps)
        np.testing.assert_array_equal(res_pg, pageable)
        for f in flags:
            np.testing.assert_array_equal(f, copied_pg)
        pinned[:] = np.nan            # and back to the full result
        b.h2_batch_execute_host(ctx, P, pa, pb, eps, pinned)
        np.testing.assert_array_equal(pinned, pageable)
        if mode == b.MODE_EXACT:
            assert copied_pg.sum() == 0
        paths = b.h2_batch_paths(ctx, P, len(blocks))
        dA = torch.from_numpy(Acat).cuda()
        dB = torch.from_numpy(Bcat).cuda()
        b.h2_batch_execute(ctx, P, dA.data_ptr(), dB.data_ptr(), eps)
        b.h2_ctx_synchronize(ctx)
        pieces = _decode_check(ctx, P, Zl, len(blocks), pageable, dA, dB, u)
        return paths, pieces, int(copied_pg.sum())
    finally:
        b.h2_batch_free(P)


@pytest.mark.parametrize("eps,mode,exact", [(1e-8, b.MODE_AUTO, 0), (0.5, b.MODE_AUTO, 1),
                                            (1e-8, b.MODE_EXACT, 1)])
def test_host_result_pieces(ctx, eps, mode, exact):
    N, leaf, k, u = 32, 16, 6, 3
    Zo, st, _ = oracle_problem(N, k, 401, leaf)
    Zl, _, _ = lib_problem(ctx, N, k, 401, leaf)
    try:
        blocks, A, B = draw_updates(Zo, st, 6, u)
        paths, pieces, n_copied = _run(ctx, Zl, blocks, A, B, u, eps, mode)
        if exact:
            assert paths.sum() >= 1
        else:
            assert paths.sum() == 0 and n_copied > 0
        assert pieces > 6
    finally:
        b.h2_matrix_free(Zl)


def test_host_result_non_orthonormal_bases(ctx):
    """After a truncating update in place, the ancestors of its row cluster
    have bases that are not orthonormal: their one-sided couplings are not
    copied early and the late pass sends them."""
    N, leaf, k, u = 32, 16, 6, 3
    Zo, st, _ = oracle_problem(N, k, 409, leaf)
    Zl, _, _ = lib_problem(ctx, N, k, 409, leaf)
    bt = Zo.blocks
    tree = Zo.V.tree
    adm = list(bt.admissible)
    deep = max(adm, key=lambda c: tree.level[bt.row[c]])
    anc = set(tree.predecessors(bt.row[deep])[:-1])
    above = [c for c in adm if bt.row[c] in anc]
    rng = np.random.default_rng(9)
    try:
        # u x rows, row-major = rows x u column-major
        A0 = torch.from_numpy(rng.standard_normal((u, tree.size[bt.row[deep]]))).cuda()
        B0 = torch.from_numpy(rng.standard_normal((u, Zo.W.tree.size[bt.col[deep]]))).cuda()
        b.h2_lowrank_update(ctx, Zl, deep, u, A0.data_ptr(), A0.shape[1], B0.data_ptr(), B0.shape[1], 0.5)
        b.h2_ctx_synchronize(ctx)
        blocks = above[:4]
        A = [rng.standard_normal((tree.size[bt.row[c]], u)) for c in blocks]
        B = [rng.standard_normal((Zo.W.tree.size[bt.col[c]], u)) for c in blocks]
        paths, pieces, _ = _run(ctx, Zl, blocks, A, B, u, 1e-8, b.MODE_AUTO)
        assert pieces > 4
    finally:
        b.h2_matrix_free(Zl)
