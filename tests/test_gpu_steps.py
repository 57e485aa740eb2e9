"""Step-by-step parity of the CUDA update with the oracle's intermediates.

For every cluster task the basis-invariant quantities of steps 2-4 are
compared with the oracle's trace: the Gram matrices R^* R of the basis
R-factors (step 2), B~^* B~ of the weights (step 3), the new rank and
R_t^* R_t of the basis-change matrices (step 4).  The check runs along a
chain of in-place updates with heavy truncation, where ranks differ from
cluster to cluster and ancestor bases have been changed by earlier commits,
in both path modes (certified Gram path with exact fallback, exact only).
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
from oracle.update import apply_delta, local_update  # noqa: E402
from problems import draw_updates, oracle_problem  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_ctx_destroy(c)


def _gram_close(X, Y, tol, what):
    _sym_close(X.T @ X, Y, tol, what)


def _sym_close(G1, Y, tol, what):
    G2 = Y.T @ Y
    scale = max(1.0, float(np.abs(G2).max()))
    err = float(np.abs(G1 - G2).max()) / scale
    assert err <= tol, (what, err)


def _check_items(ctx, P, Zs, b0, A, B, u, eps):
    tr = {}
    d = local_update(Zs, b0, A, B, eps, trace=tr)
    first, last = b.h2_batch_update_items(P, 0)
    for item in range(first, last):
        info = b.h2_batch_item_info(P, item)
        c, k = info["cluster"], info["k"]
        K = k + u
        side = "V" if info["side"] == 0 else "W"
        Gq = b.h2_batch_item_tile(ctx, P, item, 0)[:K, :K]
        _sym_close(Gq, tr["R" + side][c], 1e-12, ("R-factor", side, c))
        Gw = b.h2_batch_item_tile(ctx, P, item, 1)[:K, :K]
        _sym_close(Gw, tr["B" + side][c], 1e-11, ("weights", side, c))
        r = info["rank"]
        if d["margin"] >= 1e-6:
            assert r == d[side]["rank"][c], ("rank", side, c, r, d[side]["rank"][c])
        if r == d[side]["rank"][c]:
            Rt = b.h2_batch_item_tile(ctx, P, item, 2)[:r, :K]
            _gram_close(Rt, tr["Rt" + side][c], 1e-11, ("R_t", side, c))
    return d


@pytest.mark.parametrize("mode", [b.MODE_AUTO, b.MODE_EXACT])
@pytest.mark.parametrize("eps", [0.5, 2.0, 1e-8])
def test_chain_intermediates_match_oracle(ctx, eps, mode):
    N, leaf, k, u = 24, 16, 5, 3
    Zo, st, _ = oracle_problem(N, k, 21, leaf)
    blocks, A, B = draw_updates(Zo, st, 6, u)
    blocks = blocks + [blocks[0]]
    A = A + [A[0] * 0.5]
    B = B + [B[0]]
    Zl, _, _ = lib_problem(ctx, N, k, 21, leaf)
    try:
        for j, b0 in enumerate(blocks):
            Zs = to_oracle(ctx, Zl, Zo)
            P = b.h2_batch_create(ctx, Zl, [b0], u)
            b.h2_batch_set_mode(P, mode)
            try:
                dA = torch.from_numpy(np.asfortranarray(A[j]).ravel(order="F")).cuda()
                dB = torch.from_numpy(np.asfortranarray(B[j]).ravel(order="F")).cuda()
                b.h2_batch_execute(ctx, P, dA.data_ptr(), dB.data_ptr(), eps)
                b.h2_ctx_synchronize(ctx)
                d = _check_items(ctx, P, Zs, b0, A[j], B[j], u, eps)
                b.h2_batch_apply(ctx, P, 0, dA.data_ptr(), dB.data_ptr(), Zl)
            finally:
                b.h2_batch_free(P)
            ref = apply_delta(Zs, d).dense()
            got = to_oracle(ctx, Zl, Zo).dense()
            assert_blockwise_dense(got, ref, Zo.blocks, Zo.V.tree, Zo.W.tree, 1e-10, j)
    finally:
        b.h2_matrix_free(Zl)
