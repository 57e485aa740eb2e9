"""The two paths of the CUDA update: certified Gram path and exact path.

* Where the rank rule keeps every extended rank (eps = 1e-8, random
  factors, admissible blocks) the certificate holds and the certified path
  computes the update; where it truncates (heavy truncation at eps = 0.5,
  clusters without weight) the exact path takes over.
* Both modes (automatic selection, exact only) agree with the oracle on the
  same batch, entry by entry on the assembled matrices, and with each other.
* The new leaf bases of certified updates are orthonormal and span the
  extended bases (V_t, A|_t).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

from blockwise import assert_blockwise_dense  # noqa: E402
from gpu_util import applied_delta, concat_factors  # noqa: E402
from libside import lib_problem, to_oracle  # noqa: E402
from oracle.tree import BlockTree  # noqa: E402
from oracle.update import apply_delta, local_update  # noqa: E402
from problems import draw_updates, oracle_problem  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_ctx_destroy(c)


def _batch(ctx, Zl, blocks, A, B, u, eps, mode):
    P = b.h2_batch_create(ctx, Zl, blocks, u)
    b.h2_batch_set_mode(P, mode)
    Acat, Bcat = concat_factors(P, A, B, u)
    dA = torch.from_numpy(Acat).cuda()
    dB = torch.from_numpy(Bcat).cuda()
    torch.cuda.synchronize()
    b.h2_batch_execute(ctx, P, dA.data_ptr(), dB.data_ptr(), eps)
    b.h2_ctx_synchronize(ctx)
    return P, dA, dB


def _bw(got, ref, Zo, what):
    assert_blockwise_dense(got, ref, Zo.blocks, Zo.V.tree, Zo.W.tree, TOL, what)


def _dense(ctx, Zl, Zo, P, j, dA, dB):
    C = b.h2_matrix_clone(ctx, Zl)
    try:
        b.h2_batch_apply(ctx, P, j, dA.data_ptr(), dB.data_ptr(), C)
        return to_oracle(ctx, C, Zo).dense()
    finally:
        b.h2_matrix_free(C)


def _mixed(Zo, st, count, u, seed):
    blocks, A, B = draw_updates(Zo, st, count, u)
    bt = Zo.blocks
    rng = np.random.default_rng(seed)
    sub = [c for c in range(1, bt.n_blocks) if bt.kind[c] == BlockTree.SUB]
    for c in (0, sub[len(sub) // 2], bt.inadmissible[len(bt.inadmissible) // 2]):
        blocks.append(c)
        A.append(rng.standard_normal((Zo.V.tree.size[bt.row[c]], u)))
        B.append(rng.standard_normal((Zo.W.tree.size[bt.col[c]], u)))
    return blocks, A, B


def _keeps_extended_ranks(Zo, d, u):
    return all(r == Zo.V.rank[t] + u for t, r in d["V"]["rank"].items()) and \
        all(r == Zo.W.rank[t] + u for t, r in d["W"]["rank"].items())


@pytest.mark.parametrize("N,leaf,k,u", [(24, 16, 6, 3), (32, 32, 8, 4)])
def test_certified_path_without_truncation(ctx, N, leaf, k, u):
    """eps = 1e-8: the updates of admissible blocks keep every extended rank
    and take the certified path; updates of the root block and of large
    inadmissible blocks truncate (clusters without admissible blocks have no
    weight, so the rank rule drops their bases) and take the exact path."""
    seed = 300 + N
    Zo, st, _ = oracle_problem(N, k, seed, leaf)
    blocks, A, B = _mixed(Zo, st, 8, u, seed)
    Zl, _, _ = lib_problem(ctx, N, k, seed, leaf)
    try:
        P, dA, dB = _batch(ctx, Zl, blocks, A, B, u, 1e-8, b.MODE_AUTO)
        try:
            exact = b.h2_batch_paths(ctx, P, len(blocks))
            assert exact[:8].sum() == 0, exact
            ph = b.h2_batch_phase_stats(ctx, P, b.PHASES.index("truncate"))
            assert ph["flops"] > 0
            for j, b0 in enumerate(blocks):
                d = local_update(Zo, b0, A[j], B[j], 1e-8)
                full = _keeps_extended_ranks(Zo, d, u)
                assert exact[j] == (0 if full else 1), (j, b0)
                ref = apply_delta(Zo, d).dense()
                got = _dense(ctx, Zl, Zo, P, j, dA, dB)
                _bw(got, ref, Zo, j)
        finally:
            b.h2_batch_free(P)
    finally:
        b.h2_matrix_free(Zl)


def test_truncation_falls_back_to_exact_path(ctx):
    N, leaf, k, u, eps = 24, 16, 6, 3, 0.5
    Zo, st, _ = oracle_problem(N, k, 311, leaf)
    blocks, A, B = _mixed(Zo, st, 8, u, 311)
    Zl, _, _ = lib_problem(ctx, N, k, 311, leaf)
    try:
        P, dA, dB = _batch(ctx, Zl, blocks, A, B, u, eps, b.MODE_AUTO)
        try:
            exact = b.h2_batch_paths(ctx, P, len(blocks))
            truncating = []
            for j, b0 in enumerate(blocks):
                d = local_update(Zo, b0, A[j], B[j], eps)
                full = _keeps_extended_ranks(Zo, d, u)
                truncating.append(not full)
                if not full:
                    # the certificate cannot hold where the rank rule truncates
                    assert exact[j] == 1, j
                ref = apply_delta(Zo, d).dense()
                got = _dense(ctx, Zl, Zo, P, j, dA, dB)
                _bw(got, ref, Zo, j)
            assert any(truncating)
            assert b.h2_batch_phase_stats(ctx, P, b.PHASES.index("exact"))["flops"] > 0
        finally:
            b.h2_batch_free(P)
    finally:
        b.h2_matrix_free(Zl)


@pytest.mark.parametrize("eps", [1e-8, 0.5])
def test_modes_agree_with_oracle_and_each_other(ctx, eps):
    N, leaf, k, u = 32, 16, 6, 4
    Zo, st, _ = oracle_problem(N, k, 321, leaf)
    blocks, A, B = _mixed(Zo, st, 6, u, 321)
    Zl, _, _ = lib_problem(ctx, N, k, 321, leaf)
    try:
        refs = [apply_delta(Zo, local_update(Zo, b0, A[j], B[j], eps)).dense() for j, b0 in enumerate(blocks)]
        got = {}
        for mode in (b.MODE_AUTO, b.MODE_EXACT):
            P, dA, dB = _batch(ctx, Zl, blocks, A, B, u, eps, mode)
            try:
                if mode == b.MODE_EXACT:
                    assert b.h2_batch_paths(ctx, P, len(blocks)).sum() == len(blocks)
                got[mode] = [_dense(ctx, Zl, Zo, P, j, dA, dB) for j in range(len(blocks))]
            finally:
                b.h2_batch_free(P)
        for j, ref in enumerate(refs):
            for mode in got:
                _bw(got[mode][j], ref, Zo, (mode, j))
            _bw(got[b.MODE_AUTO][j], got[b.MODE_EXACT][j], Zo, ("auto vs exact", j))
    finally:
        b.h2_matrix_free(Zl)


def test_certified_leaf_bases_orthonormal_and_spanning(ctx):
    N, leaf, k, u = 32, 32, 8, 4
    Zo, st, _ = oracle_problem(N, k, 331, leaf)
    blocks, A, B = draw_updates(Zo, st, 6, u)
    Zl, _, _ = lib_problem(ctx, N, k, 331, leaf)
    try:
        P, dA, dB = _batch(ctx, Zl, blocks, A, B, u, 1e-8, b.MODE_AUTO)
        try:
            assert b.h2_batch_paths(ctx, P, len(blocks)).sum() == 0
            for j, b0 in enumerate(blocks):
                got_m, _, _ = applied_delta(ctx, Zl, P, j, dA, dB, Zo, b0)
                t0 = Zo.blocks.row[b0]
                r0 = Zo.V.tree.offset[t0]
                for t in Zo.V.tree.descendants(t0):
                    if not Zo.V.tree.is_leaf(t):
                        continue
                    Q = got_m.V.leaf[t]
                    np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-13)
                    off = Zo.V.tree.offset[t] - r0
                    Vt = np.hstack([Zo.V.leaf[t], A[j][off:off + Zo.V.tree.size[t]]])
                    # range(Q) = range(V~_t): the residual of projecting V~_t on Q
                    res = Vt - Q @ (Q.T @ Vt)
                    assert np.linalg.norm(res) <= 1e-12 * np.linalg.norm(Vt)
        finally:
            b.h2_batch_free(P)
    finally:
        b.h2_matrix_free(Zl)


def test_certified_path_on_non_orthonormal_bases(ctx):
    """A truncating update leaves the ancestors of its row cluster with
    non-orthonormal bases (E_t0 <- R_t0 [E_t0; 0]); a later update without
    truncation on a block above it runs the certified path with the general
    (non-block) Gram formulas for those clusters and still matches the oracle
    applied to the library's state."""
    N, leaf, k, u = 32, 16, 6, 3
    Zo, st, _ = oracle_problem(N, k, 341, leaf)
    Zl, _, _ = lib_problem(ctx, N, k, 341, leaf)
    bt = Zo.blocks
    tree = Zo.V.tree
    adm = list(bt.admissible)
    deep = max(adm, key=lambda c: tree.level[bt.row[c]])
    anc = set(tree.predecessors(bt.row[deep])[:-1])
    above = [c for c in adm if bt.row[c] in anc]
    assert above
    high = min(above, key=lambda c: tree.level[bt.row[c]])
    rng = np.random.default_rng(5)
    try:
        for b0, eps, want_exact in ((deep, 0.5, 1), (high, 1e-8, 0)):
            A = rng.standard_normal((tree.size[bt.row[b0]], u))
            B = rng.standard_normal((Zo.W.tree.size[bt.col[b0]], u))
            before = to_oracle(ctx, Zl, Zo)
            d = local_update(before, b0, A, B, eps)
            ref = apply_delta(before, d).dense()
            P, dA, dB = _batch(ctx, Zl, [b0], [A], [B], u, eps, b.MODE_AUTO)
            try:
                assert b.h2_batch_paths(ctx, P, 1)[0] == want_exact, (b0, eps)
                if not want_exact:
                    # some cluster of the update has a non-orthonormal basis
                    first, last = b.h2_batch_update_items(P, 0)
                    dev = 0.0
                    for item in range(first, last):
                        info = b.h2_batch_item_info(P, item)
                        kk = info["k"]
                        G = b.h2_batch_item_tile(ctx, P, item, 0)[:kk, :kk]
                        dev = max(dev, float(np.abs(G - np.eye(kk)).max()) if kk else 0.0)
                    assert dev > 1e-10, dev
                b.h2_batch_apply(ctx, P, 0, dA.data_ptr(), dB.data_ptr(), Zl)
            finally:
                b.h2_batch_free(P)
            got = to_oracle(ctx, Zl, Zo).dense()
            _bw(got, ref, Zo, (b0, eps))
    finally:
        b.h2_matrix_free(Zl)


@pytest.mark.parametrize("above", [False, True])
def test_certificate_at_the_rank_threshold(ctx, above):
    """(eps/2)^2 just below / above lambda_min = sigma_min^2 of the weighted
    matrix of the cluster closest to the threshold (the oracle's G_t = R^* R,
    W_t = B~^* B~).  Below: lambda_min - (eps/2)^2 lies between the float64
    certificate's rounding allowance delta = 8 (levels + 4) (K + 32) u tr(G_t)
    tr(W_t) and the float32 one, 4 (K + 2) 2^-24 tr(G_t W_t), so only the
    float64 factorisation can prove that every rank is kept and the update
    must stay on the certified path.  Above: the rank rule drops a column, the
    certificate must fail and the exact path must reproduce the truncation."""
    N, leaf, k, u = 32, 32, 8, 4
    Zo, st, _ = oracle_problem(N, k, 351, leaf)
    blocks, A, B = draw_updates(Zo, st, 1, u)
    b0 = blocks[0]
    tr = {}
    local_update(Zo, b0, A[0], B[0], 1e-12, tr)
    levels = max(max(Zo.V.tree.level), max(Zo.W.tree.level)) + 1
    cand = []
    for side in ("V", "W"):
        for t, R in tr["R" + side].items():
            G = R.T @ R
            W = tr["B" + side][t].T @ tr["B" + side][t]
            lam = float(tr["sig" + side][t][-1]) ** 2
            K = G.shape[0]
            delta = 8.0 * (levels + 4) * (K + 32) * np.finfo(float).eps * np.trace(G) * np.trace(W)
            fp32 = 4.0 * (K + 2) * 2.0 ** -24 * np.trace(G @ W)
            cand.append((lam, delta, fp32, side, t))
    cand.sort()
    lam, delta, fp32, side, t = cand[0]
    assert delta < 1e-3 * fp32 and cand[1][0] > lam * (1 + 1e-2)
    tau = lam * (1 + 1e-3) if above else lam - np.sqrt(delta * fp32)
    eps = 2.0 * np.sqrt(tau)
    d = local_update(Zo, b0, A[0], B[0], eps)
    full = _keeps_extended_ranks(Zo, d, u)
    assert full != above
    Zl, _, _ = lib_problem(ctx, N, k, 351, leaf)
    try:
        P, dA, dB = _batch(ctx, Zl, blocks, A, B, u, eps, b.MODE_AUTO)
        try:
            assert b.h2_batch_paths(ctx, P, 1)[0] == (1 if above else 0)
            ref = apply_delta(Zo, d).dense()
            got = _dense(ctx, Zl, Zo, P, 0, dA, dB)
            _bw(got, ref, Zo, ("threshold", above))
        finally:
            b.h2_batch_free(P)
    finally:
        b.h2_matrix_free(Zl)
