"""h2_matvec against the oracle's H^2 product (oracle/matvec.py, pinned to
the dense matrix) on the same matrices: several right-hand sides, alpha
and beta, uneven ranks after updates, rank-0 bases, ragged 3-D point sets,
and the argument checks.  Both sides compute in float64 in different
orders: relative error 1e-12.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

from libside import lib_problem, lib_problem_general, to_oracle  # noqa: E402
from oracle.matvec import matvec  # noqa: E402
from problems import draw_updates, oracle_problem, oracle_problem_general  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_ctx_destroy(c)


def _lib_matvec(ctx, Zl, X, alpha, beta, Y):
    n, nrhs = X.shape
    dX = torch.from_numpy(np.asfortranarray(X).T.copy()).cuda()       # nrhs x n row-major = n x nrhs col-major
    dY = torch.from_numpy(np.asfortranarray(Y).T.copy()).cuda()
    b.h2_matvec(ctx, Zl, nrhs, alpha, dX.data_ptr(), n, beta, dY.data_ptr(), Y.shape[0])
    b.h2_ctx_synchronize(ctx)
    return dY.cpu().numpy().T


def _check(ctx, Zl, Zo, nrhs, alpha, beta, seed):
    rng = np.random.default_rng(seed)
    n = Zo.W.tree.size[0]
    m = Zo.V.tree.size[0]
    X = rng.standard_normal((n, nrhs))
    Y = rng.standard_normal((m, nrhs)) if beta != 0.0 else np.full((m, nrhs), np.nan)
    got = _lib_matvec(ctx, Zl, X, alpha, beta, Y)
    ref = matvec(Zo, X, alpha, beta, Y if beta != 0.0 else None)
    assert np.all(np.isfinite(got))
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= TOL, err


@pytest.mark.parametrize("nrhs,alpha,beta", [(1, 1.0, 0.0), (3, 2.0, -0.5), (17, -1.0, 1.0)])
def test_matvec_matches_oracle(ctx, nrhs, alpha, beta):
    Zo, _, _ = oracle_problem(32, 6, 501, 16)
    Zl, _, _ = lib_problem(ctx, 32, 6, 501, 16)
    try:
        _check(ctx, Zl, Zo, nrhs, alpha, beta, 7)
    finally:
        b.h2_matrix_free(Zl)


def test_matvec_after_truncating_updates(ctx):
    """Uneven ranks (truncation) and a grown rank capacity."""
    N, leaf, k, u = 24, 16, 5, 4
    Zo, st, _ = oracle_problem(N, k, 503, leaf)
    Zl, _, _ = lib_problem(ctx, N, k, 503, leaf)
    try:
        blocks, A, B = draw_updates(Zo, st, 4, u)
        for j, b0 in enumerate(blocks):
            a = torch.from_numpy(np.ascontiguousarray(A[j].T)).cuda()
            bb = torch.from_numpy(np.ascontiguousarray(B[j].T)).cuda()
            b.h2_lowrank_update(ctx, Zl, b0, u, a.data_ptr(), A[j].shape[0], bb.data_ptr(), B[j].shape[0],
                                0.3 if j % 2 else 1e-8)
        b.h2_ctx_synchronize(ctx)
        Zc = to_oracle(ctx, Zl, Zo)
        assert len(set(Zc.V.rank)) > 1
        _check(ctx, Zl, Zc, 4, 1.5, 0.25, 9)
    finally:
        b.h2_matrix_free(Zl)


@pytest.mark.parametrize("dim,k", [(3, 4), (2, 0)])
def test_matvec_general_points(ctx, dim, k):
    pts = np.random.default_rng(dim).uniform(size=(700, dim))
    Zo, _, _ = oracle_problem_general(pts, k, 505 + dim, 20)
    Zl, _, _ = lib_problem_general(ctx, pts, k, 505 + dim, 20)
    try:
        _check(ctx, Zl, Zo, 2, 1.0, 0.0, 11)
    finally:
        b.h2_matrix_free(Zl)


def test_matvec_argument_checks(ctx):
    Zl, _, _ = lib_problem(ctx, 20, 4, 507, 16)
    try:
        n = 400
        buf = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
        with pytest.raises(b.H2Error):
            b.h2_matvec(ctx, Zl, 1, 1.0, buf.data_ptr(), n, 0.0, buf.data_ptr() + 8 * (n // 2), n)   # overlap
        with pytest.raises(b.H2Error):
            b.h2_matvec(ctx, Zl, 1, 1.0, buf.data_ptr(), n - 1, 0.0, buf.data_ptr() + 8 * n, n)      # ldx
        b.h2_matvec(ctx, Zl, 0, 1.0, 0, n, 0.0, 0, n)   # nothing to do
    finally:
        b.h2_matrix_free(Zl)


def test_block_to_dense(ctx):
    """h2_block_to_dense on admissible, inadmissible, subdivided and root
    blocks against the oracle's block assembly (expanded bases)."""
    from oracle.tree import BlockTree
    Zo, _, _ = oracle_problem(24, 5, 509, 16)
    Zl, _, _ = lib_problem(ctx, 24, 5, 509, 16)
    try:
        bt = Zo.blocks
        sub = [c for c in range(1, bt.n_blocks) if bt.kind[c] == BlockTree.SUB]
        for blk in (0, bt.admissible[3], bt.admissible[-1], bt.inadmissible[5], sub[len(sub) // 2]):
            ref = Zo.block_dense(blk)
            nt, ns = ref.shape
            out = torch.full((ns, nt + 3), float("nan"), dtype=torch.float64, device="cuda")   # ld = nt + 3
            b.h2_block_to_dense(ctx, Zl, blk, out.data_ptr(), nt + 3)
            b.h2_ctx_synchronize(ctx)
            got = out.cpu().numpy().T[:nt]
            assert np.linalg.norm(got - ref) <= TOL * max(np.linalg.norm(ref), 1e-300), blk
    finally:
        b.h2_matrix_free(Zl)
