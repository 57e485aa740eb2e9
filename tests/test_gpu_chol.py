"""Parity of the CUDA approximate Cholesky factorisation (h2_chol_factor;
Section 7's preconditioner, built with the algorithms of Section 3) with
the CPU oracle (oracle.chol).

* without truncation (eps = 1e-14: only rounding-level singular values
  dropped) the factor equals the oracle's and numpy's dense Cholesky
  factor of the FEM matrix, per assembled block of the lower triangle;
* on the 32 x 32-cell problem (n = 961, sigma on a 4 x 4 checkerboard over
  four decades, leaf 32, eta 2, eps = 1e-4) and on a 24 x 24-cell problem
  with leaf 16: per-block parity with the oracle's factor at 1e-10, equal
  ranks and update counts, fewer updates than the LR, L L^* close to A;
* h2_chol_solve equals the oracle's solve; CG preconditioned by the factor
  (h2_pcg_chol) takes the oracle's number of steps +-1; the power-iteration
  Err (h2_chol_error) equals the oracle's.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

import synth  # noqa: E402
from blockwise import assert_blockwise_dense  # noqa: E402
from libside import to_oracle  # noqa: E402
from oracle.chol import chol_factor, chol_solve, lower  # noqa: E402
from oracle.fem import h2_from_sparse, stiffness  # noqa: E402
from oracle.lr import pcg  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_ctx_destroy(c)


def _problem(N, seed, leaf, M=4, dim=2):
    st = synth.streams(seed)
    sigma = synth.checker_sigma(st["sigma"], M, dim)
    K, pts = stiffness(N, dim, sigma, M)
    Zo = h2_from_sparse(K, pts, leaf, 2.0, 1.0 / N)
    return sigma, K, Zo, st


def _both(ctx, N, leaf, eps, seed, M=4, dim=2):
    sigma, K, Zo, st = _problem(N, seed, leaf, M, dim)
    info_o = chol_factor(Zo, eps)
    opt = b.options(eps=eps, leaf_size=leaf)
    Z = b.h2_build_fem(ctx, dim, N, M, sigma, opt)
    info = b.h2_chol_factor(ctx, Z, opt)
    return Z, Zo, K, info, info_o, st, sigma


@pytest.mark.parametrize("N,leaf,dim,M", [(16, 16, 2, 4), (20, 8, 2, 4), (8, 16, 3, 2)])
def test_chol_without_truncation_is_dense_cholesky(ctx, N, leaf, dim, M):
    Z, Zo, K, info, info_o, _, _ = _both(ctx, N, leaf, 1e-14, synth.SEED_BASE + 80 + N, M, dim)
    try:
        got = np.tril(to_oracle(ctx, Z, Zo).dense())
        bt, tr = Zo.blocks, Zo.V.tree
        perm = tr.perm
        ref = np.linalg.cholesky(K[perm][:, perm].toarray())
        fl = 1e-4 * np.linalg.norm(ref)
        assert_blockwise_dense(got, lower(Zo), bt, tr, tr, TOL, "oracle", floor=fl)
        assert_blockwise_dense(got, ref, bt, tr, tr, TOL, "dense Cholesky", floor=fl)
        assert info["updates"] > 0 and info["max_rank"] > 0
    finally:
        b.h2_matrix_free(Z)


@pytest.fixture(scope="module", params=[(32, 32, 0), (24, 16, 60)], ids=["32x32_leaf32", "24x24_leaf16"])
def factored(ctx, request):
    N, leaf, seed = request.param
    Z, Zo, K, info, info_o, st, sigma = _both(ctx, N, leaf, 1e-4, synth.SEED_BASE + seed)
    A = b.h2_build_fem(ctx, 2, N, 4, sigma, b.options(eps=1e-4, leaf_size=leaf))
    yield Z, Zo, K, info, info_o, st, A
    b.h2_matrix_free(Z)
    b.h2_matrix_free(A)


def test_chol_matches_oracle(ctx, factored):
    Z, Zo, K, info, info_o, _, _ = factored
    got = to_oracle(ctx, Z, Zo)
    assert list(got.V.rank) == list(Zo.V.rank) and list(got.W.rank) == list(Zo.W.rank)
    assert info["updates"] == info_o["updates"]
    R = lower(Zo)
    bt, tr = Zo.blocks, Zo.V.tree
    G = np.tril(got.dense())
    assert_blockwise_dense(G, R, bt, tr, tr, TOL, "Cholesky factor", floor=1e-12 * np.linalg.norm(R))
    perm = tr.perm
    A = K[perm][:, perm].toarray()
    assert np.linalg.norm(A - G @ G.T) <= 1e-5 * np.linalg.norm(A)


def test_chol_solve_and_pcg_match_oracle(ctx, factored):
    Z, Zo, K, info, info_o, st, A = factored
    n = K.shape[0]
    perm = Zo.V.tree.perm
    rhs = synth.fem_rhs(np.random.default_rng(6), n, 2)[perm]
    X = torch.from_numpy(np.asfortranarray(rhs).ravel(order="F")).cuda()
    b.h2_chol_solve(ctx, Z, 2, X.data_ptr(), n)
    got = X.cpu().numpy().reshape((n, 2), order="F")
    want = chol_solve(Zo, rhs)
    assert np.linalg.norm(got - want) <= TOL * np.linalg.norm(want)
    Kp = K[perm][:, perm].tocsr()
    r1 = synth.fem_rhs(st["rhs"], n)[:, 0][perm]
    x_o, it_o = pcg(lambda v: Kp @ v, r1, lambda r: chol_solve(Zo, r), 1e-10)
    bd = torch.from_numpy(r1.copy()).cuda()
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    it, rr = b.h2_pcg_chol(ctx, A, Z, bd.data_ptr(), xd.data_ptr(), 1e-10, 200)
    assert rr <= 1e-10 and abs(it - it_o) <= 1, (it, it_o)
    assert np.linalg.norm(Kp @ xd.cpu().numpy() - r1) <= 1e-9 * np.linalg.norm(r1)


def test_chol_takes_fewer_updates_than_lr(ctx):
    sigma, K, Zo, _ = _problem(32, synth.SEED_BASE + 0, 32)
    opt = b.options(eps=1e-4, leaf_size=32)
    Z1 = b.h2_build_fem(ctx, 2, 32, 4, sigma, opt)
    Z2 = b.h2_build_fem(ctx, 2, 32, 4, sigma, opt)
    try:
        ic = b.h2_chol_factor(ctx, Z1, opt)
        il = b.h2_lr_factor(ctx, Z2, opt)
        assert ic["updates"] < il["updates"]
    finally:
        b.h2_matrix_free(Z1)
        b.h2_matrix_free(Z2)


def test_chol_power_error_matches_oracle(ctx, factored):
    """||I - (L L^*)^-1 A||_2 by the power iteration (Section 7, Err)."""
    from oracle.lr import power_error
    Z, Zo, K, info, info_o, st, A = factored
    n = K.shape[0]
    perm = Zo.V.tree.perm
    Kp = K[perm][:, perm].tocsr()
    want = power_error(lambda v: Kp @ v, lambda r: chol_solve(Zo, r), n, 20, seed=3)
    vd = torch.from_numpy(np.random.default_rng(3).standard_normal(n)).cuda()
    got = b.h2_chol_error(ctx, A, Z, vd.data_ptr(), 20)
    assert abs(got - want) <= 1e-6 * max(want, 1e-12) + 1e-14, (got, want)
    assert want < 1e-2


@pytest.mark.parametrize("N,leaf,dim,M,eps,seed,cap", [(24, 16, 2, 4, 1e-6, 60, 3), (8, 16, 3, 2, 1e-4, 70, 0)],
                         ids=["24x24_cap3", "3d_8"])
def test_chol_capped_and_3d_match_oracle(ctx, N, leaf, dim, M, eps, seed, cap):
    """The rank cap option (reading 6) and a 3D problem (8^3 cells in Kuhn
    tetrahedra): per block at 1e-10, equal ranks and update counts."""
    sigma, K, Zo, _ = _problem(N, synth.SEED_BASE + seed, leaf, M, dim)
    info_o = chol_factor(Zo, eps, rank_cap=cap or None)
    opt = b.options(eps=eps, leaf_size=leaf, max_rank=cap)
    Z = b.h2_build_fem(ctx, dim, N, M, sigma, opt)
    try:
        info = b.h2_chol_factor(ctx, Z, opt)
        got = to_oracle(ctx, Z, Zo)
        if cap:
            assert info_o["max_rank"] == cap == info["max_rank"]
        assert list(got.V.rank) == list(Zo.V.rank) and list(got.W.rank) == list(Zo.W.rank)
        assert info["updates"] == info_o["updates"]
        R = lower(Zo)
        bt, tr = Zo.blocks, Zo.V.tree
        assert_blockwise_dense(np.tril(got.dense()), R, bt, tr, tr, TOL, "Cholesky factor",
                               floor=1e-12 * np.linalg.norm(R))
    finally:
        b.h2_matrix_free(Z)
