"""Parity of the CUDA H^2-LR path with the CPU oracle (Sections 3 and 7).

* the FEM matrix: the library's cluster and block trees equal the oracle's,
  its nearfield leaves equal the oracle's assembly (2D and 3D);
* the factorisation without truncation (eps = 1e-14: only rounding-level
  singular values dropped) equals the oracle's and dense Doolittle LU, per
  assembled block;
* the factorisation of the 32 x 32-cell problem (n = 961, sigma on a 4 x 4
  checkerboard over four decades, leaf 32, eta 2, eps = 1e-4): per-block
  parity with the oracle's factor at 1e-10, equal ranks, ||A - LR|| small,
  conjugate-gradient steps to 1e-10 within one of the oracle's, the
  block substitutions and the power-iteration error against the oracle's.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402

import synth  # noqa: E402
from blockwise import assert_blockwise_dense, blockwise_dense  # noqa: E402
from libside import to_oracle  # noqa: E402
from oracle.fem import h2_from_sparse, stiffness  # noqa: E402
from oracle.lr import lr_factor, lr_solve, lu_doolittle, pcg, power_error  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_ctx_destroy(c)


def _problem(dim, N, M, seed, leaf, eta=2.0):
    st = synth.streams(seed)
    sigma = synth.checker_sigma(st["sigma"], M, dim)
    K, pts = stiffness(N, dim, sigma, M)
    Zo = h2_from_sparse(K, pts, leaf, eta, 1.0 / N)
    return sigma, K, Zo, st


def _lib(ctx, dim, N, M, sigma, leaf, eps, eta=2.0):
    return b.h2_build_fem(ctx, dim, N, M, sigma, b.options(eps=eps, eta=eta, leaf_size=leaf))


@pytest.mark.parametrize("dim,N,M,leaf", [(2, 32, 4, 32), (2, 20, 4, 8), (3, 8, 2, 64), (3, 10, 2, 16)])
def test_fem_matrix_matches_oracle(ctx, dim, N, M, leaf):
    sigma, K, Zo, _ = _problem(dim, N, M, synth.SEED_BASE + 10 + N, leaf)
    Z = _lib(ctx, dim, N, M, sigma, leaf, 1e-4)
    try:
        tb = b.h2_tree_blocks(Z)
        assert list(tb["row"]) == Zo.blocks.row and list(tb["col"]) == Zo.blocks.col
        assert list(tb["kind"]) == Zo.blocks.kind
        np.testing.assert_array_equal(b.h2_tree_permutation(Z), Zo.V.tree.perm)
        assert max(b.h2_get_ranks(Z, 0)) == 0 and max(b.h2_get_ranks(Z, 1)) == 0
        got = to_oracle(ctx, Z, Zo)
        R = Zo.dense()
        # structurally zero entries come out of the element sums as rounding
        # noise on both sides: blocks of such entries are compared on the
        # scale of the matrix (floor 1e-3 ||K||_F, 1e-16 absolute at 1e-13)
        worst, where = blockwise_dense(got.dense(), R, Zo.blocks, Zo.V.tree, Zo.W.tree,
                                       floor=1e-3 * np.linalg.norm(R))
        assert worst <= 1e-13, (where, worst)
    finally:
        b.h2_matrix_free(Z)


def _factor_both(ctx, dim, N, M, leaf, eps, seed):
    sigma, K, Zo, st = _problem(dim, N, M, seed, leaf)
    A = Zo.copy()
    info_o = lr_factor(Zo, eps)
    Z = _lib(ctx, dim, N, M, sigma, leaf, eps)
    info = b.h2_lr_factor(ctx, Z, b.options(eps=eps, leaf_size=leaf))
    return Z, Zo, A, K, info, info_o, st


@pytest.mark.parametrize("N,leaf", [(16, 16), (20, 8)])
def test_lr_without_truncation_is_dense_lu(ctx, N, leaf):
    # eps = 1e-14 (block-relative) instead of 0: at eps = 0 every rounding-
    # level singular value would be kept and the ranks would depend on
    # rounding; 1e-14 drops exactly those and truncates nothing else
    Z, Zo, A, K, info, info_o, _ = _factor_both(ctx, 2, N, 4, leaf, 1e-14, synth.SEED_BASE + 20 + N)
    try:
        got = to_oracle(ctx, Z, Zo).dense()
        bt, tr = Zo.blocks, Zo.V.tree
        # fill-in blocks whose exact value is (nearly) zero come out at the
        # rounding level of the factor on both sides (a 6 x 6 block of norm
        # 2.6e-15 in a factor of norm 640): compared absolutely at
        # 1e-14 ||R||_F (floor 1e-4 ||R||_F at 1e-10), every block above the
        # floor relatively at 1e-10
        fl = 1e-4 * np.linalg.norm(got)
        assert_blockwise_dense(got, Zo.dense(), bt, tr, tr, TOL, "oracle", floor=fl)
        assert_blockwise_dense(got, lu_doolittle(A.dense()), bt, tr, tr, TOL, "dense LU", floor=fl)
        # the number of updates is not compared here: temporaries whose
        # singular values reach down to 1e-14 keep or drop their rounding-
        # level directions by rounding, which changes the column groups
        assert info["updates"] > 0 and info["max_rank"] > 0
    finally:
        b.h2_matrix_free(Z)


@pytest.fixture(scope="module")
def config0(ctx):
    """The 32 x 32-cell problem factorised by both sides at eps = 1e-4."""
    Z, Zo, A, K, info, info_o, st = _factor_both(ctx, 2, 32, 4, 32, 1e-4, synth.SEED_BASE + 0)
    Za = _lib(ctx, 2, 32, 4, synth.checker_sigma(synth.streams(synth.SEED_BASE + 0)["sigma"], 4, 2), 32, 1e-4)
    yield Z, Zo, A, K, info, info_o, st, Za
    b.h2_matrix_free(Z)
    b.h2_matrix_free(Za)


def test_lr_factor_matches_oracle(ctx, config0):
    Z, Zo, A, K, info, info_o, _, _ = config0
    got = to_oracle(ctx, Z, Zo)
    bt, tr = Zo.blocks, Zo.V.tree
    assert list(got.V.rank) == list(Zo.V.rank)
    assert list(got.W.rank) == list(Zo.W.rank)
    assert info["updates"] == info_o["updates"]
    R = Zo.dense()
    assert_blockwise_dense(got.dense(), R, bt, tr, tr, TOL, "factor", floor=1e-12 * np.linalg.norm(R))
    # the factor reproduces A to about the truncation accuracy
    D = got.dense()
    n = D.shape[0]
    Lm, Rm = np.tril(D, -1) + np.eye(n), np.triu(D)
    Ad = A.dense()
    assert np.linalg.norm(Ad - Lm @ Rm) <= 1e-6 * np.linalg.norm(Ad)


def test_lr_solve_matches_oracle(ctx, config0):
    Z, Zo, A, K, info, info_o, st, _ = config0
    n = K.shape[0]
    perm = Zo.V.tree.perm
    rhs = synth.fem_rhs(np.random.default_rng(5), n, 3)[perm]
    X = torch.from_numpy(np.asfortranarray(rhs).ravel(order="F")).cuda()
    b.h2_lr_solve(ctx, Z, 3, X.data_ptr(), n)
    got = X.cpu().numpy().reshape((n, 3), order="F")
    want = lr_solve(Zo, rhs)
    assert np.linalg.norm(got - want) <= TOL * np.linalg.norm(want)


def test_pcg_iterations_match_oracle(ctx, config0):
    Z, Zo, A, K, info, info_o, st, Za = config0
    n = K.shape[0]
    perm = Zo.V.tree.perm
    Kp = K[perm][:, perm].tocsr()
    rhs = synth.fem_rhs(st["rhs"], n)[:, 0][perm]
    x_o, it_o = pcg(lambda v: Kp @ v, rhs, lambda r: lr_solve(Zo, r), 1e-10)
    bd = torch.from_numpy(rhs.copy()).cuda()
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    it, rr = b.h2_pcg(ctx, Za, Z, bd.data_ptr(), xd.data_ptr(), 1e-10, 200)
    assert rr <= 1e-10
    assert abs(it - it_o) <= 1, (it, it_o)
    x = xd.cpu().numpy()
    assert np.linalg.norm(Kp @ x - rhs) <= 1e-9 * np.linalg.norm(rhs)
    # without a preconditioner CG needs far more steps (sigma spans four
    # decades: it does not reach 1e-10 in 200 steps)
    xd.zero_()
    it0, rr0 = b.h2_pcg(ctx, Za, None, bd.data_ptr(), xd.data_ptr(), 1e-10, 200)
    assert it0 == 200 and rr0 > 1e-10


def test_power_error_matches_oracle(ctx, config0):
    Z, Zo, A, K, info, info_o, st, Za = config0
    n = K.shape[0]
    perm = Zo.V.tree.perm
    Kp = K[perm][:, perm].tocsr()
    want = power_error(lambda v: Kp @ v, lambda r: lr_solve(Zo, r), n, 20, seed=3)
    v0 = np.random.default_rng(3).standard_normal(n)
    vd = torch.from_numpy(v0).cuda()
    got = b.h2_lr_error(ctx, Za, Z, vd.data_ptr(), 20)
    assert abs(got - want) <= 1e-6 * max(want, 1e-12) + 1e-14, (got, want)
    assert want < 1e-2


def test_command_line_example():
    """python -m paper_1402_5056_gb300.fem_lr: factor, PCG and error on a
    small problem."""
    from paper_1402_5056_gb300 import fem_lr
    out = fem_lr.main(["--cells", "24", "--eps", "1e-4"])
    assert out["n"] == 23 * 23
    assert out["cg_relres"] <= 1e-10 and out["cg_iterations"] <= 6
    assert out["factor"]["updates"] > 0 and 0 < out["err_power"] < 1e-2


@pytest.mark.parametrize("cap", [3, 6])
def test_lr_with_rank_cap_matches_oracle(ctx, cap):
    """The rank cap option (h2_options.max_rank, off by default; the paper
    sets no cap): every new basis keeps at most ``cap`` leading singular
    directions, on both sides, and the factor is still parity-equal."""
    N, leaf, eps = 24, 16, 1e-6
    sigma, K, Zo, _ = _problem(2, N, 4, synth.SEED_BASE + 60, leaf)
    info_o = lr_factor(Zo, eps, rank_cap=cap)
    opt = b.options(eps=eps, leaf_size=leaf, max_rank=cap)
    Z = b.h2_build_fem(ctx, 2, N, 4, sigma, opt)
    try:
        info = b.h2_lr_factor(ctx, Z, opt)
        got = to_oracle(ctx, Z, Zo)
        assert info_o["max_rank"] == cap and info["max_rank"] == cap
        assert list(got.V.rank) == list(Zo.V.rank) and list(got.W.rank) == list(Zo.W.rank)
        assert info["updates"] == info_o["updates"]
        R = Zo.dense()
        bt, tr = Zo.blocks, Zo.V.tree
        assert_blockwise_dense(got.dense(), R, bt, tr, tr, TOL, "capped factor", floor=1e-12 * np.linalg.norm(R))
    finally:
        b.h2_matrix_free(Z)


def test_rank_cap_out_of_range_is_rejected(ctx):
    sigma, K, Zo, _ = _problem(2, 12, 4, synth.SEED_BASE + 61, 8)
    opt = b.options(eps=1e-4, leaf_size=8)
    Z = b.h2_build_fem(ctx, 2, 12, 4, sigma, opt)
    try:
        for cap in (-1, 32):
            with pytest.raises(b.H2Error) as e:
                b.h2_lr_factor(ctx, Z, b.options(eps=1e-4, leaf_size=8, max_rank=cap))
            assert e.value.status == 1
    finally:
        b.h2_matrix_free(Z)


def test_lr_3d_matches_oracle(ctx):
    """The factorisation of a 3D problem (8^3 cells in Kuhn tetrahedra,
    n = 343, sigma on a 2 x 2 x 2 checkerboard, leaf 16, eps 1e-4): per-block
    parity with the oracle at 1e-10, equal ranks and update counts."""
    N, M, leaf, eps = 8, 2, 16, 1e-4
    sigma, K, Zo, _ = _problem(3, N, M, synth.SEED_BASE + 70, leaf)
    info_o = lr_factor(Zo, eps)
    Z = _lib(ctx, 3, N, M, sigma, leaf, eps)
    try:
        info = b.h2_lr_factor(ctx, Z, b.options(eps=eps, leaf_size=leaf))
        got = to_oracle(ctx, Z, Zo)
        assert info_o["max_rank"] > 0
        assert list(got.V.rank) == list(Zo.V.rank) and list(got.W.rank) == list(Zo.W.rank)
        assert info["updates"] == info_o["updates"]
        R = Zo.dense()
        bt, tr = Zo.blocks, Zo.V.tree
        assert_blockwise_dense(got.dense(), R, bt, tr, tr, TOL, "3D factor", floor=1e-12 * np.linalg.norm(R))
    finally:
        b.h2_matrix_free(Z)
