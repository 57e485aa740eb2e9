"""Parity of the CUDA approximate inverse (h2_inverse: block Gauss
elimination, Remark on inversion) with the CPU oracle.

* without truncation (eps = 1e-14: only rounding-level singular values
  dropped) the inverse equals numpy's dense inverse of the FEM matrix, per
  assembled block;
* on the 32 x 32-cell problem (n = 961, sigma on a 4 x 4 checkerboard over
  four decades, leaf 32, eta 2, eps = 1e-4): per-block parity with the
  oracle's inverse at 1e-10, equal ranks and update counts,
  ||I - C A||_2 small, and CG preconditioned by the inverse (h2_pcg_inverse)
  within one step of the oracle's;
* the input matrix is consumed (documented), the inverse is a new matrix.
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
from oracle.fem import h2_from_sparse, stiffness  # noqa: E402
from oracle.lr import inverse, pcg  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_ctx_destroy(c)


def _problem(N, seed, leaf, M=4):
    st = synth.streams(seed)
    sigma = synth.checker_sigma(st["sigma"], M, 2)
    K, pts = stiffness(N, 2, sigma, M)
    Zo = h2_from_sparse(K, pts, leaf, 2.0, 1.0 / N)
    return sigma, K, Zo, st


def _lib_inverse(ctx, N, M, sigma, leaf, eps):
    opt = b.options(eps=eps, leaf_size=leaf)
    A = b.h2_build_fem(ctx, 2, N, M, sigma, opt)
    try:
        Cm, info = b.h2_inverse(ctx, A, opt)
    finally:
        b.h2_matrix_free(A)
    return Cm, info


@pytest.mark.parametrize("N,leaf", [(12, 8), (16, 16)])
def test_inverse_without_truncation_is_dense_inverse(ctx, N, leaf):
    sigma, K, Zo, _ = _problem(N, synth.SEED_BASE + 40 + N, leaf)
    Cm, info = _lib_inverse(ctx, N, 4, sigma, leaf, 1e-14)
    try:
        got = to_oracle(ctx, Cm, Zo).dense()
        perm = Zo.V.tree.perm
        ref = np.linalg.inv(K[perm][:, perm].toarray())
        bt, tr = Zo.blocks, Zo.V.tree
        assert_blockwise_dense(got, ref, bt, tr, tr, TOL, "dense inverse", floor=1e-4 * np.linalg.norm(ref))
        assert info["updates"] > 0 and info["max_rank"] > 0
    finally:
        b.h2_matrix_free(Cm)


@pytest.fixture(scope="module")
def config0(ctx):
    sigma, K, Zo, st = _problem(32, synth.SEED_BASE + 0, 32)
    Co, info_o = inverse(Zo.copy(), 1e-4)
    Cm, info = _lib_inverse(ctx, 32, 4, sigma, 32, 1e-4)
    Za = b.h2_build_fem(ctx, 2, 32, 4, sigma, b.options(eps=1e-4, leaf_size=32))
    yield Cm, Co, Zo, K, st, info, info_o, Za
    b.h2_matrix_free(Cm)
    b.h2_matrix_free(Za)


def test_inverse_matches_oracle(ctx, config0):
    Cm, Co, Zo, K, st, info, info_o, _ = config0
    got = to_oracle(ctx, Cm, Co)
    assert list(got.V.rank) == list(Co.V.rank) and list(got.W.rank) == list(Co.W.rank)
    assert info["updates"] == info_o["updates"]
    R = Co.dense()
    bt, tr = Zo.blocks, Zo.V.tree
    assert_blockwise_dense(got.dense(), R, bt, tr, tr, TOL, "inverse", floor=1e-12 * np.linalg.norm(R))
    perm = Zo.V.tree.perm
    A = K[perm][:, perm].toarray()
    n = A.shape[0]
    assert np.linalg.norm(np.eye(n) - got.dense() @ A, 2) <= 1e-2


def test_pcg_with_the_inverse_matches_oracle(ctx, config0):
    Cm, Co, Zo, K, st, info, info_o, Za = config0
    n = K.shape[0]
    perm = Zo.V.tree.perm
    Kp = K[perm][:, perm].tocsr()
    D = Co.dense()
    rhs = synth.fem_rhs(st["rhs"], n)[:, 0][perm]
    x_o, it_o = pcg(lambda v: Kp @ v, rhs, lambda r: D @ r, 1e-10)
    bd = torch.from_numpy(rhs.copy()).cuda()
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    it, rr = b.h2_pcg_inverse(ctx, Za, Cm, bd.data_ptr(), xd.data_ptr(), 1e-10, 200)
    assert rr <= 1e-10
    assert abs(it - it_o) <= 1, (it, it_o)
    x = xd.cpu().numpy()
    assert np.linalg.norm(Kp @ x - rhs) <= 1e-9 * np.linalg.norm(rhs)


def test_inverse_rejects_a_negative_accuracy(ctx):
    sigma, K, Zo, _ = _problem(12, synth.SEED_BASE + 52, 8)
    opt = b.options(eps=1e-4, leaf_size=8)
    A = b.h2_build_fem(ctx, 2, 12, 4, sigma, opt)
    try:
        with pytest.raises(b.H2Error) as e:
            b.h2_inverse(ctx, A, b.options(eps=-1.0, leaf_size=8))
        assert e.value.status == 1
    finally:
        b.h2_matrix_free(A)


def test_inverse_with_rank_cap_matches_oracle(ctx):
    """The rank cap option in the inverse (16 x 16 cells, leaf 16,
    eps 1e-4, cap 4, below the uncapped inverse's largest rank 6)."""
    sigma, K, Zo, _ = _problem(16, synth.SEED_BASE + 71, 16)
    Co, info_o = inverse(Zo.copy(), 1e-4, rank_cap=4)
    opt = b.options(eps=1e-4, leaf_size=16, max_rank=4)
    A = b.h2_build_fem(ctx, 2, 16, 4, sigma, opt)
    try:
        Cm, info = b.h2_inverse(ctx, A, opt)
    finally:
        b.h2_matrix_free(A)
    try:
        got = to_oracle(ctx, Cm, Co)
        assert max(Co.V.rank) == 4
        assert list(got.V.rank) == list(Co.V.rank) and list(got.W.rank) == list(Co.W.rank)
        assert info["updates"] == info_o["updates"]
        R = Co.dense()
        bt, tr = Zo.blocks, Zo.V.tree
        assert_blockwise_dense(got.dense(), R, bt, tr, tr, TOL, "capped inverse", floor=1e-12 * np.linalg.norm(R))
    finally:
        b.h2_matrix_free(Cm)
