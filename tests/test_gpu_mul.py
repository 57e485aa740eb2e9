"""Parity of the CUDA product h2_mul with the CPU oracle (Section 3; Cases 1
and 2 of Section 6).

Three H^2 matrices on one block tree with different nested bases and
couplings (the seeded draws of the update tests), and every combination of
block kinds of the triple (x, y, z) = ((t,s), (s,r), (t,r)) that the tree
offers -- subdivided targets, admissible targets of two subdivided factors
(temporaries), low-rank and dense terms: Z|_z += alpha X|_x Y|_y by the
library and by the oracle, compared per assembled block of Z at 1e-10
(block norms floored at 1e-12 of the matrix for rounding-level blocks),
with equal ranks, at an accuracy that truncates nothing (1e-12) and one
that truncates (0.3); X and Y unchanged; the product in place (X = Y = Z).
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
from oracle.lr import mul  # noqa: E402
from problems import block_triples, oracle_problem  # noqa: E402

N, LEAF = 16, 8
SPECS = {"X": (3, 81), "Y": (4, 82), "Z": (2, 83)}   # rank, seed


@pytest.fixture(scope="module")
def ctx():
    c = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    b.h2_ctx_destroy(c)


@pytest.fixture(scope="module")
def mats(ctx):
    ora = {k: oracle_problem(N, r, sd, LEAF)[0] for k, (r, sd) in SPECS.items()}
    lib = {k: lib_problem(ctx, N, r, sd, LEAF, kcap=16)[0] for k, (r, sd) in SPECS.items()}
    yield ora, lib
    for Zl in lib.values():
        b.h2_matrix_free(Zl)


@pytest.mark.parametrize("eps", [1e-12, 0.3])
def test_mul_matches_oracle_for_every_kind_of_triple(ctx, mats, eps):
    ora, lib = mats
    bt, ct = ora["Z"].blocks, ora["Z"].V.tree
    triples = block_triples(bt, ct)
    assert len(triples) >= 8
    Xd, Yd = ora["X"].dense(), ora["Y"].dense()
    for key, (x, y, z) in sorted(triples.items()):
        Zo = ora["Z"].copy()
        mul(Zo, ora["X"], ora["Y"], -0.7, x, y, z, eps)
        Zl = b.h2_matrix_clone(ctx, lib["Z"])
        try:
            b.h2_mul(ctx, -0.7, lib["X"], x, lib["Y"], y, Zl, z, eps)
            got = to_oracle(ctx, Zl, Zo)
            R = Zo.dense()
            assert_blockwise_dense(got.dense(), R, bt, ct, ct, 1e-10, (key, eps), floor=1e-12 * np.linalg.norm(R))
            assert list(got.V.rank) == list(Zo.V.rank) and list(got.W.rank) == list(Zo.W.rank), key
            # the factors are read only
            np.testing.assert_array_equal(to_oracle(ctx, lib["X"], ora["X"]).dense(), Xd)
            np.testing.assert_array_equal(to_oracle(ctx, lib["Y"], ora["Y"]).dense(), Yd)
        finally:
            b.h2_matrix_free(Zl)


def test_mul_in_place_matches_oracle(ctx, mats):
    """X = Y = Z (the factorisation's Schur update): every term is computed
    from the matrix as it was when the product started."""
    ora, lib = mats
    bt, ct = ora["Z"].blocks, ora["Z"].V.tree
    triples = block_triples(bt, ct)
    for key, (x, y, z) in sorted(triples.items())[:6]:
        Zo = ora["Z"].copy()
        mul(Zo, Zo, Zo, 0.4, x, y, z, 1e-8)
        Zl = b.h2_matrix_clone(ctx, lib["Z"])
        try:
            b.h2_mul(ctx, 0.4, Zl, x, Zl, y, Zl, z, 1e-8)
            got = to_oracle(ctx, Zl, Zo)
            R = Zo.dense()
            assert_blockwise_dense(got.dense(), R, bt, ct, ct, 1e-10, key, floor=1e-12 * np.linalg.norm(R))
        finally:
            b.h2_matrix_free(Zl)


def test_mul_rejects_mismatched_blocks(ctx, mats):
    ora, lib = mats
    bt = ora["Z"].blocks
    adm = bt.admissible[0]
    with pytest.raises(b.H2Error) as e:
        b.h2_mul(ctx, 1.0, lib["X"], adm, lib["Y"], adm, lib["Z"], adm, 1e-8)
    assert e.value.status == 1
