"""The per-block comparison used by the GPU parity tests (CPU checks).

An error confined to one admissible block must be seen at the block's own
scale, where the whole-matrix norm would hide it; the compressed form for
large problems must agree with the dense slices.
"""
import numpy as np

from blockwise import blockwise_dense, blockwise_h2, leaf_blocks
from problems import oracle_problem


def test_compressed_form_agrees_with_dense_slices():
    Zo, _, _ = oracle_problem(24, 5, 17, 16)
    other = Zo.copy()
    rng = np.random.default_rng(0)
    bt = Zo.blocks
    for b in bt.admissible[::3]:
        other.S[b] = other.S[b] + 1e-7 * rng.standard_normal(other.S[b].shape)
    for b in bt.inadmissible[::4]:
        other.N[b] = other.N[b] + 1e-8 * rng.standard_normal(other.N[b].shape)
    wd, bd = blockwise_dense(other.dense(), Zo.dense(), bt, Zo.V.tree, Zo.W.tree)
    wh, bh = blockwise_h2(other, Zo, leaf_blocks(bt))
    assert bd == bh and abs(wd - wh) <= 1e-6 * wd, (wd, wh, bd, bh)


def test_error_in_one_small_block_is_seen_at_its_scale():
    Zo, _, _ = oracle_problem(24, 5, 19, 16)
    bt = Zo.blocks
    small = min(bt.admissible, key=lambda b: np.linalg.norm(Zo.block_dense(b)))
    other = Zo.copy()
    other.S[small] = other.S[small] * (1 + 1e-9)
    D, R = other.dense(), Zo.dense()
    whole = np.linalg.norm(D - R) / np.linalg.norm(R)
    worst, where = blockwise_dense(D, R, bt, Zo.V.tree, Zo.W.tree)
    assert where == small and abs(worst - 1e-9) < 1e-12
    assert whole < 1e-10 < worst            # the whole-matrix check would pass
    wh, bh = blockwise_h2(other, Zo, [small])
    assert bh == small and abs(wh - 1e-9) < 1e-12
