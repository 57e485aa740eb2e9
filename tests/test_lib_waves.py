"""Host logic of h2_lowrank_update_sequence: its waves against a direct
formulation of the footprints (no GPU).

An update of the block b0 = (t0, s0) reads the bases of T_t0 and the
ancestors of t0 (row side), of T_s0 and the ancestors of s0 (column side),
and the couplings of every admissible block in the rows of those row
clusters or the columns of those column clusters; it writes the bases of
T_t0 and T_s0 and the couplings of the blocks with row in T_t0 or column in
T_s0.  Update j must come after every earlier update whose writes it reads
and not before an earlier update that reads what j writes; the waves are
the earliest such.
"""
import numpy as np
import pytest

import synth
from paper_1402_5056_gb300 import binding as b


def _footprints(Z, blocks):
    tc = b.h2_tree_clusters(Z)
    tb = b.h2_tree_blocks(Z)
    father = [int(x) for x in tc["father"]]
    nc = len(father)
    sons = [[] for _ in range(nc)]
    for c in range(nc):
        if father[c] >= 0:
            sons[father[c]].append(c)

    def subtree(c):
        out, stack = [], [c]
        while stack:
            x = stack.pop()
            out.append(x)
            stack.extend(sons[x])
        return out

    def ancestors(c):
        out = []
        while father[c] >= 0:
            c = father[c]
            out.append(c)
        return out

    kind, row, col = np.asarray(tb["kind"]), np.asarray(tb["row"]), np.asarray(tb["col"])
    adm = np.flatnonzero(kind == 1)
    by_row = {}
    by_col = {}
    for blk in adm:
        by_row.setdefault(int(row[blk]), set()).add(int(blk))
        by_col.setdefault(int(col[blk]), set()).add(int(blk))
    fps = []
    for b0 in blocks:
        t0, s0 = int(row[b0]), int(col[b0])
        Tt, Ts = subtree(t0), subtree(s0)
        At, As = ancestors(t0), ancestors(s0)
        rd = {("r", c) for c in Tt + At} | {("c", c) for c in Ts + As}
        wr = {("r", c) for c in Tt} | {("c", c) for c in Ts}
        for c in Tt + At:
            rd |= {("S", x) for x in by_row.get(c, ())}
        for c in Ts + As:
            rd |= {("S", x) for x in by_col.get(c, ())}
        for c in Tt:
            wr |= {("S", x) for x in by_row.get(c, ())}
        for c in Ts:
            wr |= {("S", x) for x in by_col.get(c, ())}
        fps.append((rd, wr))
    return fps


def _expected_waves(fps):
    waves = []
    for j, (rd, wr) in enumerate(fps):
        w = 0
        for i in range(j):
            ri, wi = fps[i]
            if wi & rd:
                w = max(w, waves[i] + 1)
            if ri & wr:
                w = max(w, waves[i])
        waves.append(w)
    return waves


@pytest.mark.parametrize("case", ["grid", "ragged2d", "ragged3d"])
def test_waves_match_the_footprints(case):
    if case == "grid":
        pts = synth.grid_points_2d(32)
    else:   # leaves at several levels
        dim = 2 if case == "ragged2d" else 3
        pts = np.random.default_rng(dim).uniform(size=(900, dim)) ** 2
    Z = b.h2_matrix_create(None, pts, 16, 2.0, 0.0, 6)
    try:
        tb = b.h2_tree_blocks(Z)
        kind = np.asarray(tb["kind"])
        rng = np.random.default_rng(17)
        adm = np.flatnonzero(kind == 1)
        other = np.flatnonzero(kind != 1)
        blocks = [int(x) for x in rng.choice(adm, 50)] + [int(x) for x in rng.choice(other, 8)]
        blocks = blocks + blocks[:3] + [0]          # repeats and the root
        rng.shuffle(blocks)
        wave, n = b.h2_sequence_waves(Z, blocks)
        exp = _expected_waves(_footprints(Z, blocks))
        assert list(wave) == exp
        assert n == max(exp) + 1
        assert n < len(blocks)
        # a repeated block always comes after its earlier copy
        last = {}
        for j, blk in enumerate(blocks):
            if blk in last:
                assert wave[j] > wave[last[blk]]
            last[blk] = j
    finally:
        b.h2_matrix_free(Z)


def test_waves_of_an_empty_sequence():
    Z = b.h2_matrix_create(None, synth.grid_points_2d(16), 16, 2.0, 0.0, 4)
    try:
        wave, n = b.h2_sequence_waves(Z, [])
        assert len(wave) == 0 and n == 0
    finally:
        b.h2_matrix_free(Z)
