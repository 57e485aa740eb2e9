"""GPU test helpers: factor upload, isolated batches, deltas (test helper)."""
from __future__ import annotations

import numpy as np

from paper_1402_5056_gb300 import binding as b


def concat_factors(P, A_list, B_list, u):
    lenA, lenB = b.h2_batch_factor_sizes(P)
    Acat = np.zeros(lenA)
    Bcat = np.zeros(lenB)
    for j, (A, B) in enumerate(zip(A_list, B_list)):
        ra, oa, rb, ob = b.h2_batch_factor_layout(P, j)
        assert A.shape == (ra, u) and B.shape == (rb, u)
        Acat[oa:oa + ra * u] = np.asarray(A).ravel(order="F")
        Bcat[ob:ob + rb * u] = np.asarray(B).ravel(order="F")
    return Acat, Bcat


def run_isolated(torch, ctx, Z, blocks, A_list, B_list, u, eps):
    """Plan and execute an isolated batch with device factors."""
    P = b.h2_batch_create(ctx, Z, blocks, u)
    Acat, Bcat = concat_factors(P, A_list, B_list, u)
    dA = torch.from_numpy(Acat).to("cuda")
    dB = torch.from_numpy(Bcat).to("cuda")
    torch.cuda.synchronize()
    b.h2_batch_execute(ctx, P, dA.data_ptr(), dB.data_ptr(), eps)
    b.h2_ctx_synchronize(ctx)
    return P, dA, dB


def applied_delta(ctx, Zlib, P, j, dA, dB, Zo, b0):
    """Commit update j into a clone of the library matrix and patch a copy of
    the oracle base matrix Zo with the clone's new parts (subtree bases,
    transfers, affected couplings, nearfield blocks inside b0)."""
    from oracle.tree import BlockTree
    C = b.h2_matrix_clone(ctx, Zlib)
    try:
        b.h2_batch_apply(ctx, P, j, dA.data_ptr(), dB.data_ptr(), C)
        out = Zo.copy()
        bt = Zo.blocks
        t0, s0 = bt.row[b0], bt.col[b0]
        rV = b.h2_get_ranks(C, 0)
        rW = b.h2_get_ranks(C, 1)
        for side, root, basis, ranks in ((0, t0, out.V, rV), (1, s0, out.W, rW)):
            tree = basis.tree
            sub = tree.descendants(root)
            for t in sub:
                basis.rank[t] = int(ranks[t])
            for t in sub:
                if tree.is_leaf(t):
                    basis.leaf[t] = b.h2_get_leaf(ctx, C, side, t, tree.size[t], basis.rank[t])
                if t != 0:
                    basis.transfer[t] = b.h2_get_transfer(ctx, C, side, t, basis.rank[t],
                                                          basis.rank[tree.father[t]])
        Tt = set(out.V.tree.descendants(t0))
        Ts = set(out.W.tree.descendants(s0))
        for c in bt.admissible:
            if bt.row[c] in Tt or bt.col[c] in Ts:
                out.S[c] = b.h2_get_coupling(ctx, C, c, out.V.rank[bt.row[c]], out.W.rank[bt.col[c]])
        near = [c for c in bt.descendants(b0) if bt.kind[c] == BlockTree.NEAR]
        if near:
            N = b.h2_get_nearfield(ctx, C)
            pos = 0
            for c in bt.inadmissible:
                m, n = out.V.tree.size[bt.row[c]], out.W.tree.size[bt.col[c]]
                if c in near:
                    out.N[c] = N[pos:pos + m * n].reshape((m, n), order="F")
                pos += m * n
        return out, rV, rW
    finally:
        b.h2_matrix_free(C)
