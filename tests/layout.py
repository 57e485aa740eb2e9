"""The documented layout of a batch's host result (h2_batch_result_offsets,
h2_batch_task_info, h2_batch_item_info), checked from the plan alone.

Each piece is allotted its largest size: a leaf's basis #t x (k_t + u), a
transfer (k_t + u) x (k_f + u), or (k_t + u) x k_f at the subtree root (its
committed E_t0), none at the tree root; a coupling (k_t [+ u]) x (l_s [+ u]),
the u added on each changed side.  The pieces tile [n_cluster_tasks,
result_size) in the order [two-sided couplings][bases and transfers]
[one-sided couplings], without gap or overlap.
"""

LEAF, SUBTREE_ROOT, TREE_ROOT = 1, 2, 8
TWO, ITEM, ONE = 1, 2, 3


def check_result_layout(b, P, Z, u):
    """Asserts the tiling; returns the set of regions that hold pieces."""
    st = b.h2_batch_stats(None, P, flops=False)
    io, to = b.h2_batch_result_offsets(P)
    tc = b.h2_tree_clusters(Z)
    ranks = (b.h2_get_ranks(Z, 0), b.h2_get_ranks(Z, 1))
    pieces = []
    for i in range(st["cluster_tasks"]):
        info = b.h2_batch_item_info(P, i)
        c, K = info["cluster"], info["k"] + u
        length = 0
        if info["flags"] & LEAF:
            length += int(tc["size"][c]) * K
        if not info["flags"] & TREE_ROOT:
            kf = int(ranks[info["side"]][tc["father"][c]])
            length += K * (kf if info["flags"] & SUBTREE_ROOT else kf + u)
        pieces.append((int(io[i]), length, ITEM))
    for t in range(st["block_tasks"]):
        ti = b.h2_batch_task_info(P, t)
        R = ti["kt"] + (u if ti["row_item"] >= 0 else 0)
        C = ti["ls"] + (u if ti["col_item"] >= 0 else 0)
        two = ti["row_item"] >= 0 and ti["col_item"] >= 0
        pieces.append((int(to[t]), R * C, TWO if two else ONE))
    pieces.sort(key=lambda p: (p[0], p[2]))
    order = [p[2] for p in pieces]
    assert order == sorted(order)
    start = st["cluster_tasks"]
    for off, length, _ in pieces:
        assert off == start
        start += length
    assert start == b.h2_batch_result_size(P)
    return {p[2] for p in pieces if p[1] > 0}
