"""Host-side multi-rank logic of the benchmark harness (gloo, 2 ranks, CPU):
shard ranges cover a batch exactly once, the timing reductions agree, and an
isolated batch split over ranks (oracle) equals the serial batch bit for
bit."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1402_5056_gb300.dist import rank_seed, reduce_max, reduce_sum, shard_range  # noqa: E402


def test_shard_ranges_partition():
    for count in (0, 1, 7, 4096):
        for world in (1, 2, 3, 8):
            got = [shard_range(count, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == count
            assert all(got[i][1] == got[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(5, 2, 2)
    assert len({rank_seed(7, r) for r in range(8)}) == 8


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b, e = shard_range(10, rank, world)
        n = reduce_sum(e - b, dist)
        t = reduce_max(1.0 + rank, dist)
        out[rank] = (n, t)
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (10.0, 2.0)


def _fingerprint(delta):
    """The delta of one update as plain numbers: ranks and every matrix."""
    out = []
    for key in ("V", "W"):
        d = delta[key]
        out.append(sorted(d["rank"].items()))
        out.append([(t, d["leaf"][t].tobytes()) for t in sorted(d["leaf"])])
        out.append([(t, d["transfer"][t].tobytes()) for t in sorted(d["transfer"])])
    out.append([(b, delta["S"][b].tobytes()) for b in sorted(delta["S"])])
    out.append([(b, delta["N"][b].tobytes()) for b in sorted(delta["N"])])
    return out


def _batch_problem():
    from problems import draw_updates, oracle_problem
    Zo, st, _ = oracle_problem(16, 4, 601, 8)
    blocks, A, B = draw_updates(Zo, st, 7, 2)
    return Zo, blocks, A, B


def _shard_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle.update import local_update
        Zo, blocks, A, B = _batch_problem()
        b, e = shard_range(len(blocks), rank, world)
        mine = [_fingerprint(local_update(Zo, blocks[j], A[j], B[j], 1e-6)) for j in range(b, e)]
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        out[rank] = [fp for part in parts for fp in part]
    finally:
        dist.destroy_process_group()


def test_sharded_isolated_batch_equals_serial():
    """Isolated updates need no exchange between ranks: a batch split by
    index over 2 gloo ranks, each rank computing its updates on its own copy
    of the base matrix (the oracle), gives bit for bit the serial batch."""
    from oracle.update import isolated_batch
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    Zo, blocks, A, B = _batch_problem()
    serial = [_fingerprint(d) for d in isolated_batch(Zo, blocks, A, B, 1e-6)]
    assert res[0] == res[1] == serial


def _plan_fingerprint(b, P, first, count):
    """Cluster tasks and coupling tasks of updates first..first+count-1 of a
    host-only plan, update by update (update index relative to `first`)."""
    items, tasks = {}, {}
    st = b.h2_batch_stats(None, P, flops=False)
    for i in range(st["cluster_tasks"]):
        d = b.h2_batch_item_info(P, i)
        items.setdefault(d["update"] - first, []).append((d["side"], d["cluster"], d["k"], d["flags"]))
    for t in range(st["block_tasks"]):
        d = b.h2_batch_task_info(P, t)
        tasks.setdefault(d["update"] - first, []).append((d["block"], d["kt"], d["ls"],
                                                          d["row_item"] >= 0, d["col_item"] >= 0))
    return [(items.get(j, []), tasks.get(j, [])) for j in range(count)]


def _lib_batch():
    import numpy as np
    import synth
    from paper_1402_5056_gb300 import binding as b
    Z = b.h2_matrix_create(None, synth.grid_points_2d(48), 16, 2.0, 0.0, 8)
    tb = b.h2_tree_blocks(Z)
    adm = np.flatnonzero(np.asarray(tb["kind"]) == 1)
    blocks = [int(x) for x in synth.choose_blocks(np.random.default_rng(602), adm, 23)]
    blocks += [0, int(np.flatnonzero(np.asarray(tb["kind"]) == 0)[3])]   # root and a subdivided block
    return b, Z, blocks


def _plan_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b, Z, blocks = _lib_batch()
        lo, hi = shard_range(len(blocks), rank, world)
        P = b.h2_batch_create(None, Z, blocks[lo:hi], 3)
        mine = _plan_fingerprint(b, P, 0, hi - lo)
        b.h2_batch_free(P)
        b.h2_matrix_free(Z)
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        out[rank] = [fp for part in parts for fp in part]
    finally:
        dist.destroy_process_group()


def test_shard_plans_tile_the_batch_plan():
    """The library's plans of the ranks' slices (host-only, gloo ranks on
    CPU) hold, update by update, exactly the cluster tasks and coupling
    tasks of the plan of the whole batch: sharding by index splits the work
    without changing it."""
    b, Z, blocks = _lib_batch()
    P = b.h2_batch_create(None, Z, blocks, 3)
    full = _plan_fingerprint(b, P, 0, len(blocks))
    b.h2_batch_free(P)
    b.h2_matrix_free(Z)
    for world in (2, 3):
        port = _free_port()
        with mp.Manager() as m:
            out = m.dict()
            mp.spawn(_plan_worker, args=(world, port, out), nprocs=world, join=True)
            res = dict(out)
        for r in range(world):
            assert res[r] == full, (world, r)
