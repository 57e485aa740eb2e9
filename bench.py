#!/usr/bin/env python3
"""Benchmark of the isolated batched local low-rank update on one GB300.

Workload: 4096 rank-8 local low-rank updates Z|_{t0 x s0} <- trunc_eps(
Z|_{t0 x s0} + A B^*) (Section 5 of arXiv:1402.5056) on an H^2 matrix over
the 256 x 256 grid of cell centres (n = 65,536, leaf size 32, eta = 2),
nested orthonormal bases of rank 16, couplings N(0,1)/16, target blocks
drawn uniformly from the admissible leaves, A and B N(0,1), eps = 1e-8,
float64.  Isolated mode: every update reads the same base matrix and writes
its own result.  A step is one execution of the whole batch.

Output: one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead (bounded samples of the same workload on the host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

# kernels behind each phase of h2_batch_phase_stats
PHASE_KERNELS = {"base_weights": "k_orth_local+k_vgram+k_bgram+k_bgram_down", "rfactor": "k_fgram+k_fgram_inner",
                 "norms": "k_fnorms", "weights": "k_fweights+k_fweights_wide", "truncate": "k_certify",
                 "bases": "k_fbasis", "reproject": "k_onesided+k_reproject",
                 "exact": "exact path (k_blockweights..k_truncate)"}

# DRAM bytes (read + write) per cluster task of a phase's kernels, from ncu
# captures on the 1024-update batch of the same matrix (13,220 cluster
# tasks): dram__bytes_read.sum + dram__bytes_write.sum summed over the
# phase's launches of one execution, divided by its cluster tasks; the
# roofline's `traffic` scales them to one launch of the benchmark batch.
# Valid for the kernel versions of this commit.
TRAFFIC_BYTES_PER_TASK = {"k_fweights+k_fweights_wide": 5815, "k_certify": 10972, "k_fbasis": 15438}

METRIC = "H²-LR setup s & low-rank updates/s, mixed vs FP64 GPU at equal ε; % roofline"
UNIT = "updates/s"
WORK = dict(N=256, leaf=32, eta=2.0, k=16, u=8, eps=1e-8, count=4096, seed=synth.SEED_BASE + 1)
WORKLOAD_NAME = ("isolated H2 low-rank updates: 4096 rank-8 updates, 256x256-point H2 matrix "
                 "(n=65536, leaf 32, eta 2, k=16), eps=1e-8, float64")
# Float64 FMA peak of one GB300: 2 DFMA per clock per SM (confirmed by an
# FMA throughput measurement: 1.254 TFLOP/s at 2070 MHz) x 152 SMs x 2 flop
# x 2.070 GHz; the roofline denominator of this ALU-bound path.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def _hbm_peak():
    """Copy bandwidth measured on the GB300s (GB/s), else the
    fallback figure of an earlier measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


HBM_PEAK_GBS, HBM_PEAK_KIND = _hbm_peak()
FP64_PEAK_SOURCE = "derived: 152 SM x 2 DFMA/clk x 2 flop x 2070 MHz (DFMA probe: 1.254 TFLOP/s measured)"
L2_FLUSH_BYTES = 512 << 20


def lib_workload(b, ctx, total: int = WORK["count"], lo: int = 0, hi: int | None = None):
    """Library-side H^2 matrix of the workload (the same on every rank) and
    updates lo..hi-1 of a batch of `total` updates drawn from it (blocks and
    factors are drawn in update order, so a shard of the batch is the same
    whichever ranks share it)."""
    hi = total if hi is None else hi
    w = WORK
    pts = synth.grid_points_2d(w["N"])
    Z = b.h2_matrix_create(ctx, pts, w["leaf"], w["eta"], 0.0, w["k"])
    tc = b.h2_tree_clusters(Z)
    tb = b.h2_tree_blocks(Z)
    nc = len(tc["offset"])
    leaves = [(t, int(tc["size"][t])) for t in range(nc) if tc["son0"][t] < 0]
    pairs = [(int(tc["son0"][t]), int(tc["son1"][t])) for t in range(nc) if tc["son0"][t] >= 0]
    adm = np.flatnonzero(tb["kind"] == 1)
    near = np.flatnonzero(tb["kind"] == 2)
    st = synth.streams(w["seed"])
    V = synth.nested_orthonormal_bases(st["bases"], leaves, pairs, nc, w["k"])
    W = synth.nested_orthonormal_bases(st["bases"], leaves, pairs, nc, w["k"])
    S = synth.gaussian_couplings(st["couplings"], len(adm), w["k"], 1.0 / w["k"])
    Nf = synth.gaussian_nearfield(st["couplings"], [(int(tc["size"][tb["row"][c]]), int(tc["size"][tb["col"][c]]))
                                                    for c in near], 1.0 / 16)
    blocks = [int(x) for x in synth.choose_blocks(st["blocks"], adm, total)]
    rows = [int(tc["size"][tb["row"][c]]) for c in blocks]
    cols = [int(tc["size"][tb["col"][c]]) for c in blocks]
    synth.update_factors(st["ab"], rows[:lo], cols[:lo], w["u"])       # the other ranks' updates
    A, B = synth.update_factors(st["ab"], rows[lo:hi], cols[lo:hi], w["u"])
    blocks = blocks[lo:hi]
    if ctx is not None:
        b.h2_set_basis(ctx, Z, 0, *V)
        b.h2_set_basis(ctx, Z, 1, *W)
        b.h2_set_couplings(ctx, Z, S)
        b.h2_set_nearfield(ctx, Z, Nf)
    return Z, blocks, A, B


def matvec_work(b, Z):
    """Algorithmic bytes (nrhs = 1) and flops per right-hand side of one
    H2 matrix times vector: every coupling, nearfield value, leaf basis and
    transfer matrix once, x read and y written once."""
    tc = b.h2_tree_clusters(Z)
    tb = b.h2_tree_blocks(Z)
    rv, rw = b.h2_get_ranks(Z, 0).astype(np.int64), b.h2_get_ranks(Z, 1).astype(np.int64)
    size = np.asarray(tc["size"], dtype=np.int64)
    father = np.asarray(tc["father"])
    leaf = np.asarray(tc["son0"]) < 0
    kind, row, col = np.asarray(tb["kind"]), np.asarray(tb["row"]), np.asarray(tb["col"])
    adm, near = kind == 1, kind == 2
    s_vals = int((rv[row[adm]] * rw[col[adm]]).sum())
    n_vals = int((size[row[near]] * size[col[near]]).sum())
    leaf_vals = int((size[leaf] * rv[leaf]).sum() + (size[leaf] * rw[leaf]).sum())
    inner = father >= 0
    tr_vals = int((rv[inner] * rv[father[inner]]).sum() + (rw[inner] * rw[father[inner]]).sum())
    n = int(size[0])
    vals = s_vals + n_vals + leaf_vals + tr_vals
    return 8 * (vals + 2 * n), 2 * vals


def matvec_measure(b, ctx, Z, stream, flush, steps):
    import torch
    n = int(b.h2_tree_clusters(Z)["size"][0])
    nbytes, flops = matvec_work(b, Z)
    out = {}
    for nrhs in (1, 16):
        X = torch.randn(nrhs * n, dtype=torch.float64, device="cuda")
        Y = torch.zeros(nrhs * n, dtype=torch.float64, device="cuda")
        for _ in range(3):
            b.h2_matvec(ctx, Z, nrhs, 1.0, X.data_ptr(), n, 0.0, Y.data_ptr(), n)
        ts = []
        for s in range(steps):
            flush.fill_(s)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.h2_matvec(ctx, Z, nrhs, 1.0, X.data_ptr(), n, 0.0, Y.data_ptr(), n)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = sum(ts) / len(ts)
        mb = nbytes + 16 * n * (nrhs - 1)
        gbs = mb / (ms * 1e-3) / 1e9
        tf = nrhs * flops / (ms * 1e-3) / 1e12
        out["nrhs_%d" % nrhs] = {"ms": ms, "algorithmic_bytes": mb, "GB/s": gbs, "frac_hbm": gbs / HBM_PEAK_GBS,
                                 "gflop": nrhs * flops / 1e9, "TFLOP/s": tf, "frac_fp64_peak": tf / FP64_PEAK_TFLOPS}
    out["peak_source"] = "HBM %.0f GB/s (%s); FP64: %s" % (HBM_PEAK_GBS, HBM_PEAK_KIND, FP64_PEAK_SOURCE)
    return out


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during timing."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus_id = (bus_id or "").lower()
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        rows = [r for r in self.rows if len(r) >= 10]
        if self.bus_id:
            mine = [r for r in rows if self.bus_id.endswith(r[1].lower()[-12:]) or r[1].lower().endswith(self.bus_id[-12:])]
            rows = mine or rows
        if not rows:
            return None
        idx = rows[0][0]
        rows = [r for r in rows if r[0] == idx]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        mx = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


_ORACLE = {}


def _oracle_init():
    """Host process of the CPU baseline: builds the oracle's matrix and the
    batch once (one BLAS thread; spawned, never forked from a GPU process)."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from problems import draw_updates, oracle_problem
    w = WORK
    Zo, st, _ = oracle_problem(w["N"], w["k"], w["seed"], w["leaf"], w["eta"])
    _ORACLE["Z"] = Zo
    _ORACLE["batch"] = draw_updates(Zo, st, w["count"], w["u"])


def _oracle_updates(idx):
    from oracle.update import local_update
    blocks, A, B = _ORACLE["batch"]
    for j in idx:
        local_update(_ORACLE["Z"], blocks[j], A[j], B[j], WORK["eps"])
    return len(idx)


class OraclePool:
    """The oracle as it stands on `procs` host processes (one per core)."""

    def __init__(self, procs: int):
        import multiprocessing as mp
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(procs, initializer=_oracle_init)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.procs = procs
        self.pool.map(_oracle_updates, [[] for _ in range(procs)])   # every process built its matrix

    def run(self, start: int, count: int):
        """Updates start .. start+count-1 of the batch (mod 4096), spread
        over the processes; returns the wall time."""
        n = WORK["count"]
        idx = [(start + i) % n for i in range(count)]
        chunks = [idx[p::self.procs] for p in range(self.procs)]
        t0 = time.perf_counter()
        self.pool.map(_oracle_updates, chunks, chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


LR_EPS = 1e-4


def lr_problem(cells: int):
    """The 2D FEM problems: 32 x 32 cells, 4 x 4 checkerboard (seed + 0), and
    512 x 512 cells, 16 x 16 checkerboard (seed + 2); other sizes use a 4 x 4
    checkerboard and their own seed."""
    if cells == 32:
        return 4, synth.SEED_BASE + 0
    if cells == 512:
        return 16, synth.SEED_BASE + 2
    return 4, synth.SEED_BASE + 100 + cells


def lr_measure(b, ctx, cells_list, reps: int, oracle_cells, chol=False):
    """FEM matrix, H^2-LR setup (build + factorisation, wall clock; the
    recursion is driven from the host, every arithmetic step on the device),
    PCG steps to 1e-10 and the power-iteration error; the oracle's setup
    timed beside it on the host for the sizes in oracle_cells.  chol: the
    approximate Cholesky factorisation instead (h2_chol_factor)."""
    import torch
    out = {}
    for cells in cells_list:
        M, seed = lr_problem(cells)
        st = synth.streams(seed)
        sigma = synth.checker_sigma(st["sigma"], M, 2)
        opt = b.options(eps=LR_EPS, eta=2.0, leaf_size=32)
        builds, factors, info = [], [], None
        F = A = None
        for rep in range(reps):
            for X in (F, A):
                if X is not None:
                    b.h2_matrix_free(X)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            A = b.h2_build_fem(ctx, 2, cells, M, sigma, opt)
            F = b.h2_build_fem(ctx, 2, cells, M, sigma, opt) if rep == 0 else b.h2_matrix_clone(ctx, A)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            info = b.h2_chol_factor(ctx, F, opt) if chol else b.h2_lr_factor(ctx, F, opt)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            builds.append(t1 - t0)
            factors.append(t2 - t1)
        n = (cells - 1) ** 2
        perm = b.h2_tree_permutation(A)
        rhs = synth.fem_rhs(st["rhs"], n)[:, 0][perm]
        bd = torch.from_numpy(np.ascontiguousarray(rhs)).cuda()
        xd = torch.zeros(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, rr = (b.h2_pcg_chol if chol else b.h2_pcg)(ctx, A, F, bd.data_ptr(), xd.data_ptr(), 1e-10, 100)
        torch.cuda.synchronize()
        cg_s = time.perf_counter() - t0
        v0 = torch.from_numpy(np.random.default_rng(3).standard_normal(n)).cuda()
        err = (b.h2_chol_error if chol else b.h2_lr_error)(ctx, A, F, v0.data_ptr(), 20)
        rec = {"n": n, "cells": cells, "checker": M, "eps": LR_EPS, "leaf": 32, "eta": 2.0,
               "setup_s": min(factors), "factor_s_all": factors, "build_s": min(builds),
               "updates": info["updates"], "products": info["products"], "max_rank": info["max_rank"],
               "seconds_by_activity": info.get("seconds"),
               "cg_iterations": it, "cg_relres": rr, "cg_s": cg_s, "err_power": err}
        if cells in oracle_cells:
            sys.path.insert(0, os.path.join(ROOT, "tests"))
            from oracle.fem import h2_from_sparse, stiffness
            from oracle.chol import chol_factor, chol_solve
            from oracle.lr import lr_factor, lr_solve, pcg
            t0 = time.perf_counter()
            K, pts = stiffness(cells, 2, sigma, M)
            Zo = h2_from_sparse(K, pts, 32, 2.0, 1.0 / cells)
            t1 = time.perf_counter()
            (chol_factor if chol else lr_factor)(Zo, LR_EPS)
            t2 = time.perf_counter()
            Kp = K[Zo.V.tree.perm][:, Zo.V.tree.perm].tocsr()
            solve = chol_solve if chol else lr_solve
            _, it_o = pcg(lambda v: Kp @ v, rhs, lambda r: solve(Zo, r), 1e-10)
            rec["oracle"] = {"setup_s": t2 - t1, "build_s": t1 - t0, "cg_iterations": it_o, "cores": 1,
                             "kind": "oracle"}
        out["%dx%d" % (cells, cells)] = rec
        b.h2_matrix_free(F)
        b.h2_matrix_free(A)
    return out


def lr_batch_measure(b, ctx, count: int, lo: int, hi: int, chol=False):
    """A batch of independent 2D FEM problems of uneven sizes (cells per
    side uniform in lo..hi, 4 x 4 checkerboards, seeded): factorised one after
    the other (h2_lr_factor) and side by side (h2_lr_factor_many, one host
    thread and stream per problem in flight); factorisations per second of
    both, and whether the results agree (update counts).  chol: the
    Cholesky factorisation (h2_chol_factor, h2_chol_factor_many)."""
    factor = b.h2_chol_factor if chol else b.h2_lr_factor
    factor_many = b.h2_chol_factor_many if chol else b.h2_lr_factor_many
    import torch
    rng = np.random.default_rng(synth.SEED_BASE + 4)
    cells = [int(c) for c in rng.integers(lo, hi + 1, count)]
    sigmas = [synth.checker_sigma(np.random.default_rng(synth.SEED_BASE + 400 + i), 4, 2) for i in range(count)]
    opt = b.options(eps=LR_EPS, eta=2.0, leaf_size=32)
    build = lambda: [b.h2_build_fem(ctx, 2, c, 4, sg, opt) for c, sg in zip(cells, sigmas)]
    Zs = build()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    one = [factor(ctx, Z, opt) for Z in Zs]
    torch.cuda.synchronize()
    seq = time.perf_counter() - t0
    for Z in Zs:
        b.h2_matrix_free(Z)
    Zs = build()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    many = factor_many(ctx, Zs, opt, threads=count)
    torch.cuda.synchronize()
    par = time.perf_counter() - t0
    for Z in Zs:
        b.h2_matrix_free(Z)
    return {"problems": count, "cells": cells, "n": [(c - 1) ** 2 for c in cells], "eps": LR_EPS,
            "one_at_a_time_s": seq, "side_by_side_s": par,
            "factorisations_per_s": {"one_at_a_time": count / seq, "side_by_side": count / par},
            "speedup": seq / par,
            "same_update_counts": [o["updates"] for o in one] == [m["updates"] for m in many]}


def inverse_measure(b, ctx, cells_list, oracle_cells):
    """Approximate inverse of the 2D FEM matrix (h2_inverse, block Gauss
    elimination): setup wall time, CG steps to 1e-10 preconditioned by the
    inverse, ||I - C A||_2 estimated by the power iteration; the oracle's
    inverse timed beside it for the sizes in oracle_cells."""
    import torch
    out = {}
    for cells in cells_list:
        M, seed = lr_problem(cells)
        st = synth.streams(seed)
        sigma = synth.checker_sigma(st["sigma"], M, 2)
        opt = b.options(eps=LR_EPS, eta=2.0, leaf_size=32)
        A = b.h2_build_fem(ctx, 2, cells, M, sigma, opt)
        W = b.h2_build_fem(ctx, 2, cells, M, sigma, opt)   # consumed by the inversion
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Cm, info = b.h2_inverse(ctx, W, opt)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        b.h2_matrix_free(W)
        n = (cells - 1) ** 2
        perm = b.h2_tree_permutation(A)
        rhs = synth.fem_rhs(st["rhs"], n)[:, 0][perm]
        bd = torch.from_numpy(np.ascontiguousarray(rhs)).cuda()
        xd = torch.zeros(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, rr = b.h2_pcg_inverse(ctx, A, Cm, bd.data_ptr(), xd.data_ptr(), 1e-10, 100)
        torch.cuda.synchronize()
        cg_s = time.perf_counter() - t0
        rec = {"n": n, "cells": cells, "checker": M, "eps": LR_EPS, "leaf": 32, "eta": 2.0, "setup_s": setup,
               "updates": info["updates"], "products": info["products"], "max_rank": info["max_rank"],
               "cg_iterations": it, "cg_relres": rr, "cg_s": cg_s}
        if cells in oracle_cells:
            from oracle.fem import h2_from_sparse, stiffness
            from oracle.lr import inverse, pcg
            K, pts = stiffness(cells, 2, sigma, M)
            Zo = h2_from_sparse(K, pts, 32, 2.0, 1.0 / cells)
            t0 = time.perf_counter()
            Co, _ = inverse(Zo, LR_EPS)
            t1 = time.perf_counter()
            D = Co.dense()
            Kp = K[Zo.V.tree.perm][:, Zo.V.tree.perm].tocsr()
            _, it_o = pcg(lambda v: Kp @ v, rhs, lambda r: D @ r, 1e-10)
            rec["oracle"] = {"setup_s": t1 - t0, "cg_iterations": it_o, "cores": 1, "kind": "oracle"}
        out["%dx%d" % (cells, cells)] = rec
        b.h2_matrix_free(Cm)
        b.h2_matrix_free(A)
    return out


def run_reference(args, rank):
    if rank != 0:
        return 0
    procs = args.cpu_procs or os.cpu_count() or 1
    op = OraclePool(procs)
    sample = args.ref_sample * procs
    per_step = []
    start = 0
    for step in range(args.warmup + args.steps):
        dt = op.run(start, sample)
        start += sample
        if step >= args.warmup:
            per_step.append(dt)
    op.close()
    wall_tot = sum(per_step)
    done_tot = sample * len(per_step)
    value = done_tot / wall_tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall_tot / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME,
                       "step": "%d consecutive updates of the batch per step (bounded sample)" % sample,
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": "%d updates per step x %d steps, in batch order, on %d host processes "
                                       "(one per core, one BLAS thread each)" % (sample, args.steps, procs)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--matvec-steps", type=int, default=10, help="timed h2_matvec calls per case (0: none)")
    ap.add_argument("--mode", choices=("auto", "exact"), default="auto",
                    help="path of the timed steps: auto (certified path, exact path where it fails) or exact")
    ap.add_argument("--exact-steps", type=int, default=2,
                    help="executions with every update on the exact path (reported beside the line)")
    ap.add_argument("--serial-steps", type=int, default=2,
                    help="executions with every phase on one stream, for per-phase device times")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-sample", type=int, default=24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lr-cells", default="32,64",
                    help="comma-separated cells per side of the 2D FEM H2-LR problems to time ('' for none)")
    ap.add_argument("--lr-reps", type=int, default=3)
    ap.add_argument("--chol-cells", default="32,64,128",
                    help="comma-separated cells per side of the 2D FEM Cholesky factorisations to time ('' for none)")
    ap.add_argument("--batch-problems", type=int, default=16,
                    help="independent FEM problems of the uneven batch (0: none)")
    ap.add_argument("--inv-cells", default="32",
                    help="comma-separated cells per side of the 2D FEM approximate inverses to time ('' for none)")
    ap.add_argument("--cpu-procs", type=int, default=0, help="host processes of the CPU baseline (0: all cores)")
    ap.add_argument("--count", type=int, default=WORK["count"],
                    help="updates per batch (profiling runs use fewer; the benchmark uses 4096)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1402_5056_gb300 import binding as b
    from paper_1402_5056_gb300.dist import reduce_max, shard_range

    stream = torch.cuda.current_stream()
    ctx = b.h2_ctx_create(torch.cuda.current_device(), stream.cuda_stream)
    # one batch of world x count updates on the same matrix, sharded by index
    # (isolated updates: no exchange between ranks)
    total = world * args.count
    lo, hi = shard_range(total, rank, world)
    Z, blocks, A, B = lib_workload(b, ctx, total, lo, hi)
    w = WORK
    t_plan = time.perf_counter()
    P = b.h2_batch_create(ctx, Z, blocks, w["u"])
    plan_s = time.perf_counter() - t_plan
    if args.mode == "exact":
        b.h2_batch_set_mode(P, b.MODE_EXACT)   # every update through the exact path
    lenA, lenB = b.h2_batch_factor_sizes(P)
    Acat, Bcat = np.zeros(lenA), np.zeros(lenB)
    for j in range(len(blocks)):
        ra, oa, rb, ob = b.h2_batch_factor_layout(P, j)
        Acat[oa:oa + ra * w["u"]] = A[j].ravel(order="F")
        Bcat[ob:ob + rb * w["u"]] = B[j].ravel(order="F")
    dA = torch.from_numpy(Acat).cuda()
    dB = torch.from_numpy(Bcat).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    b.h2_batch_set_timing(P, True)
    for _ in range(args.warmup):
        b.h2_batch_execute(ctx, P, dA.data_ptr(), dB.data_ptr(), w["eps"])
    b.h2_ctx_synchronize(ctx)

    nph = len(b.PHASES)
    phase_ms = [0.0] * nph
    step_ms = []
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sampler = ClockSampler(getattr(props, "pci_bus_id", None) if hasattr(props, "pci_bus_id") else None)
    sampler.start()
    time.sleep(0.5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for s in range(args.steps):
        flush.fill_(s)                       # write 512 MB (> L2) between steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.h2_batch_execute(ctx, P, dA.data_ptr(), dB.data_ptr(), w["eps"])
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for ph in range(nph):
            phase_ms[ph] += b.h2_batch_phase_stats(ctx, P, ph, flops=False)["ms"]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    b.h2_ctx_synchronize(ctx)
    total_ms = reduce_max(sum(step_ms), dist, device="cuda")
    ms_per_step = total_ms / args.steps
    value = world * len(blocks) / (ms_per_step / 1e3)
    stats = b.h2_batch_stats(ctx, P)
    phases = {}
    for ph, name in enumerate(b.PHASES):
        ps = b.h2_batch_phase_stats(ctx, P, ph)
        phases[name] = {"launches": ps["launches"], "ms": phase_ms[ph] / args.steps,
                        "gflop": ps["flops"] / 1e9,
                        "tflops": (ps["flops"] / (phase_ms[ph] / args.steps * 1e-3) / 1e12) if phase_ms[ph] > 0 else None}
    # dominant kernel on the critical path (the weights of the unchanged matrix
    # run beside it on side streams; the exact path only returns at once here)
    if args.mode == "exact":
        dom = "exact"
    else:
        dom = max((k for k in phases if k not in ("base_weights", "exact")), key=lambda k: phases[k]["ms"])
    ach = phases[dom]["tflops"]
    n_exact = int(b.h2_batch_paths(ctx, P, len(blocks)).sum())
    kern = PHASE_KERNELS[dom]
    traffic = None
    if kern in TRAFFIC_BYTES_PER_TASK and phases[dom]["launches"]:
        traffic = TRAFFIC_BYTES_PER_TASK[kern] * stats["cluster_tasks"] / phases[dom]["launches"]
    roof = {"bound": "alu", "kernel": kern, "achieved": ach, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s",
            "frac": (ach / FP64_PEAK_TFLOPS) if ach else None, "traffic": traffic, "traffic_unit": "bytes per launch",
            "peak_source": FP64_PEAK_SOURCE,
            "launch_ms": phases[dom]["ms"] / max(1, phases[dom]["launches"])}

    # every phase alone: the same executions with all phases on one stream,
    # so that a phase's events time its own kernels without the overlap of
    # the side streams (per-kernel roofline fractions)
    phases_serial = None
    if args.serial_steps > 0:
        b.h2_batch_set_timing(P, 2)
        acc = [0.0] * nph
        for s in range(2 + args.serial_steps):     # eager run, graph capture, replays
            flush.fill_(s)
            b.h2_batch_execute(ctx, P, dA.data_ptr(), dB.data_ptr(), w["eps"])
            b.h2_ctx_synchronize(ctx)
            if s >= 2:
                for ph in range(nph):
                    acc[ph] += b.h2_batch_phase_stats(ctx, P, ph, flops=False)["ms"]
        b.h2_batch_set_timing(P, True)
        phases_serial = {}
        for ph, name in enumerate(b.PHASES):
            ms = acc[ph] / args.serial_steps
            tf = phases[name]["gflop"] / ms if ms > 0 else None
            phases_serial[name] = {"ms": ms, "tflops": tf,
                                   "frac_fp64_peak": (tf / FP64_PEAK_TFLOPS) if tf else None}

    # the same batch with every update forced through the exact path (the
    # fallback for updates whose certificate fails: Householder folds and the
    # truncation SVD), to show what a truncating workload costs
    exact_mode = None
    if args.exact_steps > 0 and args.mode == "auto":
        b.h2_batch_set_mode(P, b.MODE_EXACT)
        ts = []
        for s in range(2 + args.exact_steps):
            flush.fill_(s)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.h2_batch_execute(ctx, P, dA.data_ptr(), dB.data_ptr(), w["eps"])
            e1.record(stream)
            e1.synchronize()
            if s >= 2:
                ts.append(e0.elapsed_time(e1))
        ex = b.h2_batch_phase_stats(ctx, P, b.PHASES.index("exact"))
        ms = sum(ts) / len(ts)
        gf = b.h2_batch_stats(ctx, P)["flops"] / 1e9
        exact_mode = {"ms_per_step": ms, "value": len(blocks) / (ms / 1e3), "unit": UNIT,
                      "gflop": gf, "tflops": gf / ms, "frac_fp64_peak": gf / ms / FP64_PEAK_TFLOPS,
                      "exact_phase_ms": ex["ms"]}
        b.h2_batch_set_mode(P, b.MODE_AUTO)

    # end to end through the C ABI from pinned host buffers (no phase events:
    # recorded inside the replayed graph they keep its copies from
    # overlapping the kernels)
    e2e = e2e_compact = None
    if args.e2e_steps > 0:
        b.h2_batch_set_timing(P, False)
        pA = torch.from_numpy(Acat).pin_memory()
        pB = torch.from_numpy(Bcat).pin_memory()
        res = torch.empty(b.h2_batch_result_size(P), dtype=torch.float64).pin_memory()
        for _ in range(3):     # eager run, graph capture, replay
            b.h2_batch_execute_host(ctx, P, pA.numpy(), pB.numpy(), w["eps"], res.numpy())
        if dist:
            dist.barrier()         # every rank copies at once, as a job would
        ts = []
        for _ in range(args.e2e_steps):
            flush.fill_(7)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.h2_batch_execute_host(ctx, P, pA.numpy(), pB.numpy(), w["eps"], res.numpy())
            ts.append(time.perf_counter() - t0)
        # whole job: the updates of all ranks over the slowest rank's time;
        # bytes of all ranks
        h2d, d2h = b.h2_batch_host_bytes(P)
        t_max = reduce_max(sum(ts) / len(ts), dist, device="cuda")
        e2e = {"value": world * len(blocks) / t_max, "unit": UNIT,
               "h2d_bytes_per_step": world * h2d, "d2h_bytes_per_step": world * d2h}
        # the compact result: couplings the updates keep ([S_b; 0], [S_b, 0]
        # of the unchanged matrix) are flagged instead of copied
        copied = np.zeros(stats["block_tasks"], np.int8)
        for _ in range(3):
            b.h2_batch_execute_host_compact(ctx, P, pA.numpy(), pB.numpy(), w["eps"], res.numpy(), copied)
        if dist:
            dist.barrier()
        ts = []
        for _ in range(args.e2e_steps):
            flush.fill_(7)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.h2_batch_execute_host_compact(ctx, P, pA.numpy(), pB.numpy(), w["eps"], res.numpy(), copied)
            ts.append(time.perf_counter() - t0)
        h2d, d2h = b.h2_batch_host_bytes(P)
        t_max = reduce_max(sum(ts) / len(ts), dist, device="cuda")
        e2e_compact = {"value": world * len(blocks) / t_max, "unit": UNIT,
                       "h2d_bytes_per_step": world * h2d, "d2h_bytes_per_step": world * d2h,
                       "kept_couplings": int(copied.sum()),
                       "result": "compact: kept couplings flagged, read from the unchanged matrix"}

    # H2 matrix times vectors on the same matrix (h2_matvec): one vector
    # (bound by HBM: every value of the matrix read once) and k = 16 vectors
    # (the products of the multiplication's Case 2; bound by the FP64 pipe)
    mv = None
    if args.matvec_steps > 0:
        mv = matvec_measure(b, ctx, Z, stream, flush, args.matvec_steps)

    lr = None
    cells_list = [int(x) for x in args.lr_cells.split(",") if x.strip()]
    if rank == 0 and world == 1 and cells_list:
        lr = lr_measure(b, ctx, cells_list, args.lr_reps, oracle_cells={32})
    chol = None
    chol_cells = [int(x) for x in args.chol_cells.split(",") if x.strip()]
    if rank == 0 and world == 1 and chol_cells:
        chol = lr_measure(b, ctx, chol_cells, 1, oracle_cells={32}, chol=True)
    lr_batch = chol_batch = None
    if rank == 0 and world == 1 and args.batch_problems > 0:
        lr_batch = lr_batch_measure(b, ctx, args.batch_problems, 24, 48)
        chol_batch = lr_batch_measure(b, ctx, args.batch_problems, 24, 48, chol=True)
    inv = None
    inv_cells = [int(x) for x in args.inv_cells.split(",") if x.strip()]
    if rank == 0 and world == 1 and inv_cells:
        inv = inverse_measure(b, ctx, inv_cells, oracle_cells={32})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        procs = args.cpu_procs or os.cpu_count() or 1
        op = OraclePool(procs)
        done, wall, start = 0, 0.0, 0
        while wall < args.cpu_seconds:
            chunk = 8 * procs
            wall += op.run(start, chunk)
            start += 97 * chunk          # spread the sample over the batch (its level mix)
            done += chunk
        op.close()
        cpu = {"value": done / wall, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": "%d updates of the 4096-update batch in groups of %d spread over the batch, on %d host "
                         "processes (one per core, one BLAS thread each), %.1f s" % (done, 8 * procs, procs, wall)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "mode": "isolated (each update reads the same base matrix)",
                       "path": args.mode,
                       "l2": "512 MB buffer written between timed steps",
                       "updates": len(blocks), "cluster_tasks": stats["cluster_tasks"],
                       "block_tasks": stats["block_tasks"], "exact_path_updates": n_exact,
                       "plan_s": plan_s},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "e2e_compact": e2e_compact,
            "gpu_launches": stats["launches"] * args.steps,
            "clocks": clocks, "phases": phases, "phases_serial": phases_serial, "exact_mode": exact_mode,
            "matvec": mv, "lr": lr, "chol": chol, "lr_batch": lr_batch, "chol_batch": chol_batch, "inverse": inv,
            "gflop_per_step": stats["flops"] / 1e9}
    if rank == 0:
        print(json.dumps(line))
    b.h2_batch_free(P)
    b.h2_matrix_free(Z)
    b.h2_ctx_destroy(ctx)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
