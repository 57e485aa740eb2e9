"""Command-line example: the H^2-LR preconditioner of a 2D finite-element
problem (Section 7's model problem) on one GPU.

    python -m paper_1402_5056_gb300.fem_lr --cells 64 --checker 4 --eps 1e-4

Builds the P1 stiffness matrix of -div(sigma grad u) = f on the unit square
(u = 0 on the boundary, sigma piecewise constant on a checker x checker
board with values 10^U(-2, 2)) as an H^2 matrix, factorises a copy into
H^2-LR (or, with --chol, the approximate Cholesky factor), runs
preconditioned CG to 1e-10 for a N(0, 1) right-hand side and estimates
||I - (LR)^-1 A||_2 (or ||I - (L L^*)^-1 A||_2) by the power iteration; prints one JSON line
with the sizes, the times (wall clock around each call, synchronised) and
the statistics of the factorisation.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main(argv=None) -> dict:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--cells", type=int, default=32, help="grid cells per side")
    ap.add_argument("--checker", type=int, default=4, help="checkerboard of sigma, per side")
    ap.add_argument("--eps", type=float, default=1e-4, help="block-relative truncation accuracy")
    ap.add_argument("--leaf", type=int, default=32)
    ap.add_argument("--eta", type=float, default=2.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tol", type=float, default=1e-10, help="relative residual of CG")
    ap.add_argument("--max-rank", type=int, default=0,
                    help="rank cap of every local update (0: none, the paper's method)")
    ap.add_argument("--chol", action="store_true",
                    help="approximate Cholesky factorisation instead of the LR (Section 7's preconditioner)")
    args = ap.parse_args(argv)

    import torch
    from . import binding as b

    rng = np.random.default_rng(args.seed)
    sigma = 10.0 ** rng.uniform(-2.0, 2.0, args.checker * args.checker)
    torch.cuda.set_device(0)
    ctx = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    opt = b.options(eps=args.eps, eta=args.eta, leaf_size=args.leaf, max_rank=args.max_rank)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        A = b.h2_build_fem(ctx, 2, args.cells, args.checker, sigma, opt)
        F = b.h2_matrix_clone(ctx, A)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        info = b.h2_chol_factor(ctx, F, opt) if args.chol else b.h2_lr_factor(ctx, F, opt)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        n = (args.cells - 1) ** 2
        rhs = rng.standard_normal(n)[b.h2_tree_permutation(A)]
        bd = torch.from_numpy(np.ascontiguousarray(rhs)).cuda()
        xd = torch.zeros(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        pcg = b.h2_pcg_chol if args.chol else b.h2_pcg
        it, rr = pcg(ctx, A, F, bd.data_ptr(), xd.data_ptr(), args.tol, 1000)
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        v0 = torch.from_numpy(rng.standard_normal(n)).cuda()
        err = (b.h2_chol_error if args.chol else b.h2_lr_error)(ctx, A, F, v0.data_ptr(), 20)
        out = {"n": n, "cells": args.cells, "checker": args.checker, "eps": args.eps, "max_rank": args.max_rank,
               "factorisation": "cholesky" if args.chol else "lr",
               "build_s": t1 - t0, "factor_s": t2 - t1, "cg_iterations": it, "cg_relres": rr,
               "cg_s": t4 - t3, "err_power": err, "factor": info}
        b.h2_matrix_free(F)
        b.h2_matrix_free(A)
    finally:
        b.h2_ctx_destroy(ctx)
    print(json.dumps(out, default=float))
    return out


if __name__ == "__main__":
    main()
