"""Seeded synthetic inputs for the H^2 local low-rank update.

This module is shared by the tests, the benchmark and the CPU oracle.  It
draws random numbers and lays them out in the canonical orders the library
and the oracle both accept; it holds none of the method's arithmetic and
builds no tree.  Callers pass in the structural counts (leaf sizes, sibling
pairs, number of admissible blocks, ...) that their own tree builder
produced.

Canonical host layouts (all column-major, float64):

* leaf bases  -- concatenation over leaf clusters in cluster order of the
  m_t x k_t leaf matrices V_t (Section 2, Def. "Cluster basis");
* transfers   -- concatenation over non-root clusters in cluster order of
  the k_t x k_{t+} transfer matrices E_t (Eq. (nested));
* couplings   -- concatenation over admissible blocks in block order of the
  k_t x l_s coupling matrices S_b (Eq. (vsw));
* nearfield   -- concatenation over inadmissible leaves in block order of
  the dense #t x #s blocks.

Random-stream recipe for the isolated-update workload (n = 256 x 256 grid
points, k = 16, 4096 rank-8 updates, eps = 1e-8): a ``numpy.random.
SeedSequence(seed)`` is spawned into six child streams in the order
[sigma, rhs, bases, couplings, block choice, A/B]; the first two are unused
by this workload and reserved for the FEM problems.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1402505600

STREAM_NAMES = ("sigma", "rhs", "bases", "couplings", "blocks", "ab")


def streams(seed: int) -> dict:
    """Six independent PCG64 generators spawned from ``seed``."""
    children = np.random.SeedSequence(seed).spawn(len(STREAM_NAMES))
    return {name: np.random.Generator(np.random.PCG64(ss))
            for name, ss in zip(STREAM_NAMES, children)}


def grid_points_2d(N: int) -> np.ndarray:
    """Points ((i+0.5)/N, (j+0.5)/N), numbered i + N*j (x fastest); (N*N, 2)."""
    i = np.arange(N, dtype=np.float64)
    x = np.tile((i + 0.5) / N, N)
    y = np.repeat((i + 0.5) / N, N)
    return np.ascontiguousarray(np.stack([x, y], axis=1))


def _orthonormal_columns(g: np.ndarray) -> np.ndarray:
    """Orthonormal Q of a Gaussian draw, sign-fixed so that diag(R) >= 0."""
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


def nested_orthonormal_bases(rng: np.random.Generator, leaf_sizes, sibling_pairs,
                             n_clusters: int, k: int):
    """Random orthonormal nested cluster basis of constant rank ``k``.

    leaf_sizes    -- list of (cluster id, m_t) for every leaf, in cluster order
    sibling_pairs -- list of (son1 id, son2 id) for every inner cluster, in
                     cluster order of the father
    Returns (ranks[n_clusters], leaf_data, transfer_data) in the canonical
    layouts.  Each leaf matrix is the orthonormalised Gaussian m_t x k draw;
    each sibling pair's transfers are the two halves of one orthonormalised
    Gaussian 2k x k draw, which keeps every V_t orthonormal.  Draw order:
    all leaves in cluster order, then all sibling pairs in cluster order.
    """
    ranks = np.full(n_clusters, k, dtype=np.int32)
    leaves = []
    for _, m in leaf_sizes:
        if m < k:
            raise ValueError("leaf smaller than the rank")
        leaves.append(_orthonormal_columns(rng.standard_normal((m, k))))
    transfers = {}
    for s1, s2 in sibling_pairs:
        q = _orthonormal_columns(rng.standard_normal((2 * k, k)))
        transfers[s1] = q[:k]
        transfers[s2] = q[k:]
    leaf_data = np.concatenate([v.ravel(order="F") for v in leaves]) if leaves else np.zeros(0)
    nonroot = sorted(transfers)
    transfer_data = (np.concatenate([transfers[c].ravel(order="F") for c in nonroot])
                     if nonroot else np.zeros(0))
    return ranks, leaf_data, transfer_data


def nested_orthonormal_bases_general(rng: np.random.Generator, sizes, sons, k: int):
    """Random orthonormal nested cluster basis with ranks capped by the sizes.

    sizes -- #t for every cluster in cluster order
    sons  -- (son1, son2) or None for every cluster in cluster order
    Ranks: r_t = min(k, #t) for leaves, min(k, r_son1 + r_son2) above.  Draws
    as in ``nested_orthonormal_bases`` (leaves in cluster order, then one
    orthonormalised Gaussian (r_son1 + r_son2) x r_t matrix per inner cluster
    in cluster order, split into the sons' transfers), so both agree when
    every leaf has at least k indices.
    """
    n = len(sizes)
    ranks = np.zeros(n, dtype=np.int32)
    for t in reversed(range(n)):
        ranks[t] = min(k, sizes[t]) if sons[t] is None else min(k, ranks[sons[t][0]] + ranks[sons[t][1]])
    leaves = []
    for t in range(n):
        if sons[t] is None:
            leaves.append(_orthonormal_columns(rng.standard_normal((sizes[t], ranks[t]))))
    transfers = {}
    for t in range(n):
        if sons[t] is not None:
            s1, s2 = sons[t]
            q = _orthonormal_columns(rng.standard_normal((ranks[s1] + ranks[s2], ranks[t])))
            transfers[s1] = q[:ranks[s1]]
            transfers[s2] = q[ranks[s1]:]
    leaf_data = np.concatenate([v.ravel(order="F") for v in leaves]) if leaves else np.zeros(0)
    nonroot = sorted(transfers)
    transfer_data = (np.concatenate([transfers[c].ravel(order="F") for c in nonroot])
                     if nonroot else np.zeros(0))
    return ranks, leaf_data, transfer_data


def gaussian_couplings(rng: np.random.Generator, n_adm: int, k: int, scale: float) -> np.ndarray:
    """n_adm coupling matrices k x k with entries N(0,1)*scale, canonical layout."""
    s = rng.standard_normal((n_adm, k, k)) * scale
    # canonical layout is column-major per block
    return np.ascontiguousarray(np.transpose(s, (0, 2, 1))).ravel()


def gaussian_nearfield(rng: np.random.Generator, shapes, scale: float) -> np.ndarray:
    """Dense nearfield blocks (rows x cols per entry of ``shapes``), N(0,1)*scale."""
    parts = [rng.standard_normal(r * c) * scale for r, c in shapes]
    return np.concatenate(parts) if parts else np.zeros(0)


def gaussian_blocks(rng: np.random.Generator, shapes, scale: float) -> np.ndarray:
    """Dense blocks (rows x cols per entry of ``shapes``), N(0,1)*scale,
    concatenated column-major (coupling matrices of varying ranks)."""
    return gaussian_nearfield(rng, shapes, scale)


def choose_blocks(rng: np.random.Generator, candidates, count: int) -> np.ndarray:
    """``count`` block ids drawn uniformly with replacement from ``candidates``."""
    cand = np.asarray(candidates, dtype=np.int64)
    return cand[rng.integers(0, len(cand), size=count)]


def update_factors(rng: np.random.Generator, row_sizes, col_sizes, u: int):
    """Factors A_j (#t0 x u) and B_j (#s0 x u), N(0,1), column-major, per update.

    Draw order: A_0, B_0, A_1, B_1, ...
    Returns two lists of Fortran-ordered arrays.
    """
    A, B = [], []
    for mt, ms in zip(row_sizes, col_sizes):
        A.append(np.asfortranarray(rng.standard_normal((mt, u))))
        B.append(np.asfortranarray(rng.standard_normal((ms, u))))
    return A, B


# ------------------------------------------------------------ FEM problems
# Recipe of the finite-element problems (Section 7's model problem with a
# variable coefficient): seed = SEED_BASE + config index, the streams of
# ``streams(seed)``; sigma = 10^U(-2, 2) on an M^dim checkerboard (x
# fastest) from the "sigma" stream, right-hand sides N(0, 1) from the "rhs"
# stream in the unknowns' original order (interior nodes, x fastest).

def checker_sigma(rng: np.random.Generator, M: int, dim: int, decades=(-2.0, 2.0)) -> np.ndarray:
    """Checkerboard coefficients 10^U(lo, hi), M^dim values, x fastest."""
    return 10.0 ** rng.uniform(decades[0], decades[1], M ** dim)


def fem_rhs(rng: np.random.Generator, n: int, nrhs: int = 1) -> np.ndarray:
    """N(0, 1) right-hand sides, n x nrhs (column-major order of draws)."""
    return rng.standard_normal((nrhs, n)).T.copy()
