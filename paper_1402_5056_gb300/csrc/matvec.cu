// H^2-matrix times a block of vectors (Section 2: Eq. (vsw) for the
// admissible leaves, dense inadmissible leaves, nested bases Eq. (nested)),
// the product the multiplication of Section 3 applies where a factor block
// is a leaf (Section 6, Case 2: X|_{t x s} V_s by k such products).
//
//   forward transformation, bottom-up over the column tree:
//     xh_s = W_s^* X|_s (leaf), xh_s = sum over sons E_{s'}^* xh_{s'};
//   coupling, every row cluster at once: yh_t = sum over row(t) S_b xh_s;
//   backward transformation, top-down over the row tree:
//     yh_{t'} += E_{t'} yh_t for the sons t' of t;
//   leaves of the row tree: Y|_t = alpha (V_t yh_t + the rows of t of every
//     nearfield block N_b X|_s whose row cluster contains t) + beta Y|_t
//     (a nearfield block pairs a leaf with a cluster that may be larger).
//
// One warp per cluster; lanes take the entries (i, r) of the k x nrhs
// results (entry e = i + k r) or, at the leaves, the rows.  Every value of
// the matrix is read once per call; the per-level launches follow the tree.
#include "matvec.h"

namespace h2 {
namespace {

constexpr int kMvWarps = 4;

__device__ __forceinline__ bool is_leaf(const int32_t* subtree, int c) { return subtree[c] == 1; }

// xh_c of one column cluster (one warp)
__device__ __forceinline__ void forward_cluster(const MatvecArgs& a, int c, int lane) {
  const int kc = a.rank[1][c];
  const int kcap = a.kcap;
  double* out = a.xh + (size_t)c * kcap * a.nrhs;
  const int ne = kc * a.nrhs;
  if (is_leaf(a.subtree[1], c)) {
    const int m = a.size[1][c];
    const double* Wl = a.leaf[1] + a.leaf_off[1][c];
    const double* X = a.X + a.off[1][c];
    for (int e = lane; e < ne; e += 32) {
      const int i = e % kc, r = e / kc;
      double v = 0.0;
      for (int p = 0; p < m; ++p) v = fma(Wl[p + (size_t)i * m], X[p + r * a.ldx], v);
      out[i + r * kcap] = v;
    }
  } else {
    const int s0 = c + 1;
    const int s1 = c + 1 + a.subtree[1][c + 1];
    const int k0 = a.rank[1][s0], k1 = a.rank[1][s1];
    const double* E0 = a.transfer[1] + (size_t)s0 * kcap * kcap;
    const double* E1 = a.transfer[1] + (size_t)s1 * kcap * kcap;
    const double* x0 = a.xh + (size_t)s0 * kcap * a.nrhs;
    const double* x1 = a.xh + (size_t)s1 * kcap * a.nrhs;
    for (int e = lane; e < ne; e += 32) {
      const int i = e % kc, r = e / kc;
      double v = 0.0;
      for (int q = 0; q < k0; ++q) v = fma(E0[q + i * kcap], x0[q + r * kcap], v);
      for (int q = 0; q < k1; ++q) v = fma(E1[q + i * kcap], x1[q + r * kcap], v);
      out[i + r * kcap] = v;
    }
  }
}

__global__ void k_mv_forward(MatvecArgs a, const int32_t* __restrict__ list, int n) {
  const int w = blockIdx.x * kMvWarps + (threadIdx.x >> 5);
  if (w >= n) return;
  forward_cluster(a, list[w], threadIdx.x & 31);
}

// Coupling: lane = (row i of yh_t, group g); the groups split the
// right-hand sides (RB at a time, sharing each S_b load) or, with fewer
// right-hand sides than groups, the blocks of row(t) (partial sums added by
// shuffles in a fixed order).
template <int RB>
__global__ void k_mv_coupling(MatvecArgs a) {
  const int t = blockIdx.x * kMvWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= a.n_clusters[0]) return;
  const int kt = a.rank[0][t];
  if (kt == 0) return;
  const int kcap = a.kcap;
  const int groups = kt <= 32 ? 32 / kt : 1;
  const int i = lane % kt, g = lane / kt;
  const bool in = g < groups;
  double* out = a.yh + (size_t)t * kcap * a.nrhs;
  const int e0 = a.row_ptr[t], e1 = a.row_ptr[t + 1];
  const int rsteps = (a.nrhs + RB - 1) / RB;
  const bool split_blocks = rsteps < groups;   // few right-hand sides: the groups share the blocks
  for (int r0 = (split_blocks ? 0 : g) * RB; r0 < a.nrhs; r0 += (split_blocks ? 1 : groups) * RB) {
    double acc[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) acc[j] = 0.0;
    if (in)
      for (int x = e0 + (split_blocks ? g : 0); x < e1; x += split_blocks ? groups : 1) {
        const int slot = a.row_adm[x];
        const int s = a.blk_col[slot];
        const int ls = a.rank[1][s];
        const double* S = a.S + (size_t)slot * kcap * kcap + i;
        const double* xs = a.xh + (size_t)s * kcap * a.nrhs + (size_t)r0 * kcap;
        // unrolled: the loads of several columns in flight (the sums keep
        // their order)
#pragma unroll 8
        for (int q = 0; q < ls; ++q) {
          const double sv = S[q * kcap];
#pragma unroll
          for (int j = 0; j < RB; ++j)
            if (r0 + j < a.nrhs) acc[j] = fma(sv, xs[q + j * kcap], acc[j]);
        }
      }
    if (split_blocks) {
      // add the groups' partial sums: group 0 collects g = 1, 2, ... in order
#pragma unroll
      for (int j = 0; j < RB; ++j)
        for (int h = 1; h < groups; ++h) {
          const double o = __shfl_sync(0xffffffffu, acc[j], (lane + h * kt) & 31);
          if (g == 0) acc[j] += o;
        }
      if (g != 0 || !in) continue;
    } else if (!in) {
      continue;
    }
#pragma unroll
    for (int j = 0; j < RB; ++j)
      if (r0 + j < a.nrhs) out[i + (r0 + j) * kcap] = acc[j];
  }
}

// yh_c += E_c yh_{c+} for one row cluster (one warp)
__device__ __forceinline__ void backward_cluster(const MatvecArgs& a, int c, int lane) {
  const int f = a.father[0][c];
  if (f < 0) return;
  const int kc = a.rank[0][c], kf = a.rank[0][f];
  const int kcap = a.kcap;
  const double* E = a.transfer[0] + (size_t)c * kcap * kcap;   // kc x kf
  const double* yf = a.yh + (size_t)f * kcap * a.nrhs;
  double* yc = a.yh + (size_t)c * kcap * a.nrhs;
  const int ne = kc * a.nrhs;
  for (int e = lane; e < ne; e += 32) {
    const int i = e % kc, r = e / kc;
    double v = yc[i + r * kcap];
    for (int q = 0; q < kf; ++q) v = fma(E[i + q * kcap], yf[q + r * kcap], v);
    yc[i + r * kcap] = v;
  }
}

__global__ void k_mv_backward(MatvecArgs a, const int32_t* __restrict__ list, int n) {
  const int w = blockIdx.x * kMvWarps + (threadIdx.x >> 5);
  if (w >= n) return;
  backward_cluster(a, list[w], threadIdx.x & 31);
}

// The levels of a tree that hold few clusters, in one block: level after
// level (the order of `lev`), a barrier between levels.  A launch per level
// would cost more than their work.
constexpr int kTopWarps = 32;
constexpr int kTopMax = 2 * kTopWarps;   // clusters x right-hand sides per level handled this way
struct TopLevels {
  int n;             // levels
  int first[17];     // offsets into the level list, n + 1 entries, in processing order
  int count[16];
};

template <bool kForward>
__global__ void __launch_bounds__(32 * kTopWarps) k_mv_top(MatvecArgs a, const int32_t* __restrict__ list,
                                                             TopLevels t) {
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  for (int l = 0; l < t.n; ++l) {
    const int32_t* lv = list + t.first[l];
    const int n = t.count[l];
    for (int x = w; x < n; x += kTopWarps) {
      if constexpr (kForward)
        forward_cluster(a, lv[x], lane);
      else
        backward_cluster(a, lv[x], lane);
    }
    __syncthreads();
  }
}

// Leaves: lane = row; RB right-hand sides at a time share every load of the
// leaf basis and of the nearfield blocks.
template <int RB>
__global__ void k_mv_leaves(MatvecArgs a) {
  const int w = blockIdx.x * kMvWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= a.n_leaves) return;
  const int t = a.leaves[w];
  const int m = a.size[0][t];
  const int kt = a.rank[0][t];
  const int kcap = a.kcap;
  const double* Vl = a.leaf[0] + a.leaf_off[0][t];
  const double* yt = a.yh + (size_t)t * kcap * a.nrhs;
  for (int r0 = 0; r0 < a.nrhs; r0 += RB)
    for (int p = lane; p < m; p += 32) {
      double acc[RB];
#pragma unroll
      for (int j = 0; j < RB; ++j) acc[j] = 0.0;
#pragma unroll 8
      for (int i = 0; i < kt; ++i) {
        const double v = Vl[p + (size_t)i * m];
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if (r0 + j < a.nrhs) acc[j] = fma(v, yt[i + (r0 + j) * kcap], acc[j]);
      }
      // nearfield blocks whose row cluster contains t (the leaf itself, or
      // an ancestor paired with a leaf of the column tree): their rows of t
      for (int c = t; c >= 0; c = a.father[0][c]) {
        const int mc = a.size[0][c];
        const int64_t row = a.off[0][t] - a.off[0][c] + p;
        for (int x = a.near_ptr[c]; x < a.near_ptr[c + 1]; ++x) {
          const int s = a.near_col[x];
          const int ms = a.size[1][s];
          const double* Nb = a.N + a.near_off[x] + row;
          const double* X = a.X + a.off[1][s] + (size_t)r0 * a.ldx;
#pragma unroll 8
          for (int q = 0; q < ms; ++q) {
            const double nv = Nb[(size_t)q * mc];
#pragma unroll
            for (int j = 0; j < RB; ++j)
              if (r0 + j < a.nrhs) acc[j] = fma(nv, X[q + j * a.ldx], acc[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < RB; ++j)
        if (r0 + j < a.nrhs) {
          double* y = a.Y + a.off[0][t] + p + (size_t)(r0 + j) * a.ldy;
          *y = a.beta == 0.0 ? a.alpha * acc[j] : fma(a.beta, *y, a.alpha * acc[j]);
        }
    }
}

int blocks_of(int n) { return (n + kMvWarps - 1) / kMvWarps; }

}  // namespace

int launch_matvec(const MatvecArgs& a, cudaStream_t st) {
  int launches = 0;
  // levels [0, top) of a tree whose work is small (clusters x right-hand
  // sides at most kTopMax, at most 16 levels) go into one block
  const auto top_of = [&](int sd) {
    int top = 0;
    while (top < a.levels[sd] && top < 16 &&
           (int64_t)(a.lvl_ptr[sd][top + 1] - a.lvl_ptr[sd][top]) * a.nrhs <= kTopMax)
      ++top;
    return top;
  };
  // forward transformation: deepest level first, the upper levels in one block
  const int top1 = top_of(1);
  for (int l = a.levels[1] - 1; l >= top1; --l) {
    const int n = a.lvl_ptr[1][l + 1] - a.lvl_ptr[1][l];
    if (n <= 0) continue;
    k_mv_forward<<<blocks_of(n), 32 * kMvWarps, 0, st>>>(a, a.lvl_list[1] + a.lvl_ptr[1][l], n);
    ++launches;
  }
  if (top1 > 0) {
    TopLevels t{};
    t.n = top1;
    for (int i = 0; i < top1; ++i) {   // levels top1 - 1, ..., 0
      const int l = top1 - 1 - i;
      t.first[i] = a.lvl_ptr[1][l];
      t.count[i] = a.lvl_ptr[1][l + 1] - a.lvl_ptr[1][l];
    }
    k_mv_top<true><<<1, 32 * kTopWarps, 0, st>>>(a, a.lvl_list[1], t);
    ++launches;
  }
  if (a.n_clusters[0] > 0) {
    if (a.nrhs >= 8)
      k_mv_coupling<8><<<blocks_of(a.n_clusters[0]), 32 * kMvWarps, 0, st>>>(a);
    else
      k_mv_coupling<1><<<blocks_of(a.n_clusters[0]), 32 * kMvWarps, 0, st>>>(a);
    ++launches;
  }
  // backward transformation: level 1 down (the root has no father), the
  // upper levels in one block
  const int top0 = top_of(0);
  if (top0 > 1) {
    TopLevels t{};
    t.n = top0 - 1;
    for (int i = 0; i < top0 - 1; ++i) {   // levels 1, ..., top0 - 1
      t.first[i] = a.lvl_ptr[0][i + 1];
      t.count[i] = a.lvl_ptr[0][i + 2] - a.lvl_ptr[0][i + 1];
    }
    k_mv_top<false><<<1, 32 * kTopWarps, 0, st>>>(a, a.lvl_list[0], t);
    ++launches;
  }
  for (int l = top0 > 1 ? top0 : 1; l < a.levels[0]; ++l) {
    const int n = a.lvl_ptr[0][l + 1] - a.lvl_ptr[0][l];
    if (n <= 0) continue;
    k_mv_backward<<<blocks_of(n), 32 * kMvWarps, 0, st>>>(a, a.lvl_list[0] + a.lvl_ptr[0][l], n);
    ++launches;
  }
  if (a.n_leaves > 0) {
    if (a.nrhs >= 8)
      k_mv_leaves<8><<<blocks_of(a.n_leaves), 32 * kMvWarps, 0, st>>>(a);
    else if (a.nrhs >= 2)
      k_mv_leaves<2><<<blocks_of(a.n_leaves), 32 * kMvWarps, 0, st>>>(a);
    else
      k_mv_leaves<1><<<blocks_of(a.n_leaves), 32 * kMvWarps, 0, st>>>(a);
    ++launches;
  }
  return launches;
}

}  // namespace h2
