// Cluster tree and block tree (Section 2, Defs. "Cluster tree", "Block tree").
//
// Host C++, run once per matrix.  Every floating-point decision here
// (bisection midpoint, admissibility) is written without fused
// multiply-adds (the file is compiled with -ffp-contract=off) so that the
// trees are reproducible bit for bit on any host.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "h2_internal.h"

namespace h2 {
namespace {

struct CBuilder {
  const double* pts;
  int dim;
  int leaf_size;
  double pad;
  std::vector<int64_t>& idx;
  ClusterTree& ct;

  int32_t build(int64_t b, int64_t e, int32_t father, int32_t level) {
    const int32_t t = ct.count();
    std::vector<double> lo(dim), hi(dim);
    for (int a = 0; a < dim; ++a) {
      lo[a] = pts[idx[b] * dim + a];
      hi[a] = lo[a];
    }
    for (int64_t i = b + 1; i < e; ++i)
      for (int a = 0; a < dim; ++a) {
        const double x = pts[idx[i] * dim + a];
        lo[a] = std::min(lo[a], x);
        hi[a] = std::max(hi[a], x);
      }
    ct.off.push_back(b);
    ct.size.push_back(e - b);
    ct.father.push_back(father);
    ct.son0.push_back(-1);
    ct.son1.push_back(-1);
    ct.level.push_back(level);
    for (int a = 0; a < dim; ++a) {
      ct.lo.push_back(lo[a] - pad);
      ct.hi.push_back(hi[a] + pad);
    }
    if (e - b > leaf_size) {
      int axis = 0;
      for (int a = 1; a < dim; ++a)
        if (hi[a] - lo[a] > hi[axis] - lo[axis]) axis = a;
      const double mid = 0.5 * (lo[axis] + hi[axis]);
      auto it = std::stable_partition(idx.begin() + b, idx.begin() + e, [&](int64_t i) {
        return pts[i * dim + axis] < mid;
      });
      const int64_t m = it - idx.begin();
      if (m > b && m < e) {
        const int32_t t1 = build(b, m, t, level + 1);
        const int32_t t2 = build(m, e, t, level + 1);
        ct.son0[t] = t1;
        ct.son1[t] = t2;
      }
    }
    return t;
  }
};

double box_diam(const ClusterTree& ct, int32_t t) {
  double s = 0.0;
  for (int a = 0; a < ct.dim; ++a) {
    const double d = ct.hi[t * ct.dim + a] - ct.lo[t * ct.dim + a];
    const double d2 = d * d;
    s = s + d2;
  }
  return std::sqrt(s);
}

double box_dist(const ClusterTree& rt, int32_t t, const ClusterTree& ct, int32_t s) {
  double sum = 0.0;
  for (int a = 0; a < rt.dim; ++a) {
    const double g1 = ct.lo[s * ct.dim + a] - rt.hi[t * rt.dim + a];
    const double g2 = rt.lo[t * rt.dim + a] - ct.hi[s * ct.dim + a];
    const double g = std::max(0.0, std::max(g1, g2));
    const double g2sq = g * g;
    sum = sum + g2sq;
  }
  return std::sqrt(sum);
}

struct BBuilder {
  const ClusterTree& rt;
  const ClusterTree& ct;
  double eta;
  BlockTree& bt;

  int32_t build(int32_t t, int32_t s, int32_t father) {
    const int32_t b = bt.count();
    bt.row.push_back(t);
    bt.col.push_back(s);
    bt.father.push_back(father);
    for (int i = 0; i < 4; ++i) bt.son4.push_back(-1);
    bt.slot.push_back(-1);
    const double d = box_dist(rt, t, ct, s);
    const double diam = std::max(box_diam(rt, t), box_diam(ct, s));
    const double lim = eta * d;
    if (d > 0.0 && diam <= lim) {
      bt.kind.push_back(kAdm);
    } else if (rt.leaf(t) || ct.leaf(s)) {
      bt.kind.push_back(kNear);
    } else {
      bt.kind.push_back(kSub);
      const int32_t ts[2] = {rt.son0[t], rt.son1[t]};
      const int32_t ss[2] = {ct.son0[s], ct.son1[s]};
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          const int32_t c = build(ts[i], ss[j], b);
          bt.son4[4 * b + 2 * i + j] = c;
        }
    }
    return b;
  }
};

}  // namespace

void build_cluster_tree(const double* pts, int64_t n, int dim, int leaf_size, double pad,
                        ClusterTree& ct) {
  H2_REQUIRE(n > 0 && dim > 0 && leaf_size > 0, "build_cluster_tree: bad sizes");
  ct = ClusterTree();
  ct.n = n;
  ct.dim = dim;
  std::vector<int64_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  CBuilder cb{pts, dim, leaf_size, pad, idx, ct};
  cb.build(0, n, -1, 0);
  ct.perm = idx;
  const int32_t nc = ct.count();
  ct.subtree.assign(nc, 1);
  for (int32_t t = nc - 1; t >= 0; --t)
    if (!ct.leaf(t)) ct.subtree[t] += ct.subtree[ct.son0[t]] + ct.subtree[ct.son1[t]];
  ct.depth = 0;
  ct.max_leaf = 0;
  for (int32_t t = 0; t < nc; ++t) {
    ct.depth = std::max(ct.depth, ct.level[t]);
    if (ct.leaf(t)) ct.max_leaf = std::max<int>(ct.max_leaf, (int)ct.size[t]);
  }
}

void build_block_tree(const ClusterTree& rt, const ClusterTree& ct, double eta, BlockTree& bt) {
  bt = BlockTree();
  BBuilder bb{rt, ct, eta, bt};
  bb.build(0, 0, -1);
  const int32_t nb = bt.count();
  for (int32_t b = 0; b < nb; ++b) {
    if (bt.kind[b] == kAdm) {
      bt.slot[b] = (int32_t)bt.adm.size();
      bt.adm.push_back(b);
    } else if (bt.kind[b] == kNear) {
      bt.slot[b] = (int32_t)bt.near.size();
      bt.near.push_back(b);
    }
  }
  // CSR of admissible slots per row cluster and per column cluster, in block order
  bt.row_ptr.assign(rt.count() + 1, 0);
  bt.col_ptr.assign(ct.count() + 1, 0);
  for (int32_t b : bt.adm) {
    bt.row_ptr[bt.row[b] + 1]++;
    bt.col_ptr[bt.col[b] + 1]++;
  }
  for (int32_t t = 0; t < rt.count(); ++t) bt.row_ptr[t + 1] += bt.row_ptr[t];
  for (int32_t s = 0; s < ct.count(); ++s) bt.col_ptr[s + 1] += bt.col_ptr[s];
  bt.row_adm.assign(bt.adm.size(), 0);
  bt.col_adm.assign(bt.adm.size(), 0);
  std::vector<int32_t> rp(bt.row_ptr.begin(), bt.row_ptr.end() - 1);
  std::vector<int32_t> cp(bt.col_ptr.begin(), bt.col_ptr.end() - 1);
  for (int32_t b : bt.adm) {
    bt.row_adm[rp[bt.row[b]]++] = bt.slot[b];
    bt.col_adm[cp[bt.col[b]]++] = bt.slot[b];
  }
}

}  // namespace h2
