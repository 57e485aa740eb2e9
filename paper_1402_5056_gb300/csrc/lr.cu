// H^2-LR factorisation of a finite-element stiffness matrix on one GPU
// (Section 3, with the complexity structure of Section 6), its block
// forward/backward substitutions, and the preconditioned conjugate
// gradients of the experiments (Section 7).
//
// The host walks the recursion of Section 3 on ONE H^2 matrix that holds A
// on entry and L (strictly lower part, unit diagonal implied) and R (upper
// part with the diagonal) on exit; every arithmetic step runs on the device:
// leaf LU and triangular solves, products of one block with dense columns
// (forward/backward transformations through the nested bases), small dense
// products, the truncation of factor pairs, and the local low-rank updates
// of Section 5 (the batched update kernels of this library).
//
// Readings of what the paper leaves open (the same as the CPU oracle's):
//  1. the terms of one product Z|_z += alpha X|_x Y|_y are all computed
//     from the matrix as it is when the product starts, then added in the
//     order the recursion produces them; the terms for one target block
//     that is not an inadmissible leaf are concatenated into one factor
//     pair and added by one update where the block's first term stands;
//  2. a target z that is an admissible leaf while X and Y are subdivided
//     receives temporaries (t', r') for t' in sons(t), r' in sons(r): the
//     terms below each are stacked into one factor pair, extended by zeros
//     to z, truncated (Householder QR of both factors, SVD of the core) to
//     the smallest rank r with sum_{i>r} sigma_i^2 <= (eps/2)^2 sum
//     sigma_i^2, and added by one local update;
//  3. a dense term P = alpha X Y for a target that is not an inadmissible
//     leaf becomes the factor pair through its smallest dimension:
//     (alpha X, Y^*) when the inner cluster is the smallest, else (I, P^*)
//     when #t <= #r, else (P, I);
//  4. forward substitution on an admissible leaf Y = V_t S W_s^*: S is set
//     to zero and (L^-1 V_t S) W_s^* added by a local update; X R = Y
//     likewise with V_t (R^-* W_s S^*)^*;
//  5. an update of rank u is applied in consecutive column groups of at
//     most 32 - (largest rank among the clusters of both subtrees) columns
//     (at least 1, at most 31), each group one local update (the update
//     kernels hold k_t + u <= 32 columns and u <= 31).
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <thread>
#include <vector>

#include "h2_internal.h"
#include "lr.h"

using namespace h2;

namespace {

template <typename F>
h2_status lr_guard(h2_ctx* ctx, F&& f) {
  try {
    f();
    return H2_OK;
  } catch (const Error& e) {
    if (ctx) ctx->last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->last_error = "host allocation failed";
    return H2_ENOMEM;
  } catch (const std::exception& e) {
    if (ctx) ctx->last_error = e.what();
    return H2_EINTERNAL;
  }
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Timer {
  double& acc;
  double t0;
  explicit Timer(double& a) : acc(a), t0(now_s()) {}
  ~Timer() { acc += now_s() - t0; }
};

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) H2_CUDA(cudaSetDevice(dev));
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// stream-ordered device array of doubles
struct DArr {
  double* p = nullptr;
  cudaStream_t st = nullptr;
  DArr() = default;
  DArr(size_t n, cudaStream_t s) : st(s) {
    p = static_cast<double*>(device_alloc_async(n * sizeof(double), s));
  }
  DArr(const DArr&) = delete;
  DArr& operator=(const DArr&) = delete;
  DArr(DArr&& o) noexcept : p(o.p), st(o.st) { o.p = nullptr; }
  DArr& operator=(DArr&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      st = o.st;
      o.p = nullptr;
    }
    return *this;
  }
  void release() {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
  }
  ~DArr() { release(); }
};

void zero(double* p, size_t n, cudaStream_t st) {
  if (n) H2_CUDA(cudaMemsetAsync(p, 0, n * sizeof(double), st));
}

// ------------------------------------------------------------- the driver
struct Lr {
  h2_ctx* ctx = nullptr;
  h2_matrix* Z = nullptr;
  const h2_matrix* X = nullptr;   // factors of the current product (nullptr: Z itself)
  const h2_matrix* Y = nullptr;
  double eps = 0.0;
  int max_rank = 0;               // rank cap of every local update (0: none)
  bool yt = false;       // the product's second factor is read transposed (Cholesky)
  bool lower = false;    // a diagonal target gets only its son blocks on or below the diagonal
  cudaStream_t st = nullptr;
  int64_t updates = 0;
  int64_t products = 0;
  // wall time (s) by activity: local updates, product terms, temporaries,
  // dense solves through diagonal blocks, leaf LU
  double t_update = 0, t_terms = 0, t_temps = 0, t_solves = 0, t_lu = 0;
  double t_temp_wait = 0;   // of t_temps: waiting for the rank of the truncation
  int64_t n_temps = 0, temp_cols = 0;
  // block-product workspace: per cluster kcap x m slots
  double* xh = nullptr;
  double* yh = nullptr;
  size_t wcap = 0;
  int32_t* dlist = nullptr;
  size_t lcap = 0;
  int64_t* dnear_off = nullptr;   // per nearfield slot, offset in Z->d_N
  UpdateEngine* eng = nullptr;    // persistent workspace of the local updates
  ~Lr() {
    engine_delete(eng);
    if (dnear_off) cudaFree(dnear_off);
    if (xh) cudaFree(xh);
    if (yh) cudaFree(yh);
    if (dlist) cudaFree(dlist);
  }
};

// per-slot offsets of the nearfield blocks on the device (once per driver)
const int64_t* near_offsets(Lr& L) {
  if (!L.dnear_off && !L.Z->near_off.empty()) {
    const size_t n = L.Z->near_off.size();
    L.dnear_off = static_cast<int64_t*>(device_alloc(n * sizeof(int64_t)));
    H2_CUDA(cudaMemcpy(L.dnear_off, L.Z->near_off.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice));
  }
  return L.dnear_off;
}

void ensure_work(Lr& L, int m, int kcap) {
  const size_t need = (size_t)L.Z->rows.count() * kcap * std::max(m, 1);
  if (need <= L.wcap) return;
  H2_CUDA(cudaStreamSynchronize(L.st));
  if (L.xh) cudaFree(L.xh);
  if (L.yh) cudaFree(L.yh);
  L.xh = L.yh = nullptr;
  L.wcap = 0;
  L.xh = static_cast<double*>(device_alloc(need * sizeof(double)));
  L.yh = static_cast<double*>(device_alloc(need * sizeof(double)));
  L.wcap = need;
}

int32_t* upload_list(Lr& L, const std::vector<int32_t>& v) {
  if (v.size() > L.lcap) {
    H2_CUDA(cudaStreamSynchronize(L.st));
    if (L.dlist) cudaFree(L.dlist);
    L.dlist = nullptr;
    const size_t cap = std::max<size_t>(v.size(), 2 * L.lcap);
    L.lcap = 0;
    L.dlist = static_cast<int32_t*>(device_alloc(cap * sizeof(int32_t)));
    L.lcap = cap;
  }
  // pageable source: the copy is staged before the call returns, and the
  // previous user of the device list ran earlier on the same stream
  if (!v.empty()) H2_CUDA(cudaMemcpyAsync(L.dlist, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice, L.st));
  return L.dlist;
}

BasisView view(const h2_matrix* Z, int side) {
  const DeviceBasis& b = side == 0 ? Z->V : Z->W;
  BasisView v;
  v.off = side == 0 ? Z->d_row_off : Z->d_col_off;
  v.size = side == 0 ? Z->d_row_size : Z->d_col_size;
  v.rank = b.d_rank;
  v.subtree = side == 0 ? Z->d_subtree_r : Z->d_subtree_c;
  v.leaf = b.d_leaf;
  v.leaf_off = b.d_leaf_off;
  v.transfer = b.d_transfer;
  return v;
}

const ClusterTree& tree(const h2_matrix* Z, int side) { return side == 0 ? Z->rows : Z->cols; }

// clusters of T_c grouped by level (runs), deepest first or top-down
void level_runs(const ClusterTree& ct, int32_t c, bool bottom_up, bool skip_root, std::vector<int32_t>& list,
                std::vector<int32_t>& fathers, std::vector<std::pair<int, int>>& runs) {
  const int32_t end = c + ct.subtree[c];
  int lmin = ct.level[c], lmax = lmin;
  for (int32_t x = c; x < end; ++x) lmax = std::max(lmax, (int)ct.level[x]);
  for (int step = 0; step <= lmax - lmin; ++step) {
    const int lv = bottom_up ? lmax - step : lmin + step;
    if (skip_root && lv == lmin) continue;
    const int start = (int)list.size();
    for (int32_t x = c; x < end; ++x)
      if (ct.level[x] == lv) {
        list.push_back(x);
        fathers.push_back(ct.father[x]);
      }
    if ((int)list.size() > start) runs.push_back({start, (int)list.size() - start});
  }
}

// Y (Y-side rows of b x m) += alpha op(Z|_b) X (X-side rows x m)
void block_prod(Lr& L, const h2_matrix* Zb, int32_t b, int trans, double alpha, const double* X, int64_t ldx,
                double* Y, int64_t ldy, int m) {
  if (m <= 0) return;
  const h2_matrix* Z = Zb;
  const BlockTree& bt = Z->blocks;
  const int in_side = trans ? 0 : 1, out_side = trans ? 1 : 0;
  const ClusterTree& tin = tree(Z, in_side);
  const ClusterTree& tout = tree(Z, out_side);
  const int32_t cin = trans ? bt.row[b] : bt.col[b];
  const int32_t cout = trans ? bt.col[b] : bt.row[b];
  std::vector<int32_t> adm, near;
  std::vector<int32_t> stack{b};
  while (!stack.empty()) {
    const int32_t x = stack.back();
    stack.pop_back();
    if (bt.kind[x] == kAdm) adm.push_back(x);
    else if (bt.kind[x] == kNear) near.push_back(x);
    else
      for (int k = 3; k >= 0; --k)
        if (bt.son4[4 * x + k] >= 0) stack.push_back(bt.son4[4 * x + k]);
  }
  if (adm.empty() && near.empty()) return;
  ensure_work(L, m, Z->kcap);
  BlockProd a{};
  a.in = view(Z, in_side);
  a.out = view(Z, out_side);
  a.kcap = Z->kcap;
  a.trans = trans;
  a.in_off0 = tin.off[cin];
  a.out_off0 = tout.off[cout];
  a.S = Z->d_S;
  a.N = Z->d_N;
  a.near_off = near_offsets(L);
  a.m = m;
  a.alpha = alpha;
  a.X = X;
  a.ldx = ldx;
  a.Y = Y;
  a.ldy = ldy;
  a.xh = L.xh;
  a.yh = L.yh;
  // one host list, uploaded at once
  std::vector<int32_t> H;
  std::vector<std::pair<int, int>> fwd, bwd;
  std::vector<int32_t> fl, ff, bl, bf;
  int o_fwd = 0, o_bl = 0, o_bf = 0, o_cl = 0, o_cp = 0, o_ce = 0, n_cout = 0;
  if (!adm.empty()) {
    level_runs(tin, cin, true, false, fl, ff, fwd);
    level_runs(tout, cout, false, true, bl, bf, bwd);
    // couplings grouped by Y-side cluster
    std::map<int32_t, std::vector<std::pair<int32_t, int32_t>>> by;
    for (int32_t x : adm) {
      const int32_t co = trans ? bt.col[x] : bt.row[x];
      const int32_t ci = trans ? bt.row[x] : bt.col[x];
      by[co].push_back({bt.slot[x], ci});
    }
    o_fwd = (int)H.size();
    H.insert(H.end(), fl.begin(), fl.end());
    o_bl = (int)H.size();
    H.insert(H.end(), bl.begin(), bl.end());
    o_bf = (int)H.size();
    H.insert(H.end(), bf.begin(), bf.end());
    o_cl = (int)H.size();
    for (auto& kv : by) H.push_back(kv.first);
    n_cout = (int)by.size();
    o_cp = (int)H.size();
    int acc = 0;
    for (auto& kv : by) {
      H.push_back(acc);
      acc += (int)kv.second.size();
    }
    H.push_back(acc);
    o_ce = (int)H.size();
    for (auto& kv : by)
      for (auto& e : kv.second) {
        H.push_back(e.first);
        H.push_back(e.second);
      }
  }
  // leaves of the Y side with the nearfield blocks containing them
  const int32_t oend = cout + tout.subtree[cout];
  std::vector<int32_t> leaves;
  for (int32_t x = cout; x < oend; ++x)
    if (tout.leaf(x)) leaves.push_back(x);
  std::vector<std::vector<std::array<int32_t, 3>>> per(leaves.size());
  if (!near.empty()) {
    std::vector<int32_t> pos(oend - cout, -1);
    for (size_t i = 0; i < leaves.size(); ++i) pos[leaves[i] - cout] = (int32_t)i;
    for (int32_t x : near) {
      const int32_t co = trans ? bt.col[x] : bt.row[x];
      const int32_t ci = trans ? bt.row[x] : bt.col[x];
      for (int32_t l = co; l < co + tout.subtree[co]; ++l)
        if (tout.leaf(l)) per[pos[l - cout]].push_back({bt.slot[x], ci, co});
    }
  }
  const int o_lv = (int)H.size();
  H.insert(H.end(), leaves.begin(), leaves.end());
  const int o_lp = (int)H.size();
  int acc = 0;
  for (auto& v : per) {
    H.push_back(acc);
    acc += (int)v.size();
  }
  H.push_back(acc);
  const int o_le = (int)H.size();
  for (auto& v : per)
    for (auto& e : v) H.insert(H.end(), e.begin(), e.end());
  int32_t* D = upload_list(L, H);
  const size_t slot = (size_t)Z->kcap * m;
  zero(L.yh + (size_t)cout * slot, (size_t)tout.subtree[cout] * slot, L.st);
  if (!adm.empty()) {
    for (auto& r : fwd) launch_bp_forward(a, D + o_fwd + r.first, r.second, L.st);
    launch_bp_coupling(a, D + o_cl, n_cout, D + o_cp, D + o_ce, L.st);
    for (auto& r : bwd) launch_bp_backward(a, D + o_bl + r.first, D + o_bf + r.first, r.second, L.st);
  }
  launch_bp_leaves(a, D + o_lv, (int)leaves.size(), D + o_lp, D + o_le, L.st);
  H2_CUDA(cudaGetLastError());
}

// out (#c x k_c, ld) = the basis of cluster c of one side (Eq. (nested))
void expand(Lr& L, const h2_matrix* Z, int side, int32_t c, double* out, int64_t ld) {
  const ClusterTree& ct = tree(Z, side);
  const int k = (side == 0 ? Z->V : Z->W).rank[c];
  if (k == 0) return;
  ensure_work(L, k, Z->kcap);
  BlockProd a{};
  a.in = view(Z, side);
  a.out = view(Z, side);
  a.kcap = Z->kcap;
  a.trans = 0;
  a.in_off0 = a.out_off0 = ct.off[c];
  a.S = Z->d_S;
  a.N = Z->d_N;
  a.near_off = near_offsets(L);
  a.m = k;
  a.alpha = 1.0;
  a.X = nullptr;
  a.ldx = 0;
  a.Y = out;
  a.ldy = ld;
  a.xh = L.xh;
  a.yh = L.yh;
  std::vector<int32_t> bl, bf, H;
  std::vector<std::pair<int, int>> bwd;
  level_runs(ct, c, false, true, bl, bf, bwd);
  H = bl;
  H.insert(H.end(), bf.begin(), bf.end());
  const int o_lv = (int)H.size();
  int nl = 0;
  for (int32_t x = c; x < c + ct.subtree[c]; ++x)
    if (ct.leaf(x)) {
      H.push_back(x);
      ++nl;
    }
  const int o_lp = (int)H.size();
  for (int i = 0; i <= nl; ++i) H.push_back(0);
  int32_t* D = upload_list(L, H);
  const size_t slot = (size_t)Z->kcap * k;
  zero(L.yh + (size_t)c * slot, (size_t)ct.subtree[c] * slot, L.st);
  launch_identity(L.yh + (size_t)c * slot, k, Z->kcap, L.st);
  for (auto& r : bwd) launch_bp_backward(a, D + r.first, D + (int)bl.size() + r.first, r.second, L.st);
  H2_CUDA(cudaMemset2DAsync(out, ld * sizeof(double), 0, ct.size[c] * sizeof(double), k, L.st));
  launch_bp_leaves(a, D + o_lv, nl, D + o_lp, D + o_lp, L.st);
  H2_CUDA(cudaGetLastError());
}

inline int64_t csize(const h2_matrix* Z, int32_t c) { return Z->rows.size[c]; }
inline int rank_of(const h2_matrix* Z, int side, int32_t c) { return (side == 0 ? Z->V : Z->W).rank[c]; }
inline double* near_ptr(const h2_matrix* Z, int32_t b) { return Z->d_N + Z->near_off[Z->blocks.slot[b]]; }
inline double* coupling_ptr(const h2_matrix* Z, int32_t b) {
  return Z->d_S + (size_t)Z->blocks.slot[b] * Z->kcap * Z->kcap;
}

int32_t son(const BlockTree& bt, int32_t b, int32_t t, int32_t s) {
  for (int k = 0; k < 4; ++k) {
    const int32_t c = bt.son4[4 * b + k];
    if (c >= 0 && bt.row[c] == t && bt.col[c] == s) return c;
  }
  throw Error(H2_EINTERNAL, "block tree: missing son");
}


// ----------------------------------------------------------- local updates
void apply_update(Lr& L, int32_t b, const double* A, int64_t lda, const double* B, int64_t ldb, int u) {
  Timer tm(L.t_update);
  h2_matrix* Z = L.Z;
  const BlockTree& bt = Z->blocks;
  int j = 0;
  while (j < u) {
    int kmax = 0;
    const int32_t t = bt.row[b], s = bt.col[b];
    for (int32_t c = t; c < t + Z->rows.subtree[t]; ++c) kmax = std::max(kmax, Z->V.rank[c]);
    for (int32_t c = s; c < s + Z->cols.subtree[s]; ++c) kmax = std::max(kmax, Z->W.rank[c]);
    const int w = std::min(std::min(kMaxCols - 1, std::max(1, kMaxCols - kmax)), u - j);
    if (!L.eng) L.eng = engine_new();
    engine_update(L.ctx, Z, L.eng, b, w, A + (size_t)j * lda, lda, B + (size_t)j * ldb, ldb, L.eps,
                  L.max_rank);
    ++L.updates;
    j += w;
  }
}

// ------------------------------------------------------ products (Section 3)
struct Term {
  int32_t z = -1;          // target block
  int32_t tc = -1, rc = -1;  // row and column cluster of the product
  bool dense = false;      // P for a nearfield target
  int u = 0;               // columns of the factor pair
  DArr A, B;               // factor pair (#tc x u, #rc x u) or P (#tc x #rc) in A
};

struct Temp {
  int32_t z = -1;
  std::vector<Term> terms;
};

struct Item {
  bool temp = false;
  Term term;
  Temp tmp;
};

DArr identity(Lr& L, int64_t n) {
  DArr I(n * n, L.st);
  launch_eye(I.p, (int)n, n, L.st);
  return I;
}

// the term alpha X|_x (Y|_yh)^* when x or yh is a leaf (the product of the
// Cholesky factorisation: x = (t, s), yh = (r, s), the product (t, r));
// the transpose of an admissible block V_r S W_s^* is W_s S^* V_r^*, of a
// dense leaf its transpose
Term case2_t(Lr& L, double alpha, int32_t x, int32_t yh, bool near_target) {
  const h2_matrix* Z = L.Z;
  const h2_matrix* MX = L.X ? L.X : L.Z;
  const h2_matrix* MY = L.Y ? L.Y : L.Z;
  const BlockTree& bt = Z->blocks;
  const int32_t t = bt.row[x], s = bt.col[x], r = bt.row[yh];
  const int64_t mt = csize(Z, t), ms = csize(Z, s), mr = csize(Z, r);
  Term T;
  T.tc = t;
  T.rc = r;
  if (bt.kind[yh] == kAdm) {
    // (X|_x W_s) S_yh^*, V_r
    const int ks = rank_of(MY, 1, s), lr = rank_of(MY, 0, r);
    T.u = lr;
    if (lr == 0) return T;
    DArr Ws(ms * std::max(ks, 1), L.st), Xt(mt * std::max(ks, 1), L.st);
    T.A = DArr(mt * lr, L.st);
    T.B = DArr(mr * lr, L.st);
    if (ks > 0) {
      expand(L, MY, 1, s, Ws.p, ms);
      zero(Xt.p, mt * ks, L.st);
      block_prod(L, MX, x, 0, 1.0, Ws.p, ms, Xt.p, mt, ks);
      launch_gemm((int)mt, lr, ks, alpha, Xt.p, mt, 0, coupling_ptr(MY, yh), MY->kcap, 1, 0.0, T.A.p, mt, L.st);
    } else {
      zero(T.A.p, mt * lr, L.st);
    }
    expand(L, MY, 0, r, T.B.p, mr);
    ++L.products;
    return T;
  }
  if (bt.kind[x] == kAdm) {
    // V_t, (Y|_yh W_s) S_x^*
    const int kt = rank_of(MX, 0, t), ls = rank_of(MX, 1, s);
    T.u = kt;
    if (kt == 0) return T;
    DArr Ws(ms * std::max(ls, 1), L.st), Yt(mr * std::max(ls, 1), L.st);
    T.A = DArr(mt * kt, L.st);
    T.B = DArr(mr * kt, L.st);
    expand(L, MX, 0, t, T.A.p, mt);
    if (ls > 0) {
      expand(L, MX, 1, s, Ws.p, ms);
      zero(Yt.p, mr * ls, L.st);
      block_prod(L, MY, yh, 0, 1.0, Ws.p, ms, Yt.p, mr, ls);
      launch_gemm((int)mr, kt, ls, alpha, Yt.p, mr, 0, coupling_ptr(MX, x), MX->kcap, 1, 0.0, T.B.p, mr, L.st);
    } else {
      zero(T.B.p, mr * kt, L.st);
    }
    ++L.products;
    return T;
  }
  ++L.products;
  const bool xn = bt.kind[x] == kNear, yn = bt.kind[yh] == kNear;
  if (near_target) {
    // P = alpha X Y^* (#t x #r)
    T.dense = true;
    T.A = DArr(mt * mr, L.st);
    zero(T.A.p, mt * mr, L.st);
    if (xn && yn) {
      launch_gemm((int)mt, (int)mr, (int)ms, alpha, near_ptr(MX, x), mt, 0, near_ptr(MY, yh), mr, 1, 0.0, T.A.p, mt,
                  L.st);
    } else if (yn) {   // X subdivided: X (Y^*) by the block product
      DArr Yt(ms * mr, L.st);
      launch_transpose((int)mr, (int)ms, 1.0, near_ptr(MY, yh), mr, Yt.p, ms, L.st);
      block_prod(L, MX, x, 0, alpha, Yt.p, ms, T.A.p, mt, (int)mr);
    } else {           // Y subdivided: P^* = Y (alpha X^*)
      DArr Xt(ms * mt, L.st), Pt(mr * mt, L.st);
      launch_transpose((int)mt, (int)ms, alpha, near_ptr(MX, x), mt, Xt.p, ms, L.st);
      zero(Pt.p, mr * mt, L.st);
      block_prod(L, MY, yh, 0, 1.0, Xt.p, ms, Pt.p, mr, (int)mt);
      launch_transpose((int)mr, (int)mt, 1.0, Pt.p, mr, T.A.p, mt, L.st);
    }
    return T;
  }
  // factor pair through the smallest dimension (reading 3)
  if (xn && yn && ms <= std::min(mt, mr)) {
    // alpha X and Y
    T.u = (int)ms;
    T.A = DArr(mt * ms, L.st);
    T.B = DArr(mr * ms, L.st);
    launch_axpby(mt * ms, alpha, near_ptr(MX, x), 0.0, T.A.p, L.st);
    H2_CUDA(cudaMemcpyAsync(T.B.p, near_ptr(MY, yh), mr * ms * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
    return T;
  }
  if (mt <= mr) {
    // (I, P^*): P^* = alpha Y X^* (#r x #t)
    T.u = (int)mt;
    T.A = identity(L, mt);
    T.B = DArr(mr * mt, L.st);
    zero(T.B.p, mr * mt, L.st);
    if (xn && yn) {
      launch_gemm((int)mr, (int)mt, (int)ms, alpha, near_ptr(MY, yh), mr, 0, near_ptr(MX, x), mt, 1, 0.0, T.B.p, mr,
                  L.st);
    } else if (xn) {   // Y subdivided: Y (alpha X^*) by the block product
      DArr Xt(ms * mt, L.st);
      launch_transpose((int)mt, (int)ms, alpha, near_ptr(MX, x), mt, Xt.p, ms, L.st);
      block_prod(L, MY, yh, 0, 1.0, Xt.p, ms, T.B.p, mr, (int)mt);
    } else {
      throw Error(H2_EINTERNAL, "dense term: unexpected block kinds");
    }
    return T;
  }
  // (P, I): P = alpha X Y^* (#t x #r)
  T.u = (int)mr;
  T.A = DArr(mt * mr, L.st);
  T.B = identity(L, mr);
  zero(T.A.p, mt * mr, L.st);
  if (xn && yn) {
    launch_gemm((int)mt, (int)mr, (int)ms, alpha, near_ptr(MX, x), mt, 0, near_ptr(MY, yh), mr, 1, 0.0, T.A.p, mt,
                L.st);
  } else if (yn) {
    DArr Yt(ms * mr, L.st);
    launch_transpose((int)mr, (int)ms, 1.0, near_ptr(MY, yh), mr, Yt.p, ms, L.st);
    block_prod(L, MX, x, 0, alpha, Yt.p, ms, T.A.p, mt, (int)mr);
  } else {
    throw Error(H2_EINTERNAL, "dense term: unexpected block kinds");
  }
  return T;
}

// the term alpha X|_x Y|_y when x or y is a leaf (Section 6, Case 2)
Term case2(Lr& L, double alpha, int32_t x, int32_t y, bool near_target) {
  if (L.yt) return case2_t(L, alpha, x, y, near_target);
  const h2_matrix* Z = L.Z;
  const h2_matrix* MX = L.X ? L.X : L.Z;   // the factors (the product's X and Y)
  const h2_matrix* MY = L.Y ? L.Y : L.Z;
  const BlockTree& bt = Z->blocks;
  const int32_t t = bt.row[x], s = bt.col[x], r = bt.col[y];
  const int64_t mt = csize(Z, t), ms = csize(Z, s), mr = csize(Z, r);
  Term T;
  T.tc = t;
  T.rc = r;
  if (bt.kind[y] == kAdm) {
    // (X|_x V_s) S_y, W_r
    const int ks = rank_of(MY, 0, s), lr = rank_of(MY, 1, r);
    T.u = lr;
    if (lr == 0) return T;
    DArr Vs(ms * std::max(ks, 1), L.st), Xt(mt * std::max(ks, 1), L.st);
    T.A = DArr(mt * lr, L.st);
    T.B = DArr(mr * lr, L.st);
    if (ks > 0) {
      expand(L, MY, 0, s, Vs.p, ms);
      zero(Xt.p, mt * ks, L.st);
      block_prod(L, MX, x, 0, 1.0, Vs.p, ms, Xt.p, mt, ks);
      launch_gemm((int)mt, lr, ks, alpha, Xt.p, mt, 0, coupling_ptr(MY, y), MY->kcap, 0, 0.0, T.A.p, mt, L.st);
    } else {
      zero(T.A.p, mt * lr, L.st);
    }
    expand(L, MY, 1, r, T.B.p, mr);
    ++L.products;
    return T;
  }
  if (bt.kind[x] == kAdm) {
    // V_t, (Y|_y^* W_s) S_x^*
    const int kt = rank_of(MX, 0, t), ls = rank_of(MX, 1, s);
    T.u = kt;
    if (kt == 0) return T;
    DArr Ws(ms * std::max(ls, 1), L.st), Yt(mr * std::max(ls, 1), L.st);
    T.A = DArr(mt * kt, L.st);
    T.B = DArr(mr * kt, L.st);
    expand(L, MX, 0, t, T.A.p, mt);
    if (ls > 0) {
      expand(L, MX, 1, s, Ws.p, ms);
      zero(Yt.p, mr * ls, L.st);
      block_prod(L, MY, y, 1, 1.0, Ws.p, ms, Yt.p, mr, ls);
      launch_gemm((int)mr, kt, ls, alpha, Yt.p, mr, 0, coupling_ptr(MX, x), MX->kcap, 1, 0.0, T.B.p, mr, L.st);
    } else {
      zero(T.B.p, mr * kt, L.st);
    }
    ++L.products;
    return T;
  }
  // both inadmissible leaves, or one inadmissible and one subdivided
  ++L.products;
  const bool xn = bt.kind[x] == kNear, yn = bt.kind[y] == kNear;
  if (near_target) {
    // P = alpha X Y (#t x #r); a nearfield target has a leaf row or column
    T.dense = true;
    T.A = DArr(mt * mr, L.st);
    zero(T.A.p, mt * mr, L.st);
    if (xn && yn) {
      launch_gemm((int)mt, (int)mr, (int)ms, alpha, near_ptr(MX, x), mt, 0, near_ptr(MY, y), ms, 0, 0.0, T.A.p, mt,
                  L.st);
    } else if (yn) {   // X subdivided: X Y by the block product with Y's columns
      block_prod(L, MX, x, 0, alpha, near_ptr(MY, y), ms, T.A.p, mt, (int)mr);
    } else {           // Y subdivided: P^* = Y^* (alpha X^*) by the transposed block product
      DArr Xt(ms * mt, L.st), Pt(mr * mt, L.st);
      launch_transpose((int)mt, (int)ms, alpha, near_ptr(MX, x), mt, Xt.p, ms, L.st);
      zero(Pt.p, mr * mt, L.st);
      block_prod(L, MY, y, 1, 1.0, Xt.p, ms, Pt.p, mr, (int)mt);
      launch_transpose((int)mr, (int)mt, 1.0, Pt.p, mr, T.A.p, mt, L.st);
    }
    return T;
  }
  // factor pair through the smallest dimension (reading 3)
  if (xn && yn && ms <= std::min(mt, mr)) {
    // alpha X and Y^*
    T.u = (int)ms;
    T.A = DArr(mt * ms, L.st);
    T.B = DArr(mr * ms, L.st);
    launch_axpby(mt * ms, alpha, near_ptr(MX, x), 0.0, T.A.p, L.st);
    launch_transpose((int)ms, (int)mr, 1.0, near_ptr(MY, y), ms, T.B.p, mr, L.st);
    return T;
  }
  if (mt <= mr) {
    // (I, P^*): P^* = alpha Y^* X^* (#r x #t)
    T.u = (int)mt;
    T.A = identity(L, mt);
    T.B = DArr(mr * mt, L.st);
    zero(T.B.p, mr * mt, L.st);
    if (xn && yn) {
      launch_gemm((int)mr, (int)mt, (int)ms, alpha, near_ptr(MY, y), ms, 1, near_ptr(MX, x), mt, 1, 0.0, T.B.p, mr,
                  L.st);
    } else if (xn) {   // Y subdivided: Y^* (alpha X^*) by the transposed block product
      DArr Xt(ms * mt, L.st);
      launch_transpose((int)mt, (int)ms, alpha, near_ptr(MX, x), mt, Xt.p, ms, L.st);
      block_prod(L, MY, y, 1, 1.0, Xt.p, ms, T.B.p, mr, (int)mt);
    } else {
      throw Error(H2_EINTERNAL, "dense term: unexpected block kinds");
    }
    return T;
  }
  // (P, I): P = alpha X Y (#t x #r)
  T.u = (int)mr;
  T.A = DArr(mt * mr, L.st);
  T.B = identity(L, mr);
  zero(T.A.p, mt * mr, L.st);
  if (xn && yn) {
    launch_gemm((int)mt, (int)mr, (int)ms, alpha, near_ptr(MX, x), mt, 0, near_ptr(MY, y), ms, 0, 0.0, T.A.p, mt,
                L.st);
  } else if (yn) {
    block_prod(L, MX, x, 0, alpha, near_ptr(MY, y), ms, T.A.p, mt, (int)mr);
  } else {
    throw Error(H2_EINTERNAL, "dense term: unexpected block kinds");
  }
  return T;
}

void collect_virtual(Lr& L, double alpha, int32_t x, int32_t y, std::vector<Term>& bucket) {
  const BlockTree& bt = L.Z->blocks;
  const ClusterTree& ct = L.Z->rows;
  if (bt.kind[x] == kSub && bt.kind[y] == kSub) {
    // with the second factor read transposed, y = (r, s)
    const int32_t t = bt.row[x], s = bt.col[x], r = L.yt ? bt.row[y] : bt.col[y];
    for (int32_t s1 : {ct.son0[s], ct.son1[s]})
      for (int32_t t1 : {ct.son0[t], ct.son1[t]})
        for (int32_t r1 : {ct.son0[r], ct.son1[r]})
          collect_virtual(L, alpha, son(bt, x, t1, s1), L.yt ? son(bt, y, r1, s1) : son(bt, y, s1, r1), bucket);
    return;
  }
  bucket.push_back(case2(L, alpha, x, y, false));
}

void collect(Lr& L, double alpha, int32_t x, int32_t y, int32_t z, std::vector<Item>& out) {
  const BlockTree& bt = L.Z->blocks;
  const ClusterTree& ct = L.Z->rows;
  if (bt.kind[x] == kSub && bt.kind[y] == kSub) {
    const int32_t t = bt.row[x], s = bt.col[x], r = L.yt ? bt.row[y] : bt.col[y];
    if (bt.kind[z] == kSub) {
      const bool diag = bt.row[z] == bt.col[z];
      for (int32_t s1 : {ct.son0[s], ct.son1[s]})
        for (int32_t t1 : {ct.son0[t], ct.son1[t]})
          for (int32_t r1 : {ct.son0[r], ct.son1[r]}) {
            if (L.lower && diag && ct.off[t1] < ct.off[r1]) continue;   // strictly above the diagonal
            collect(L, alpha, son(bt, x, t1, s1), L.yt ? son(bt, y, r1, s1) : son(bt, y, s1, r1), son(bt, z, t1, r1),
                    out);
          }
      return;
    }
    if (bt.kind[z] != kAdm) throw Error(H2_EINTERNAL, "inadmissible target of subdivided factors");
    std::map<std::pair<int32_t, int32_t>, std::vector<Term>> temps;
    for (int32_t s1 : {ct.son0[s], ct.son1[s]})
      for (int32_t t1 : {ct.son0[t], ct.son1[t]})
        for (int32_t r1 : {ct.son0[r], ct.son1[r]})
          collect_virtual(L, alpha, son(bt, x, t1, s1), L.yt ? son(bt, y, r1, s1) : son(bt, y, s1, r1),
                          temps[{t1, r1}]);
    for (int32_t t1 : {ct.son0[t], ct.son1[t]})
      for (int32_t r1 : {ct.son0[r], ct.son1[r]}) {
        Item it;
        it.temp = true;
        it.tmp.z = z;
        it.tmp.terms = std::move(temps[{t1, r1}]);
        out.push_back(std::move(it));
      }
    return;
  }
  Item it;
  it.term = case2(L, alpha, x, y, bt.kind[z] == kNear);
  it.term.z = z;
  out.push_back(std::move(it));
}

void apply_term(Lr& L, const Term& T) {
  h2_matrix* Z = L.Z;
  const BlockTree& bt = Z->blocks;
  const int64_t mt = csize(Z, T.tc), mr = csize(Z, T.rc);
  if (bt.kind[T.z] == kNear) {
    double* N = near_ptr(Z, T.z);
    if (T.dense)
      launch_axpby(mt * mr, 1.0, T.A.p, 1.0, N, L.st);
    else if (T.u > 0)
      launch_gemm((int)mt, (int)mr, T.u, 1.0, T.A.p, mt, 0, T.B.p, mr, 1, 1.0, N, mt, L.st);
    return;
  }
  if (T.u > 0) apply_update(L, T.z, T.A.p, mt, T.B.p, mr, T.u);
}

// Scratch of one temporary's truncation (reading 2).
struct TempWork {
  int64_t mt = 0, mr = 0;
  int m = 0, ka = 0, kb = 0;
  DArr A, B, tauA, tauB, C, W, TA, TB;
};

// The terms of every temporary of a product stacked into factor pairs,
// extended by zeros to the target, and truncated at once: Householder QR of
// both factors and the SVD of the core R_A R_B^* with the rank rule (one
// block per temporary).  The temporaries depend only on the terms (reading
// 1), so one batch of launches and one synchronisation serve the whole
// product.  ranks[i] receives the rank of item i's temporary.
void compress_temps(Lr& L, const std::vector<Item>& items, std::vector<TempWork>& work, std::vector<int>& ranks) {
  const double t0 = now_s();
  const double u0 = L.t_update;
  struct Done {
    Lr& L;
    double t0, u0;
    ~Done() { L.t_temps += (now_s() - t0) - (L.t_update - u0); }
  } done{L, t0, u0};
  h2_matrix* Z = L.Z;
  const BlockTree& bt = Z->blocks;
  std::vector<Compress> desc;
  std::vector<size_t> which;
  int max_core = 0;
  for (size_t i = 0; i < items.size(); ++i) {
    if (!items[i].temp) continue;
    const Temp& tmp = items[i].tmp;
    const int32_t t = bt.row[tmp.z], r = bt.col[tmp.z];
    const int64_t mt = csize(Z, t), mr = csize(Z, r);
    int m = 0;
    for (const Term& T : tmp.terms) m += T.u;
    if (m == 0) continue;
    if (m > kCompressMax)
      throw Error(H2_EINTERNAL, "temporary stacking more than " + std::to_string(kCompressMax) + " columns");
    TempWork& w = work[i];
    w.mt = mt;
    w.mr = mr;
    w.m = m;
    w.ka = (int)std::min<int64_t>(mt, m);
    w.kb = (int)std::min<int64_t>(mr, m);
    w.A = DArr(mt * m, L.st);
    w.B = DArr(mr * m, L.st);
    zero(w.A.p, mt * m, L.st);
    zero(w.B.p, mr * m, L.st);
    int c = 0;
    for (const Term& T : tmp.terms) {
      if (T.u == 0) continue;
      const int64_t a0 = Z->rows.off[T.tc] - Z->rows.off[t];
      const int64_t b0 = Z->cols.off[T.rc] - Z->cols.off[r];
      const int64_t rt = csize(Z, T.tc), rr = csize(Z, T.rc);
      H2_CUDA(cudaMemcpy2DAsync(w.A.p + a0 + (size_t)c * mt, mt * sizeof(double), T.A.p, rt * sizeof(double),
                                rt * sizeof(double), T.u, cudaMemcpyDeviceToDevice, L.st));
      H2_CUDA(cudaMemcpy2DAsync(w.B.p + b0 + (size_t)c * mr, mr * sizeof(double), T.B.p, rr * sizeof(double),
                                rr * sizeof(double), T.u, cudaMemcpyDeviceToDevice, L.st));
      c += T.u;
    }
    w.tauA = DArr(m, L.st);
    w.tauB = DArr(m, L.st);
    w.C = DArr((size_t)m * m, L.st);
    w.W = DArr((size_t)m * m, L.st);
    w.TA = DArr((size_t)m * m, L.st);
    w.TB = DArr((size_t)m * m, L.st);
    desc.push_back({w.A.p, w.B.p, (int)mt, (int)mr, m, w.ka, w.kb, w.tauA.p, w.tauB.p, w.C.p, w.W.p, w.TA.p, w.TB.p,
                    nullptr});
    which.push_back(i);
    max_core = std::max(max_core, w.ka * w.kb + w.kb * w.kb);
    ++L.n_temps;
    L.temp_cols += m;
  }
  const int n = (int)desc.size();
  if (n == 0) return;
  // device copies of the descriptors and the flags (rank, nonzero A, nonzero B)
  const size_t dsz = (n * sizeof(Compress) + sizeof(double) - 1) / sizeof(double);
  DArr dd(dsz, L.st), df((3 * (size_t)n * sizeof(int) + sizeof(double) - 1) / sizeof(double), L.st);
  int* flags = reinterpret_cast<int*>(df.p);
  for (int k = 0; k < n; ++k) desc[k].flags = flags + 3 * k;
  H2_CUDA(cudaMemcpyAsync(dd.p, desc.data(), n * sizeof(Compress), cudaMemcpyHostToDevice, L.st));
  launch_compress_batch(reinterpret_cast<const Compress*>(dd.p), n, max_core, L.eps, L.st);
  H2_CUDA(cudaGetLastError());
  std::vector<int> h(3 * (size_t)n);
  H2_CUDA(cudaMemcpyAsync(h.data(), flags, h.size() * sizeof(int), cudaMemcpyDeviceToHost, L.st));
  {
    Timer tw(L.t_temp_wait);
    H2_CUDA(cudaStreamSynchronize(L.st));
  }
  for (int k = 0; k < n; ++k) ranks[which[k]] = h[3 * k];
}

// A' = Q_A U_r Sigma_r, B' = Q_B W_r of a truncated temporary, added to its
// target by one local update
void finish_temp(Lr& L, const Temp& tmp, TempWork& w, int rk) {
  if (w.m == 0 || rk == 0) return;
  const double t0 = now_s();
  const double u0 = L.t_update;
  struct Done {
    Lr& L;
    double t0, u0;
    ~Done() { L.t_temps += (now_s() - t0) - (L.t_update - u0); }
  } done{L, t0, u0};
  DArr A2(w.mt * rk, L.st), B2(w.mr * rk, L.st);
  launch_apply_q(w.A.p, w.mt, (int)w.mt, w.tauA.p, w.TA.p, A2.p, w.B.p, w.mr, (int)w.mr, w.tauB.p, w.TB.p, B2.p,
                 w.m, rk, L.st);
  H2_CUDA(cudaGetLastError());
  apply_update(L, tmp.z, A2.p, w.mt, B2.p, w.mr, rk);
}

// The low-rank terms of a product for one target block that is not an
// inadmissible leaf, concatenated in the recursion's order into one factor
// pair and added by one local update (reading 1).
void apply_terms(Lr& L, const std::vector<Item>& items, const std::vector<size_t>& idx) {
  const Term& T0 = items[idx[0]].term;
  if (idx.size() == 1) {
    apply_term(L, T0);
    return;
  }
  h2_matrix* Z = L.Z;
  const int64_t mt = csize(Z, T0.tc), mr = csize(Z, T0.rc);
  int u = 0;
  for (size_t i : idx) u += items[i].term.u;
  if (u == 0) return;
  DArr A(mt * u, L.st), B(mr * u, L.st);
  int c = 0;
  for (size_t i : idx) {
    const Term& T = items[i].term;
    if (T.u == 0) continue;
    H2_CUDA(cudaMemcpyAsync(A.p + (size_t)c * mt, T.A.p, mt * T.u * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
    H2_CUDA(cudaMemcpyAsync(B.p + (size_t)c * mr, T.B.p, mr * T.u * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
    c += T.u;
  }
  apply_update(L, T0.z, A.p, mt, B.p, mr, u);
}

void mul(Lr& L, double alpha, int32_t x, int32_t y, int32_t z) {
  std::vector<Item> items;
  {
    Timer tm(L.t_terms);
    collect(L, alpha, x, y, z, items);
  }
  const BlockTree& bt = L.Z->blocks;
  // the terms of each target block (not an inadmissible leaf), in order
  std::map<int32_t, std::vector<size_t>> groups;
  for (size_t i = 0; i < items.size(); ++i)
    if (!items[i].temp && bt.kind[items[i].term.z] != kNear) groups[items[i].term.z].push_back(i);
  std::vector<TempWork> work(items.size());
  std::vector<int> ranks(items.size(), 0);
  compress_temps(L, items, work, ranks);
  for (size_t i = 0; i < items.size(); ++i) {
    if (items[i].temp) {
      finish_temp(L, items[i].tmp, work[i], ranks[i]);
      work[i] = TempWork();   // its scratch goes back to the stream-ordered pool
    } else if (bt.kind[items[i].term.z] == kNear) {
      apply_term(L, items[i].term);
    } else {
      auto g = groups.find(items[i].term.z);
      if (g == groups.end()) continue;   // added with the block's first term
      apply_terms(L, items, g->second);
      groups.erase(g);
    }
  }
}

// ------------------------------------------------ substitutions (Section 3)
// Y (#t x m) <- L|_{t x t}^-1 Y, d = (t, t)
void lsolve_dense(Lr& L, int32_t d, double* Y, int64_t ldy, int m) {
  const h2_matrix* Z = L.Z;
  const BlockTree& bt = Z->blocks;
  const int32_t t = bt.row[d];
  if (bt.kind[d] == kNear) {
    launch_trsm(0, near_ptr(Z, d), (int)csize(Z, t), csize(Z, t), Y, m, ldy, L.st);
    return;
  }
  const int32_t t1 = Z->rows.son0[t], t2 = Z->rows.son1[t];
  const int64_t n1 = csize(Z, t1);
  lsolve_dense(L, son(bt, d, t1, t1), Y, ldy, m);
  block_prod(L, L.Z, son(bt, d, t2, t1), 0, -1.0, Y, ldy, Y + n1, ldy, m);
  lsolve_dense(L, son(bt, d, t2, t2), Y + n1, ldy, m);
}

// Y (#t x m) <- R|_{t x t}^-1 Y
void usolve_dense(Lr& L, int32_t d, double* Y, int64_t ldy, int m) {
  const h2_matrix* Z = L.Z;
  const BlockTree& bt = Z->blocks;
  const int32_t t = bt.row[d];
  if (bt.kind[d] == kNear) {
    launch_trsm(1, near_ptr(Z, d), (int)csize(Z, t), csize(Z, t), Y, m, ldy, L.st);
    return;
  }
  const int32_t t1 = Z->rows.son0[t], t2 = Z->rows.son1[t];
  const int64_t n1 = csize(Z, t1);
  usolve_dense(L, son(bt, d, t2, t2), Y + n1, ldy, m);
  block_prod(L, L.Z, son(bt, d, t1, t2), 0, -1.0, Y + n1, ldy, Y, ldy, m);
  usolve_dense(L, son(bt, d, t1, t1), Y, ldy, m);
}

// Yt (#s x m) <- R|_{s x s}^-* Yt, i.e. X R = Y with X^* = Yt on return
void rsolve_dense_t(Lr& L, int32_t d, double* Yt, int64_t ldy, int m) {
  const h2_matrix* Z = L.Z;
  const BlockTree& bt = Z->blocks;
  const int32_t s = bt.row[d];
  if (bt.kind[d] == kNear) {
    // X R = Y on the transposed columns: x^* R = y^*
    const int64_t ms = csize(Z, s);
    DArr X(m * ms, L.st);
    launch_transpose((int)ms, m, 1.0, Yt, ldy, X.p, m, L.st);
    launch_trsm(2, near_ptr(Z, d), (int)ms, ms, X.p, m, m, L.st);
    launch_transpose(m, (int)ms, 1.0, X.p, m, Yt, ldy, L.st);
    return;
  }
  const int32_t s1 = Z->rows.son0[s], s2 = Z->rows.son1[s];
  const int64_t n1 = csize(Z, s1);
  rsolve_dense_t(L, son(bt, d, s1, s1), Yt, ldy, m);
  block_prod(L, L.Z, son(bt, d, s1, s2), 1, -1.0, Yt, ldy, Yt + n1, ldy, m);
  rsolve_dense_t(L, son(bt, d, s2, s2), Yt + n1, ldy, m);
}

void lsolve(Lr& L, int32_t d, int32_t x);
void rsolve(Lr& L, int32_t d, int32_t x);

void lsolve(Lr& L, int32_t d, int32_t x) {
  h2_matrix* Z = L.Z;
  const BlockTree& bt = Z->blocks;
  const int32_t t = bt.row[x], s = bt.col[x];
  if (bt.kind[x] == kNear) {
    Timer tm(L.t_solves);
    lsolve_dense(L, d, near_ptr(Z, x), csize(Z, t), (int)csize(Z, s));
    return;
  }
  if (bt.kind[x] == kAdm) {
    const int kt = rank_of(Z, 0, t), ls = rank_of(Z, 1, s);
    if (ls == 0 || kt == 0) return;        // the block is zero
    const int64_t mt = csize(Z, t), ms = csize(Z, s);
    DArr Vt(mt * kt, L.st), Xh(mt * ls, L.st), Ws(ms * ls, L.st);
    {
      Timer tm(L.t_solves);
      expand(L, L.Z, 0, t, Vt.p, mt);
      launch_gemm((int)mt, ls, kt, 1.0, Vt.p, mt, 0, coupling_ptr(Z, x), Z->kcap, 0, 0.0, Xh.p, mt, L.st);
      lsolve_dense(L, d, Xh.p, mt, ls);
      expand(L, L.Z, 1, s, Ws.p, ms);
    }
    engine_touch(L.eng, Z, x);   // a coupling written outside the update engine
    H2_CUDA(cudaMemsetAsync(coupling_ptr(Z, x), 0, (size_t)Z->kcap * Z->kcap * sizeof(double), L.st));
    apply_update(L, x, Xh.p, mt, Ws.p, ms, ls);
    return;
  }
  const ClusterTree& ct = Z->rows;
  const int32_t t1 = ct.son0[t], t2 = ct.son1[t];
  for (int32_t s1 : {ct.son0[s], ct.son1[s]}) lsolve(L, son(bt, d, t1, t1), son(bt, x, t1, s1));
  for (int32_t s1 : {ct.son0[s], ct.son1[s]}) mul(L, -1.0, son(bt, d, t2, t1), son(bt, x, t1, s1), son(bt, x, t2, s1));
  for (int32_t s1 : {ct.son0[s], ct.son1[s]}) lsolve(L, son(bt, d, t2, t2), son(bt, x, t2, s1));
}

void rsolve(Lr& L, int32_t d, int32_t x) {
  h2_matrix* Z = L.Z;
  const BlockTree& bt = Z->blocks;
  const int32_t t = bt.row[x], s = bt.col[x];
  if (bt.kind[x] == kNear) {
    const int64_t mt = csize(Z, t), ms = csize(Z, s);
    Timer tm(L.t_solves);
    // transpose in, solve R^* X^* = Y^*, transpose out
    DArr Yt(ms * mt, L.st);
    launch_transpose((int)mt, (int)ms, 1.0, near_ptr(Z, x), mt, Yt.p, ms, L.st);
    rsolve_dense_t(L, d, Yt.p, ms, (int)mt);
    launch_transpose((int)ms, (int)mt, 1.0, Yt.p, ms, near_ptr(Z, x), mt, L.st);
    return;
  }
  if (bt.kind[x] == kAdm) {
    const int kt = rank_of(Z, 0, t), ls = rank_of(Z, 1, s);
    if (ls == 0 || kt == 0) return;
    const int64_t mt = csize(Z, t), ms = csize(Z, s);
    DArr Ws(ms * ls, L.st), Bh(ms * kt, L.st), Vt(mt * kt, L.st);
    {
      Timer tm(L.t_solves);
      expand(L, L.Z, 1, s, Ws.p, ms);
      launch_gemm((int)ms, kt, ls, 1.0, Ws.p, ms, 0, coupling_ptr(Z, x), Z->kcap, 1, 0.0, Bh.p, ms, L.st);
      rsolve_dense_t(L, d, Bh.p, ms, kt);
      expand(L, L.Z, 0, t, Vt.p, mt);
    }
    engine_touch(L.eng, Z, x);   // a coupling written outside the update engine
    H2_CUDA(cudaMemsetAsync(coupling_ptr(Z, x), 0, (size_t)Z->kcap * Z->kcap * sizeof(double), L.st));
    apply_update(L, x, Vt.p, mt, Bh.p, ms, kt);
    return;
  }
  const ClusterTree& ct = Z->rows;
  const int32_t s1 = ct.son0[s], s2 = ct.son1[s];
  for (int32_t t1 : {ct.son0[t], ct.son1[t]}) rsolve(L, son(bt, d, s1, s1), son(bt, x, t1, s1));
  for (int32_t t1 : {ct.son0[t], ct.son1[t]}) mul(L, -1.0, son(bt, x, t1, s1), son(bt, d, s1, s2), son(bt, x, t1, s2));
  for (int32_t t1 : {ct.son0[t], ct.son1[t]}) rsolve(L, son(bt, d, s2, s2), son(bt, x, t1, s2));
}

void lr(Lr& L, int32_t d) {
  h2_matrix* Z = L.Z;
  const BlockTree& bt = Z->blocks;
  const int32_t t = bt.row[d];
  if (bt.kind[d] == kNear) {
    Timer tm(L.t_lu);
    launch_leaf_lu(near_ptr(Z, d), (int)csize(Z, t), csize(Z, t), L.ctx->d_error, L.st);
    return;
  }
  const ClusterTree& ct = Z->rows;
  const int32_t t1 = ct.son0[t], t2 = ct.son1[t];
  const int32_t d11 = son(bt, d, t1, t1), d12 = son(bt, d, t1, t2);
  const int32_t d21 = son(bt, d, t2, t1), d22 = son(bt, d, t2, t2);
  lr(L, d11);
  lsolve(L, d11, d12);
  rsolve(L, d11, d21);
  mul(L, -1.0, d21, d12, d22);
  lr(L, d22);
}

// ------------------------------------------------ Cholesky (Section 7)
// A ~ L L^* for a symmetric positive definite matrix, the recursion of the
// LR with the lower factor's transpose in place of the upper factor: on a
// diagonal block L11 = chol(A11), L21 = A21 L11^-*, A22 <- A22 - L21 L21^*,
// L22 = chol(A22).  The factor is the lower triangle of the matrix; the
// strictly upper nearfield is never read.

// Y (#t x m) <- L|_{t x t}^-1 Y (lower with its diagonal)
void lsolve_dense_n(Lr& L, int32_t d, double* Y, int64_t ldy, int m) {
  const h2_matrix* Z = L.Z;
  const BlockTree& bt = Z->blocks;
  const int32_t t = bt.row[d];
  if (bt.kind[d] == kNear) {
    launch_trsm(3, near_ptr(Z, d), (int)csize(Z, t), csize(Z, t), Y, m, ldy, L.st);
    return;
  }
  const int32_t t1 = Z->rows.son0[t], t2 = Z->rows.son1[t];
  const int64_t n1 = csize(Z, t1);
  lsolve_dense_n(L, son(bt, d, t1, t1), Y, ldy, m);
  block_prod(L, L.Z, son(bt, d, t2, t1), 0, -1.0, Y, ldy, Y + n1, ldy, m);
  lsolve_dense_n(L, son(bt, d, t2, t2), Y + n1, ldy, m);
}

// Y (#t x m) <- L|_{t x t}^-* Y
void ltsolve_dense(Lr& L, int32_t d, double* Y, int64_t ldy, int m) {
  const h2_matrix* Z = L.Z;
  const BlockTree& bt = Z->blocks;
  const int32_t t = bt.row[d];
  if (bt.kind[d] == kNear) {
    launch_trsm(4, near_ptr(Z, d), (int)csize(Z, t), csize(Z, t), Y, m, ldy, L.st);
    return;
  }
  const int32_t t1 = Z->rows.son0[t], t2 = Z->rows.son1[t];
  const int64_t n1 = csize(Z, t1);
  ltsolve_dense(L, son(bt, d, t2, t2), Y + n1, ldy, m);
  block_prod(L, L.Z, son(bt, d, t2, t1), 1, -1.0, Y + n1, ldy, Y, ldy, m);
  ltsolve_dense(L, son(bt, d, t1, t1), Y, ldy, m);
}

// Z|_z += alpha Z|_x (Z|_yh)^*
void mul_t(Lr& L, double alpha, int32_t x, int32_t yh, int32_t z, bool lower) {
  struct Reset {
    Lr& L;
    ~Reset() {
      L.yt = false;
      L.lower = false;
    }
  } reset{L};
  L.yt = true;
  L.lower = lower;
  mul(L, alpha, x, yh, z);
}

// Z|_x <- Z|_x L|_{s x s}^-* in place, x = (t, s), d = (s, s)
void chol_rsolve(Lr& L, int32_t d, int32_t x) {
  h2_matrix* Z = L.Z;
  const BlockTree& bt = Z->blocks;
  const int32_t t = bt.row[x], s = bt.col[x];
  if (bt.kind[x] == kNear) {
    const int64_t mt = csize(Z, t), ms = csize(Z, s);
    Timer tm(L.t_solves);
    // (X L^-*)^* = L^-1 X^*
    DArr Yt(ms * mt, L.st);
    launch_transpose((int)mt, (int)ms, 1.0, near_ptr(Z, x), mt, Yt.p, ms, L.st);
    lsolve_dense_n(L, d, Yt.p, ms, (int)mt);
    launch_transpose((int)ms, (int)mt, 1.0, Yt.p, ms, near_ptr(Z, x), mt, L.st);
    return;
  }
  if (bt.kind[x] == kAdm) {
    const int kt = rank_of(Z, 0, t), ls = rank_of(Z, 1, s);
    if (ls == 0 || kt == 0) return;   // the block is zero
    const int64_t mt = csize(Z, t), ms = csize(Z, s);
    DArr Ws(ms * ls, L.st), Bh(ms * kt, L.st), Vt(mt * kt, L.st);
    {
      Timer tm(L.t_solves);
      expand(L, L.Z, 1, s, Ws.p, ms);
      launch_gemm((int)ms, kt, ls, 1.0, Ws.p, ms, 0, coupling_ptr(Z, x), Z->kcap, 1, 0.0, Bh.p, ms, L.st);
      lsolve_dense_n(L, d, Bh.p, ms, kt);   // L^-1 W_s S^*
      expand(L, L.Z, 0, t, Vt.p, mt);
    }
    engine_touch(L.eng, Z, x);   // a coupling written outside the update engine
    H2_CUDA(cudaMemsetAsync(coupling_ptr(Z, x), 0, (size_t)Z->kcap * Z->kcap * sizeof(double), L.st));
    apply_update(L, x, Vt.p, mt, Bh.p, ms, kt);
    return;
  }
  const ClusterTree& ct = Z->rows;
  const int32_t s1 = ct.son0[s], s2 = ct.son1[s];
  for (int32_t t1 : {ct.son0[t], ct.son1[t]}) chol_rsolve(L, son(bt, d, s1, s1), son(bt, x, t1, s1));
  for (int32_t t1 : {ct.son0[t], ct.son1[t]})
    mul_t(L, -1.0, son(bt, x, t1, s1), son(bt, d, s2, s1), son(bt, x, t1, s2), false);
  for (int32_t t1 : {ct.son0[t], ct.son1[t]}) chol_rsolve(L, son(bt, d, s2, s2), son(bt, x, t1, s2));
}

void chol(Lr& L, int32_t d) {
  h2_matrix* Z = L.Z;
  const BlockTree& bt = Z->blocks;
  const int32_t t = bt.row[d];
  if (bt.kind[d] == kNear) {
    Timer tm(L.t_lu);
    launch_leaf_chol(near_ptr(Z, d), (int)csize(Z, t), csize(Z, t), L.ctx->d_error, L.st);
    return;
  }
  const ClusterTree& ct = Z->rows;
  const int32_t t1 = ct.son0[t], t2 = ct.son1[t];
  const int32_t d11 = son(bt, d, t1, t1), d21 = son(bt, d, t2, t1), d22 = son(bt, d, t2, t2);
  chol(L, d11);
  chol_rsolve(L, d11, d21);
  mul_t(L, -1.0, d21, d21, d22, true);
  chol(L, d22);
}

// ---------------------------------------------- inversion (Remark on inversion)
// C|_d <- (A|_d)^-1 for a diagonal block d: a leaf by Doolittle's LU and two
// triangular solves with the identity; otherwise block Gauss elimination
// with the six products of the Remark, B12 = A11^-1 A12 and B21 = A21 A11^-1
// in T, the Schur complement S = A22 - A21 B12 in place of A22 (A is
// consumed).  C and T start as zero matrices on A's trees.
void product(Lr& L, h2_matrix* Z, const h2_matrix* X, const h2_matrix* Y, double alpha, int32_t x, int32_t y,
             int32_t z) {
  L.Z = Z;
  L.X = X == Z ? nullptr : X;
  L.Y = Y == Z ? nullptr : Y;
  mul(L, alpha, x, y, z);
}

void leaf_inverse(Lr& L, const h2_matrix* A, h2_matrix* C, int32_t d) {
  Timer tm(L.t_lu);
  const int64_t m = csize(A, A->blocks.row[d]);
  DArr F(m * m, L.st);
  H2_CUDA(cudaMemcpyAsync(F.p, near_ptr(A, d), m * m * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
  launch_leaf_lu(F.p, (int)m, m, L.ctx->d_error, L.st);
  double* X = near_ptr(C, d);
  launch_eye(X, (int)m, m, L.st);
  launch_trsm(0, F.p, (int)m, m, X, (int)m, m, L.st);   // L^-1
  launch_trsm(1, F.p, (int)m, m, X, (int)m, m, L.st);   // R^-1 L^-1
  H2_CUDA(cudaGetLastError());
}

void inv(Lr& L, h2_matrix* A, h2_matrix* C, h2_matrix* T, int32_t d) {
  const BlockTree& bt = A->blocks;
  if (bt.kind[d] == kNear) {
    leaf_inverse(L, A, C, d);
    return;
  }
  const ClusterTree& ct = A->rows;
  const int32_t t = bt.row[d];
  const int32_t t1 = ct.son0[t], t2 = ct.son1[t];
  const int32_t d11 = son(bt, d, t1, t1), d12 = son(bt, d, t1, t2);
  const int32_t d21 = son(bt, d, t2, t1), d22 = son(bt, d, t2, t2);
  inv(L, A, C, T, d11);                          // C11 = A11^-1
  product(L, T, C, A, 1.0, d11, d12, d12);       // B12 = A11^-1 A12
  product(L, T, A, C, 1.0, d21, d11, d21);       // B21 = A21 A11^-1
  product(L, A, A, T, -1.0, d21, d12, d22);      // S = A22 - A21 B12
  inv(L, A, C, T, d22);                          // C22 = S^-1
  product(L, C, T, C, -1.0, d12, d22, d12);      // C12 = -B12 C22
  product(L, C, C, T, -1.0, d22, d21, d21);      // C21 = -C22 B21
  product(L, C, C, T, -1.0, d12, d21, d11);      // C11 = C11 - C12 B21
}

void check_square(const h2_matrix* Z) {
  H2_REQUIRE(Z->rows.off == Z->cols.off && Z->rows.son0 == Z->cols.son0, "the matrix must be square with one tree");
  H2_REQUIRE(Z->blocks.kind[0] != kAdm, "the root block must not be admissible");
  H2_REQUIRE(Z->rows.max_leaf <= 64, "leaf clusters above 64 indices are not supported");
}

// ---------------------------------------------------------------- the FEM
// P1 stiffness matrix of -div(sigma grad u) on the unit square (cube) with
// u = 0 on the boundary (Section 7's model problem; sigma piecewise constant
// on an M^dim checkerboard, value at each element's centroid): every cell
// split into two triangles along its (i,j)-(i+1,j+1) diagonal (2D) or into
// Kuhn's six tetrahedra around its main diagonal (3D); the element matrix
// of a simplex e is sigma_e |e| G G^* with G the gradients of its
// barycentric coordinates, its entries below 1e-12 of its largest diagonal
// entry set to zero (their exact value); interior nodes numbered x fastest.
struct Csr {
  int64_t n = 0;
  std::vector<int64_t> ptr;
  std::vector<int64_t> col;
  std::vector<double> val;
};

Csr fem_stiffness(int dim, int64_t N, int64_t M, const double* sigma, std::vector<double>& points) {
  const double h = 1.0 / (double)N;
  const int64_t ni = N - 1;
  const int64_t n = dim == 2 ? ni * ni : ni * ni * ni;
  auto interior = [&](const int64_t* v) -> int64_t {
    for (int a = 0; a < dim; ++a)
      if (v[a] <= 0 || v[a] >= N) return -1;
    int64_t idx = 0, mul = 1;
    for (int a = 0; a < dim; ++a) {
      idx += (v[a] - 1) * mul;
      mul *= ni;
    }
    return idx;
  };
  // local vertex paths of the simplices of one cell
  std::vector<std::vector<std::array<int, 3>>> simp;
  if (dim == 2) {
    simp.push_back({{0, 0, 0}, {1, 0, 0}, {1, 1, 0}});
    simp.push_back({{0, 0, 0}, {1, 1, 0}, {0, 1, 0}});
  } else {
    int perm[3] = {0, 1, 2};
    do {
      std::vector<std::array<int, 3>> path{{0, 0, 0}};
      std::array<int, 3> v{0, 0, 0};
      for (int a = 0; a < 3; ++a) {
        v[perm[a]] += 1;
        path.push_back(v);
      }
      simp.push_back(path);
    } while (std::next_permutation(perm, perm + 3));
  }
  struct Trip {
    int64_t i, j;
    double v;
  };
  std::vector<Trip> trip;
  const int64_t ncell = dim == 2 ? N * N : N * N * N;
  trip.reserve((size_t)ncell * simp.size() * (dim + 1) * (dim + 1) / 2);
  for (int64_t cidx = 0; cidx < ncell; ++cidx) {
    int64_t cell[3] = {cidx % N, (cidx / N) % N, dim == 3 ? cidx / (N * N) : 0};
    for (const auto& path : simp) {
      double X[4][3];
      int64_t gl[4];
      for (int a = 0; a <= dim; ++a) {
        int64_t v[3];
        for (int q = 0; q < dim; ++q) {
          v[q] = cell[q] + path[a][q];
          X[a][q] = (double)v[q] * h;
        }
        gl[a] = interior(v);
      }
      // J (columns X_a - X_0), its inverse gives the gradients of lambda_1..dim
      double J[3][3] = {{0}}, Ji[3][3] = {{0}}, det = 0.0;
      for (int q = 0; q < dim; ++q)
        for (int a = 0; a < dim; ++a) J[q][a] = X[a + 1][q] - X[0][q];
      if (dim == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        Ji[0][0] = J[1][1] / det;
        Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det;
        Ji[1][1] = J[0][0] / det;
      } else {
        det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
              J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
      }
      const double vol = std::fabs(det) / (dim == 2 ? 2.0 : 6.0);
      // gradient of lambda_a (a >= 1) = row a-1 of J^-1; lambda_0 = -sum
      double G[4][3];
      for (int q = 0; q < dim; ++q) {
        double sum = 0.0;
        for (int a = 0; a < dim; ++a) {
          G[a + 1][q] = Ji[a][q];
          sum += Ji[a][q];
        }
        G[0][q] = -sum;
      }
      double xc[3] = {0, 0, 0};
      for (int a = 0; a <= dim; ++a)
        for (int q = 0; q < dim; ++q) xc[q] += X[a][q];
      int64_t flat = 0, mulp = 1;
      for (int q = 0; q < dim; ++q) {
        int64_t ix = (int64_t)std::floor((double)M * (xc[q] / (dim + 1)));
        ix = std::min(std::max<int64_t>(ix, 0), M - 1);
        flat += ix * mulp;
        mulp *= M;
      }
      const double sg = sigma[flat] * vol;
      double Ke[4][4], dmax = 0.0;
      for (int a = 0; a <= dim; ++a)
        for (int c = 0; c <= dim; ++c) {
          double g = 0.0;
          for (int q = 0; q < dim; ++q) g += G[a][q] * G[c][q];
          Ke[a][c] = sg * g;
          if (a == c) dmax = std::max(dmax, std::fabs(Ke[a][a]));
        }
      for (int a = 0; a <= dim; ++a) {
        if (gl[a] < 0) continue;
        for (int c = 0; c <= dim; ++c) {
          if (gl[c] < 0) continue;
          // an entry whose exact value is zero (orthogonal gradients: the
          // edge opposite a right angle) carries only the rounding of the
          // gradients; it is zero
          const double v = std::fabs(Ke[a][c]) <= 1e-12 * dmax ? 0.0 : Ke[a][c];
          trip.push_back({gl[a], gl[c], v});
        }
      }
    }
  }
  std::stable_sort(trip.begin(), trip.end(),
                   [](const Trip& a, const Trip& b) { return a.i != b.i ? a.i < b.i : a.j < b.j; });
  Csr A;
  A.n = n;
  A.ptr.assign(n + 1, 0);
  for (size_t k = 0; k < trip.size();) {
    size_t e = k;
    double v = 0.0;
    while (e < trip.size() && trip[e].i == trip[k].i && trip[e].j == trip[k].j) v += trip[e++].v;
    A.col.push_back(trip[k].j);
    A.val.push_back(v);
    A.ptr[trip[k].i + 1] += 1;
    k = e;
  }
  for (int64_t i = 0; i < n; ++i) A.ptr[i + 1] += A.ptr[i];
  points.assign((size_t)n * dim, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    int64_t r = i;
    for (int a = 0; a < dim; ++a) {
      points[(size_t)i * dim + a] = (double)(r % ni + 1) * h;
      r /= ni;
    }
  }
  return A;
}

}  // namespace

// =================================================================== C ABI
namespace {
void check_options(const h2_options* opt) {
  H2_REQUIRE(opt, "options missing");
  H2_REQUIRE(std::isfinite(opt->eps) && opt->eps >= 0, "eps must be finite and >= 0");
  H2_REQUIRE(opt->precision == H2_FP64, "only H2_FP64 is built");
  H2_REQUIRE(opt->trunc_norm == 0 && opt->weighting == 0, "trunc_norm and weighting must be 0");
  // a basis of rank max_rank must leave room for one more column in the
  // 32-column extended basis of the next update
  H2_REQUIRE(opt->max_rank >= 0 && opt->max_rank <= 31, "max_rank must be in 0..31");
}
}  // namespace

extern "C" h2_status h2_build_fem(h2_ctx* ctx, int dim, int64_t cells, int64_t checker, const double* sigma,
                                  const h2_options* opt, h2_matrix** out) {
  if (!ctx || !out || !sigma || !opt) return H2_EINVAL;
  *out = nullptr;
  h2_matrix* Z = nullptr;
  const int leaf_size = opt->leaf_size;
  const double eta = opt->eta;
  h2_status s = lr_guard(ctx, [&] {
    H2_REQUIRE(dim == 2 || dim == 3, "h2_build_fem: dim must be 2 or 3");
    H2_REQUIRE(cells >= 2 && checker >= 1 && leaf_size >= 1 && eta > 0, "h2_build_fem: bad sizes");
    int64_t ms = 1;
    for (int a = 0; a < dim; ++a) ms *= checker;
    for (int64_t i = 0; i < ms; ++i) H2_REQUIRE(std::isfinite(sigma[i]) && sigma[i] > 0, "sigma must be positive");
    std::vector<double> pts;
    Csr A = fem_stiffness(dim, cells, checker, sigma, pts);
    // support boxes: node boxes padded by h per side
    h2_status st = h2_matrix_create(ctx, pts.data(), A.n, dim, leaf_size, eta, 1.0 / (double)cells, 16, &Z);
    if (st != H2_OK) throw Error(st, ctx->last_error);
    const ClusterTree& ct = Z->rows;
    const BlockTree& bt = Z->blocks;
    std::vector<int64_t> pos(A.n);
    for (int64_t p = 0; p < A.n; ++p) pos[ct.perm[p]] = p;
    std::vector<double> near(Z->near_len, 0.0);
    for (int64_t i = 0; i < A.n; ++i)
      for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
        const int64_t pi = pos[i], pj = pos[A.col[e]];
        int32_t b = 0;
        while (bt.kind[b] == kSub) {
          int32_t next = -1;
          for (int k = 0; k < 4 && next < 0; ++k) {
            const int32_t c = bt.son4[4 * b + k];
            if (c < 0) continue;
            const int32_t t = bt.row[c], q = bt.col[c];
            if (pi >= ct.off[t] && pi < ct.off[t] + ct.size[t] && pj >= ct.off[q] && pj < ct.off[q] + ct.size[q])
              next = c;
          }
          b = next;
        }
        if (bt.kind[b] == kAdm) {
          if (A.val[e] != 0.0) throw Error(H2_EINTERNAL, "h2_build_fem: nonzero in an admissible block");
          continue;
        }
        const int32_t t = bt.row[b], q = bt.col[b];
        near[Z->near_off[bt.slot[b]] + (pi - ct.off[t]) + (pj - ct.off[q]) * ct.size[t]] = A.val[e];
      }
    st = h2_set_nearfield(ctx, Z, near.data());
    if (st != H2_OK) throw Error(st, ctx->last_error);
  });
  if (s == H2_OK) {
    *out = Z;
  } else if (Z) {
    h2_matrix_free(Z);
  }
  return s;
}

extern "C" h2_status h2_lr_factor(h2_ctx* ctx, h2_matrix* Z, const h2_options* opt, int64_t* stats) {
  if (!ctx || !Z || !opt) return H2_EINVAL;
  return lr_guard(ctx, [&] {
    check_options(opt);
    const double eps = opt->eps;
    check_square(Z);
    DevGuard g(ctx->device);
    Lr L;
    L.ctx = ctx;
    L.Z = Z;
    L.eps = eps;
    L.max_rank = opt->max_rank;
    L.st = ctx->stream;
    lr(L, 0);
    H2_CUDA(cudaStreamSynchronize(L.st));
    h2_status s = h2_ctx_synchronize(ctx);
    if (s != H2_OK) throw Error(s, ctx->last_error);
    if (stats) {
      stats[0] = L.updates;
      stats[1] = L.products;
      int kmax = 0;
      for (int32_t r : Z->V.rank) kmax = std::max(kmax, r);
      for (int32_t r : Z->W.rank) kmax = std::max(kmax, r);
      stats[2] = kmax;
      // microseconds of wall time by activity
      stats[3] = (int64_t)(1e6 * L.t_update);
      stats[4] = (int64_t)(1e6 * L.t_terms);
      stats[5] = (int64_t)(1e6 * L.t_temps);
      stats[6] = (int64_t)(1e6 * L.t_solves);
      stats[7] = (int64_t)(1e6 * L.t_lu);
      double pl, la, wa, to;
      engine_times(L.eng, &pl, &la, &wa, &to);
      stats[8] = (int64_t)(1e6 * pl);
      stats[9] = (int64_t)(1e6 * la);
      stats[10] = (int64_t)(1e6 * wa);
      stats[11] = (int64_t)(1e6 * to);
      stats[12] = (int64_t)(1e6 * L.t_temp_wait);
      stats[13] = L.n_temps;
      stats[14] = L.temp_cols;
    }
  });
}

extern "C" h2_status h2_chol_factor(h2_ctx* ctx, h2_matrix* Z, const h2_options* opt, int64_t* stats) {
  if (!ctx || !Z || !opt) return H2_EINVAL;
  return lr_guard(ctx, [&] {
    check_options(opt);
    check_square(Z);
    DevGuard g(ctx->device);
    Lr L;
    L.ctx = ctx;
    L.Z = Z;
    L.eps = opt->eps;
    L.max_rank = opt->max_rank;
    L.st = ctx->stream;
    chol(L, 0);
    H2_CUDA(cudaStreamSynchronize(L.st));
    h2_status s = h2_ctx_synchronize(ctx);
    if (s != H2_OK) throw Error(s, ctx->last_error);
    if (stats) {
      stats[0] = L.updates;
      stats[1] = L.products;
      int kmax = 0;
      for (int32_t r : Z->V.rank) kmax = std::max(kmax, r);
      for (int32_t r : Z->W.rank) kmax = std::max(kmax, r);
      stats[2] = kmax;
    }
  });
}

extern "C" h2_status h2_chol_solve(h2_ctx* ctx, const h2_matrix* F, int64_t nrhs, double* X, int64_t ldx) {
  if (!ctx || !F || nrhs < 0 || (nrhs > 0 && !X)) return H2_EINVAL;
  return lr_guard(ctx, [&] {
    H2_REQUIRE(ldx >= F->rows.n, "h2_chol_solve: leading dimension too small");
    check_square(F);
    if (nrhs == 0) return;
    DevGuard g(ctx->device);
    Lr L;
    L.ctx = ctx;
    L.Z = const_cast<h2_matrix*>(F);   // read only: solves never modify the factor
    L.st = ctx->stream;
    lsolve_dense_n(L, 0, X, ldx, (int)nrhs);
    ltsolve_dense(L, 0, X, ldx, (int)nrhs);
    H2_CUDA(cudaGetLastError());
    H2_CUDA(cudaStreamSynchronize(L.st));
  });
}

extern "C" h2_status h2_inverse(h2_ctx* ctx, h2_matrix* A, const h2_options* opt, h2_matrix** out,
                                int64_t* stats) {
  if (!ctx || !A || !opt || !out) return H2_EINVAL;
  *out = nullptr;
  h2_matrix* C = nullptr;
  h2_matrix* T = nullptr;
  h2_status st = lr_guard(ctx, [&] {
    check_options(opt);
    check_square(A);
    DevGuard g(ctx->device);
    h2_status s = h2_matrix_clone(ctx, A, &C);
    if (s != H2_OK) throw Error(s, ctx->last_error);
    s = h2_matrix_clone(ctx, A, &T);
    if (s != H2_OK) throw Error(s, ctx->last_error);
    zero_matrix(ctx, C);
    zero_matrix(ctx, T);
    Lr L;
    L.ctx = ctx;
    L.Z = A;
    L.eps = opt->eps;
    L.max_rank = opt->max_rank;
    L.st = ctx->stream;
    inv(L, A, C, T, 0);
    H2_CUDA(cudaStreamSynchronize(L.st));
    s = h2_ctx_synchronize(ctx);
    if (s != H2_OK) throw Error(s, ctx->last_error);
    if (stats) {
      stats[0] = L.updates;
      stats[1] = L.products;
      int kmax = 0;
      for (int32_t r : C->V.rank) kmax = std::max(kmax, r);
      for (int32_t r : C->W.rank) kmax = std::max(kmax, r);
      stats[2] = kmax;
    }
  });
  h2_matrix_free(T);
  if (st == H2_OK) {
    *out = C;
  } else {
    h2_matrix_free(C);
  }
  return st;
}

namespace {
// count independent factorisations side by side: `threads` host threads,
// each with a stream and context of its own, take the matrices in turn
using FactorFn = h2_status (*)(h2_ctx*, h2_matrix*, const h2_options*, int64_t*);
void factor_many(h2_ctx* ctx, h2_matrix* const* Z, int64_t count, const h2_options* opt, int threads,
                 int64_t* stats, const char* name, FactorFn factor) {
  check_options(opt);
  for (int64_t i = 0; i < count; ++i) {
    H2_REQUIRE(Z[i] != nullptr, std::string(name) + ": matrix missing");
    H2_REQUIRE(Z[i]->device == ctx->device, std::string(name) + ": matrix on another device");
    check_square(Z[i]);
    for (int64_t j = 0; j < i; ++j) H2_REQUIRE(Z[j] != Z[i], std::string(name) + ": a matrix appears twice");
  }
  if (count == 0) return;
  DevGuard g(ctx->device);
  H2_CUDA(cudaStreamSynchronize(ctx->stream));   // the matrices are ready
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int64_t nt = std::min<int64_t>(count, threads > 0 ? threads : hw);
  std::atomic<int64_t> next{0};
  std::vector<h2_status> st(count, H2_OK);
  std::vector<std::string> msg(count);
  const int device = ctx->device;
  // one host thread per stream and context: the factorisations' launches
  // are few tasks each (the recursion applies one update at a time), so
  // independent problems side by side fill the GPU
  auto worker = [&]() {
    cudaStream_t s = nullptr;
    h2_ctx* c = nullptr;
    h2_status cs = cudaSetDevice(device) == cudaSuccess &&
                           cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess
                       ? h2_ctx_create(device, s, &c)
                       : H2_ECUDA;
    for (;;) {
      const int64_t i = next.fetch_add(1);
      if (i >= count) break;
      if (cs != H2_OK) {
        st[i] = cs;
        msg[i] = std::string(name) + ": no stream or context for a worker";
        continue;
      }
      int64_t one[15] = {};
      st[i] = factor(c, Z[i], opt, one);
      if (st[i] != H2_OK) {
        const char* m = h2_last_error(c);
        msg[i] = m ? m : "";
      } else if (stats) {
        for (int k = 0; k < 3; ++k) stats[3 * i + k] = one[k];
      }
    }
    if (c) h2_ctx_destroy(c);
    if (s) cudaStreamDestroy(s);
  };
  std::vector<std::thread> pool;
  for (int64_t t = 0; t < nt; ++t) pool.emplace_back(worker);
  for (std::thread& t : pool) t.join();
  for (int64_t i = 0; i < count; ++i)
    if (st[i] != H2_OK) throw Error(st[i], "matrix " + std::to_string(i) + ": " + msg[i]);
}
}  // namespace

extern "C" h2_status h2_lr_factor_many(h2_ctx* ctx, h2_matrix* const* Z, int64_t count, const h2_options* opt,
                                       int threads, int64_t* stats) {
  if (!ctx || count < 0 || (count > 0 && !Z) || !opt || threads < 0) return H2_EINVAL;
  return lr_guard(ctx, [&] { factor_many(ctx, Z, count, opt, threads, stats, "h2_lr_factor_many", h2_lr_factor); });
}

extern "C" h2_status h2_chol_factor_many(h2_ctx* ctx, h2_matrix* const* Z, int64_t count, const h2_options* opt,
                                         int threads, int64_t* stats) {
  if (!ctx || count < 0 || (count > 0 && !Z) || !opt || threads < 0) return H2_EINVAL;
  return lr_guard(ctx,
                  [&] { factor_many(ctx, Z, count, opt, threads, stats, "h2_chol_factor_many", h2_chol_factor); });
}

extern "C" h2_status h2_lr_solve(h2_ctx* ctx, const h2_matrix* LR, int64_t nrhs, double* X, int64_t ldx) {
  if (!ctx || !LR || nrhs < 0 || (nrhs > 0 && !X)) return H2_EINVAL;
  return lr_guard(ctx, [&] {
    H2_REQUIRE(ldx >= LR->rows.n, "h2_lr_solve: leading dimension too small");
    check_square(LR);
    if (nrhs == 0) return;
    DevGuard g(ctx->device);
    Lr L;
    L.ctx = ctx;
    L.Z = const_cast<h2_matrix*>(LR);   // read only: solves never modify the factor
    L.st = ctx->stream;
    lsolve_dense(L, 0, X, ldx, (int)nrhs);
    usolve_dense(L, 0, X, ldx, (int)nrhs);
    H2_CUDA(cudaGetLastError());
    H2_CUDA(cudaStreamSynchronize(L.st));
  });
}

namespace {
// Preconditioned conjugate gradients from x = 0 (Section 7), the
// preconditioner given as precond(in, out) on device vectors.
template <class Precond>
void pcg_run(h2_ctx* ctx, const h2_matrix* A, Precond&& precond, const double* b, double* x, double tol, int maxit,
             int* iterations, double* relres, DArr& z) {
  const int64_t n = A->rows.n;
  cudaStream_t st = ctx->stream;
  DArr r(n, st), p(n, st), q(n, st), part(kDotBlocks, st), sc(4, st);
  auto dot = [&](const double* u, const double* v) {
    launch_dot(u, v, n, part.p, sc.p, st);
    double h = 0.0;
    H2_CUDA(cudaMemcpyAsync(&h, sc.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    H2_CUDA(cudaStreamSynchronize(st));
    return h;
  };
  zero(x, n, st);
  H2_CUDA(cudaMemcpyAsync(r.p, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const double nb = std::sqrt(dot(b, b));
  int it = 0;
  double res = nb > 0 ? 1.0 : 0.0;
  if (nb > 0) {
    precond(r.p, z.p);
    H2_CUDA(cudaMemcpyAsync(p.p, z.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    double rz = dot(r.p, z.p);
    for (it = 1; it <= maxit; ++it) {
      h2_status s = h2_matvec(ctx, A, 1, 1.0, p.p, n, 0.0, q.p, n);
      if (s != H2_OK) throw Error(s, ctx->last_error);
      const double alpha = rz / dot(p.p, q.p);
      launch_axpby(n, alpha, p.p, 1.0, x, st);
      launch_axpby(n, -alpha, q.p, 1.0, r.p, st);
      res = std::sqrt(dot(r.p, r.p)) / nb;
      if (res <= tol) break;
      precond(r.p, z.p);
      const double rz2 = dot(r.p, z.p);
      launch_axpby(n, 1.0, z.p, rz2 / rz, p.p, st);
      rz = rz2;
    }
    if (it > maxit) it = maxit;
  }
  H2_CUDA(cudaStreamSynchronize(st));
  if (iterations) *iterations = it;
  if (relres) *relres = res;
}
}  // namespace

extern "C" h2_status h2_pcg(h2_ctx* ctx, const h2_matrix* A, const h2_matrix* LR, const double* b, double* x,
                            double tol, int maxit, int* iterations, double* relres) {
  if (!ctx || !A || !b || !x || maxit < 0) return H2_EINVAL;
  return lr_guard(ctx, [&] {
    const int64_t n = A->rows.n;
    DevGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    DArr z(n, st);
    auto precond = [&](const double* in, double* out) {
      H2_CUDA(cudaMemcpyAsync(out, in, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      if (LR) {
        h2_status s = h2_lr_solve(ctx, LR, 1, out, n);
        if (s != H2_OK) throw Error(s, ctx->last_error);
      }
    };
    pcg_run(ctx, A, precond, b, x, tol, maxit, iterations, relres, z);
  });
}

extern "C" h2_status h2_pcg_chol(h2_ctx* ctx, const h2_matrix* A, const h2_matrix* F, const double* b, double* x,
                                 double tol, int maxit, int* iterations, double* relres) {
  if (!ctx || !A || !F || !b || !x || maxit < 0) return H2_EINVAL;
  return lr_guard(ctx, [&] {
    const int64_t n = A->rows.n;
    H2_REQUIRE(F->rows.n == n && F->cols.n == n, "h2_pcg_chol: the factor has another size");
    DevGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    DArr z(n, st);
    auto precond = [&](const double* in, double* out) {
      H2_CUDA(cudaMemcpyAsync(out, in, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      h2_status s = h2_chol_solve(ctx, F, 1, out, n);
      if (s != H2_OK) throw Error(s, ctx->last_error);
    };
    pcg_run(ctx, A, precond, b, x, tol, maxit, iterations, relres, z);
  });
}

extern "C" h2_status h2_pcg_inverse(h2_ctx* ctx, const h2_matrix* A, const h2_matrix* Cinv, const double* b,
                                    double* x, double tol, int maxit, int* iterations, double* relres) {
  if (!ctx || !A || !Cinv || !b || !x || maxit < 0) return H2_EINVAL;
  return lr_guard(ctx, [&] {
    const int64_t n = A->rows.n;
    H2_REQUIRE(Cinv->rows.n == n && Cinv->cols.n == n, "h2_pcg_inverse: the inverse has another size");
    DevGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    DArr z(n, st);
    auto precond = [&](const double* in, double* out) {
      h2_status s = h2_matvec(ctx, Cinv, 1, 1.0, in, n, 0.0, out, n);
      if (s != H2_OK) throw Error(s, ctx->last_error);
    };
    pcg_run(ctx, A, precond, b, x, tol, maxit, iterations, relres, z);
  });
}

namespace {
// ||I - P A||_2 by the power iteration, P = solve(in place) (Section 7,
// column Err): iters steps v <- w / ||w||, w = v - P A v
template <class Solve>
double power_error(h2_ctx* ctx, const h2_matrix* A, Solve&& solve, double* v, int iters) {
  const int64_t n = A->rows.n;
  cudaStream_t st = ctx->stream;
  DArr w(n, st), part(kDotBlocks, st), sc(1, st);
  auto norm = [&](const double* u) {
    launch_dot(u, u, n, part.p, sc.p, st);
    double h = 0.0;
    H2_CUDA(cudaMemcpyAsync(&h, sc.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    H2_CUDA(cudaStreamSynchronize(st));
    return std::sqrt(h);
  };
  double nv = norm(v);
  H2_REQUIRE(nv > 0, "power iteration: zero start vector");
  launch_axpby(n, 1.0 / nv, v, 0.0, v, st);
  double lam = 0.0;
  for (int k = 0; k < iters; ++k) {
    h2_status s = h2_matvec(ctx, A, 1, 1.0, v, n, 0.0, w.p, n);
    if (s != H2_OK) throw Error(s, ctx->last_error);
    solve(w.p);
    launch_axpby(n, 1.0, v, -1.0, w.p, st);
    lam = norm(w.p);
    if (lam == 0.0) break;
    launch_axpby(n, 1.0 / lam, w.p, 0.0, v, st);
  }
  H2_CUDA(cudaStreamSynchronize(st));
  return lam;
}
}  // namespace

extern "C" h2_status h2_lr_error(h2_ctx* ctx, const h2_matrix* A, const h2_matrix* LR, double* v, int iters,
                                 double* err) {
  if (!ctx || !A || !LR || !v || iters < 1 || !err) return H2_EINVAL;
  return lr_guard(ctx, [&] {
    DevGuard g(ctx->device);
    const int64_t n = A->rows.n;
    *err = power_error(ctx, A, [&](double* w) {
      h2_status s = h2_lr_solve(ctx, LR, 1, w, n);
      if (s != H2_OK) throw Error(s, ctx->last_error);
    }, v, iters);
  });
}

extern "C" h2_status h2_chol_error(h2_ctx* ctx, const h2_matrix* A, const h2_matrix* F, double* v, int iters,
                                   double* err) {
  if (!ctx || !A || !F || !v || iters < 1 || !err) return H2_EINVAL;
  return lr_guard(ctx, [&] {
    DevGuard g(ctx->device);
    const int64_t n = A->rows.n;
    *err = power_error(ctx, A, [&](double* w) {
      h2_status s = h2_chol_solve(ctx, F, 1, w, n);
      if (s != H2_OK) throw Error(s, ctx->last_error);
    }, v, iters);
  });
}

extern "C" h2_status h2_mul(h2_ctx* ctx, double alpha, const h2_matrix* X, int64_t bx, const h2_matrix* Y,
                            int64_t by, h2_matrix* Z, int64_t bz, double eps, int64_t* updates) {
  if (!ctx || !X || !Y || !Z) return H2_EINVAL;
  return lr_guard(ctx, [&] {
    H2_REQUIRE(std::isfinite(eps) && eps >= 0 && std::isfinite(alpha), "h2_mul: eps and alpha must be finite");
    check_square(Z);
    const BlockTree& bt = Z->blocks;
    for (const h2_matrix* M : {X, Y})
      H2_REQUIRE(M->rows.off == Z->rows.off && M->rows.son0 == Z->rows.son0 && M->blocks.row == bt.row &&
                     M->blocks.col == bt.col && M->blocks.kind == bt.kind && M->device == Z->device &&
                     M->d_row_off != nullptr,
                 "h2_mul: X and Y must have Z's cluster tree, block tree and device");
    const int64_t nb = bt.count();
    H2_REQUIRE(bx >= 0 && bx < nb && by >= 0 && by < nb && bz >= 0 && bz < nb, "h2_mul: block out of range");
    H2_REQUIRE(bt.row[bx] == bt.row[bz] && bt.col[bx] == bt.row[by] && bt.col[by] == bt.col[bz],
               "h2_mul: blocks must be (t,s), (s,r), (t,r)");
    DevGuard g(ctx->device);
    Lr L;
    L.ctx = ctx;
    L.Z = Z;
    L.X = X == Z ? nullptr : X;
    L.Y = Y == Z ? nullptr : Y;
    L.eps = eps;
    L.st = ctx->stream;
    mul(L, alpha, (int32_t)bx, (int32_t)by, (int32_t)bz);
    H2_CUDA(cudaStreamSynchronize(L.st));
    h2_status s = h2_ctx_synchronize(ctx);
    if (s != H2_OK) throw Error(s, ctx->last_error);
    if (updates) *updates = L.updates;
  });
}
