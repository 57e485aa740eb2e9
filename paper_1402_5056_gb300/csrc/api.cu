// C ABI of libh2gb: contexts, H^2 storage, the batch planner and the
// execution of local low-rank updates (Sections 2, 4 and 5).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <unordered_map>

#include "h2_internal.h"
#include "matvec.h"
#include "update_kernels.h"

using namespace h2;

// ===================================================================== misc
namespace {
// allocations left before the hook fails one (0: the hook is off)
std::atomic<int64_t> g_fail_countdown{0};

bool hook_fires() {
  int64_t c = g_fail_countdown.load(std::memory_order_relaxed);
  while (c > 0)
    if (g_fail_countdown.compare_exchange_weak(c, c - 1, std::memory_order_relaxed)) return c == 1;
  return false;
}
}  // namespace

void* h2::device_alloc(size_t bytes) {
  if (bytes == 0) return nullptr;
  if (hook_fires()) throw Error(H2_ENOMEM, "device allocation failed (failure hook)");
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    throw Error(H2_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return p;
}

void* h2::device_alloc_async(size_t bytes, cudaStream_t st) {
  if (bytes == 0) return nullptr;
  if (hook_fires()) throw Error(H2_ENOMEM, "device allocation failed (failure hook)");
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, st);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    throw Error(H2_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  }
  return p;
}

extern "C" h2_status h2_debug_fail_allocation(int64_t n) {
  if (n < 0) return H2_EINVAL;
  g_fail_countdown.store(n, std::memory_order_relaxed);
  return H2_OK;
}

namespace {

thread_local std::string g_null_ctx_error;

template <typename T>
T* dalloc(size_t count) {
  if (count == 0) return nullptr;
  return static_cast<T*>(device_alloc(count * sizeof(T)));
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <typename T>
T* upload(const std::vector<T>& v, cudaStream_t st) {
  T* d = dalloc<T>(v.size());
  if (!v.empty()) {
    cudaError_t e = cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      dfree(d);
      H2_CUDA(e);
    }
  }
  return d;
}

template <typename F>
h2_status guard(h2_ctx* ctx, F&& f) {
  try {
    f();
    return H2_OK;
  } catch (const Error& e) {
    if (ctx) ctx->last_error = e.what(); else g_null_ctx_error = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->last_error = "host allocation failed"; else g_null_ctx_error = "host allocation failed";
    return H2_ENOMEM;
  } catch (const std::exception& e) {
    if (ctx) ctx->last_error = e.what(); else g_null_ctx_error = e.what();
    return H2_EINTERNAL;
  }
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) H2_CUDA(cudaSetDevice(dev));
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

const ClusterTree& tree_of(const h2_matrix* Z, int side) { return side == 0 ? Z->rows : Z->cols; }
DeviceBasis& basis_of(h2_matrix* Z, int side) { return side == 0 ? Z->V : Z->W; }
const DeviceBasis& basis_of(const h2_matrix* Z, int side) { return side == 0 ? Z->V : Z->W; }

bool has_storage(const h2_matrix* Z) { return Z->d_S != nullptr || Z->blocks.adm.empty(); }

void free_basis(DeviceBasis& b) {
  dfree(b.d_rank);
  dfree(b.d_leaf);
  dfree(b.d_transfer);
  dfree(b.d_leaf_off);
}

// Allocate basis storage for capacity kcap, zero-filled.
void alloc_basis(const ClusterTree& ct, int kcap, DeviceBasis& b, cudaStream_t st) {
  const int32_t nc = ct.count();
  b.leaf_off.assign(nc, -1);
  int64_t tot = 0;
  for (int32_t c = 0; c < nc; ++c)
    if (ct.leaf(c)) {
      b.leaf_off[c] = tot;
      tot += ct.size[c] * kcap;
    }
  b.d_leaf = dalloc<double>(tot);
  b.d_transfer = dalloc<double>((size_t)nc * kcap * kcap);
  H2_CUDA(cudaMemsetAsync(b.d_leaf, 0, tot * sizeof(double), st));
  H2_CUDA(cudaMemsetAsync(b.d_transfer, 0, (size_t)nc * kcap * kcap * sizeof(double), st));
  b.d_leaf_off = upload(b.leaf_off, st);
  if (b.rank.size() != (size_t)nc) b.rank.assign(nc, 0);
  b.d_rank = upload(b.rank, st);
}

void sync_ranks(DeviceBasis& b, cudaStream_t st) {
  H2_CUDA(cudaMemcpyAsync(b.d_rank, b.rank.data(), b.rank.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice, st));
}

MatView view_of(const h2_matrix* Z) {
  MatView M;
  for (int s = 0; s < 2; ++s) {
    const DeviceBasis& b = basis_of(Z, s);
    M.leaf[s] = b.d_leaf;
    M.transfer[s] = b.d_transfer;
    M.leaf_off[s] = b.d_leaf_off;
    M.rank[s] = b.d_rank;
  }
  M.father[0] = Z->d_father_r;
  M.father[1] = Z->d_father_c;
  M.subtree[0] = Z->d_subtree_r;
  M.subtree[1] = Z->d_subtree_c;
  M.size[0] = Z->d_row_size;
  M.size[1] = Z->d_col_size;
  M.S = Z->d_S;
  M.kcap = Z->kcap;
  return M;
}

// Re-layout the storage of Z for a larger rank capacity (device copies).
void grow_kcap(h2_ctx* ctx, h2_matrix* Z, int kcap) {
  if (kcap <= Z->kcap) return;
  H2_REQUIRE(kcap <= kMaxCols, "rank capacity above 32");
  cudaStream_t st = ctx->stream;
  std::vector<CopyDesc> cd;
  DeviceBasis nb[2];
  double* nS = nullptr;
  CopyDesc* dcd = nullptr;
  try {
  for (int s = 0; s < 2; ++s) {
    const ClusterTree& ct = tree_of(Z, s);
    DeviceBasis& ob = basis_of(Z, s);
    nb[s].rank = ob.rank;
    alloc_basis(ct, kcap, nb[s], st);
    for (int32_t c = 0; c < ct.count(); ++c) {
      if (ct.leaf(c) && ob.rank[c] > 0)
        cd.push_back({ob.d_leaf + ob.leaf_off[c], nb[s].d_leaf + nb[s].leaf_off[c], (int)ct.size[c],
                      ob.rank[c], (int)ct.size[c], (int)ct.size[c]});
      if (ct.father[c] >= 0 && ob.rank[c] > 0 && ob.rank[ct.father[c]] > 0)
        cd.push_back({ob.d_transfer + (size_t)c * Z->kcap * Z->kcap,
                      nb[s].d_transfer + (size_t)c * kcap * kcap, ob.rank[c], ob.rank[ct.father[c]],
                      Z->kcap, kcap});
    }
  }
  const size_t nadm = Z->blocks.adm.size();
  nS = dalloc<double>(nadm * kcap * kcap);
  H2_CUDA(cudaMemsetAsync(nS, 0, nadm * kcap * kcap * sizeof(double), st));
  for (size_t a = 0; a < nadm; ++a) {
    const int32_t b = Z->blocks.adm[a];
    const int kt = Z->V.rank[Z->blocks.row[b]], ls = Z->W.rank[Z->blocks.col[b]];
    if (kt > 0 && ls > 0)
      cd.push_back({Z->d_S + a * Z->kcap * Z->kcap, nS + a * kcap * kcap, kt, ls, Z->kcap, kcap});
  }
  dcd = upload(cd, st);
  launch_copy(dcd, (int)cd.size(), st);
  H2_CUDA(cudaGetLastError());
  H2_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    // Z keeps its storage; nothing of the new layout survives
    (void)cudaStreamSynchronize(st);
    free_basis(nb[0]);
    free_basis(nb[1]);
    dfree(nS);
    dfree(dcd);
    throw;
  }
  dfree(dcd);
  for (int s = 0; s < 2; ++s) {
    free_basis(basis_of(Z, s));
    basis_of(Z, s) = nb[s];
  }
  dfree(Z->d_S);
  Z->d_S = nS;
  Z->kcap = kcap;
}

}  // namespace

// =================================================================== context
extern "C" h2_status h2_ctx_create(int device, void* cuda_stream, h2_ctx** out) {
  if (!out) return H2_EINVAL;
  *out = nullptr;
  auto ctx = std::make_unique<h2_ctx>();
  h2_status s = guard(nullptr, [&] {
    int n = 0;
    H2_CUDA(cudaGetDeviceCount(&n));
    H2_REQUIRE(device >= 0 && device < n, "h2_ctx_create: no such device");
    ctx->device = device;
    DeviceGuard g(device);
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    ctx->d_error = dalloc<int>(1);
    H2_CUDA(cudaMemset(ctx->d_error, 0, sizeof(int)));
  });
  if (s == H2_OK) *out = ctx.release();
  return s;
}

extern "C" void h2_ctx_destroy(h2_ctx* ctx) {
  if (!ctx) return;
  if (ctx->d_error) cudaFree(ctx->d_error);
  delete ctx;
}

extern "C" const char* h2_last_error(const h2_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : g_null_ctx_error.c_str();
}

static void check_device_error(h2_ctx* ctx) {
  int e = 0;
  H2_CUDA(cudaMemcpyAsync(&e, ctx->d_error, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  H2_CUDA(cudaStreamSynchronize(ctx->stream));
  if (e) {
    H2_CUDA(cudaMemsetAsync(ctx->d_error, 0, sizeof(int), ctx->stream));
    std::string m = "device reported:";
    if (e & kErrRows) m += " matrix taller than the kernel tile;";
    if (e & kErrCols) m += " more than 32 columns (k + u > 32);";
    if (e & kErrJacobi) m += " one-sided Jacobi did not converge;";
    if (e & kErrRank) m += " inconsistent ranks;";
    if (e & kErrPivot) m += " zero pivot in a leaf LU;";
    if (e & kErrDefinite) m += " pivot not positive in a leaf Cholesky (matrix not positive definite);";
    throw Error(H2_EDEVICE, m);
  }
}

extern "C" h2_status h2_ctx_synchronize(h2_ctx* ctx) {
  if (!ctx) return H2_EINVAL;
  return guard(ctx, [&] {
    DeviceGuard g(ctx->device);
    H2_CUDA(cudaStreamSynchronize(ctx->stream));
    H2_CUDA(cudaGetLastError());
    check_device_error(ctx);
  });
}

// ==================================================================== matrix
extern "C" h2_status h2_matrix_create(h2_ctx* ctx, const double* points, int64_t n, int dim,
                                      int leaf_size, double eta, double pad, int kcap,
                                      h2_matrix** out) {
  if (!out) return H2_EINVAL;
  *out = nullptr;
  auto Z = std::make_unique<h2_matrix>();
  h2_status s = guard(ctx, [&] {
    H2_REQUIRE(points && n > 0 && dim >= 1 && dim <= 3, "h2_matrix_create: bad points");
    H2_REQUIRE(leaf_size >= 1 && eta > 0 && pad >= 0, "h2_matrix_create: bad parameters");
    H2_REQUIRE(kcap >= 1 && kcap <= kMaxCols, "h2_matrix_create: kcap must be in 1..32");
    for (int64_t i = 0; i < n * dim; ++i) H2_REQUIRE(std::isfinite(points[i]), "non-finite point");
    build_cluster_tree(points, n, dim, leaf_size, pad, Z->rows);
    Z->cols = Z->rows;
    build_block_tree(Z->rows, Z->cols, eta, Z->blocks);
    Z->kcap = kcap;
    Z->V.rank.assign(Z->rows.count(), 0);
    Z->W.rank.assign(Z->cols.count(), 0);
    if (!ctx) return;   // structure only (no device storage)
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    Z->device = ctx->device;
    alloc_basis(Z->rows, kcap, Z->V, st);
    alloc_basis(Z->cols, kcap, Z->W, st);
    const BlockTree& bt = Z->blocks;
    const size_t nadm = bt.adm.size();
    Z->d_S = dalloc<double>(nadm * kcap * kcap);
    H2_CUDA(cudaMemsetAsync(Z->d_S, 0, nadm * kcap * kcap * sizeof(double), st));
    Z->near_off.resize(bt.near.size());
    int64_t tot = 0;
    for (size_t i = 0; i < bt.near.size(); ++i) {
      Z->near_off[i] = tot;
      tot += Z->rows.size[bt.row[bt.near[i]]] * Z->cols.size[bt.col[bt.near[i]]];
    }
    Z->near_len = tot;
    Z->d_N = dalloc<double>(tot);
    H2_CUDA(cudaMemsetAsync(Z->d_N, 0, tot * sizeof(double), st));
    Z->d_row_off = upload(Z->rows.off, st);
    Z->d_col_off = upload(Z->cols.off, st);
    std::vector<int32_t> rs(Z->rows.size.begin(), Z->rows.size.end());
    std::vector<int32_t> cs(Z->cols.size.begin(), Z->cols.size.end());
    Z->d_row_size = upload(rs, st);
    Z->d_col_size = upload(cs, st);
    Z->d_subtree_r = upload(Z->rows.subtree, st);
    Z->d_subtree_c = upload(Z->cols.subtree, st);
    Z->d_father_r = upload(Z->rows.father, st);
    Z->d_father_c = upload(Z->cols.father, st);
    std::vector<int32_t> br(nadm), bc(nadm);
    for (size_t a = 0; a < nadm; ++a) {
      br[a] = bt.row[bt.adm[a]];
      bc[a] = bt.col[bt.adm[a]];
    }
    Z->d_blk_row = upload(br, st);
    Z->d_blk_col = upload(bc, st);
    Z->d_row_ptr = upload(bt.row_ptr, st);
    Z->d_row_adm = upload(bt.row_adm, st);
    Z->d_col_ptr = upload(bt.col_ptr, st);
    Z->d_col_adm = upload(bt.col_adm, st);
    H2_CUDA(cudaStreamSynchronize(st));
  });
  if (s == H2_OK) *out = Z.release();
  return s;
}

extern "C" void h2_matrix_free(h2_matrix* Z) {
  if (!Z) return;
  free_basis(Z->V);
  free_basis(Z->W);
  dfree(Z->d_S);
  dfree(Z->d_N);
  dfree(Z->d_row_off);
  dfree(Z->d_col_off);
  dfree(Z->d_row_size);
  dfree(Z->d_col_size);
  dfree(Z->d_subtree_r);
  dfree(Z->d_subtree_c);
  dfree(Z->d_father_r);
  dfree(Z->d_father_c);
  dfree(Z->d_blk_row);
  dfree(Z->d_blk_col);
  dfree(Z->d_row_ptr);
  dfree(Z->d_row_adm);
  dfree(Z->d_col_ptr);
  dfree(Z->d_col_adm);
  dfree(Z->d_mv_lvl[0]);
  dfree(Z->d_mv_lvl[1]);
  dfree(Z->d_mv_leaves);
  dfree(Z->d_near_ptr);
  dfree(Z->d_near_col);
  dfree(Z->d_near_off);
  delete Z;
}

extern "C" h2_status h2_matrix_clone(h2_ctx* ctx, const h2_matrix* Z, h2_matrix** out) {
  if (!ctx || !Z || !out) return H2_EINVAL;
  *out = nullptr;
  h2_matrix* C = nullptr;
  h2_status s = guard(ctx, [&] {
    H2_REQUIRE(has_storage(Z), "h2_matrix_clone: matrix has no device storage");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    std::unique_ptr<h2_matrix> Y(new h2_matrix());
    Y->rows = Z->rows;
    Y->cols = Z->cols;
    Y->blocks = Z->blocks;
    Y->kcap = Z->kcap;
    Y->device = Z->device;
    Y->near_off = Z->near_off;
    Y->near_len = Z->near_len;
    auto dup = [&](auto* src, size_t count) {
      using T = std::remove_const_t<std::remove_pointer_t<decltype(src)>>;
      T* d = dalloc<T>(count);
      if (count) H2_CUDA(cudaMemcpyAsync(d, src, count * sizeof(T), cudaMemcpyDeviceToDevice, st));
      return d;
    };
    for (int sd = 0; sd < 2; ++sd) {
      const ClusterTree& ct = tree_of(Z, sd);
      const DeviceBasis& ob = basis_of(Z, sd);
      DeviceBasis& nb = basis_of(Y.get(), sd);
      nb.rank = ob.rank;
      nb.leaf_off = ob.leaf_off;
      int64_t tot = 0;
      for (int32_t c = 0; c < ct.count(); ++c)
        if (ct.leaf(c)) tot += ct.size[c] * Z->kcap;
      nb.d_leaf = dup(ob.d_leaf, tot);
      nb.d_transfer = dup(ob.d_transfer, (size_t)ct.count() * Z->kcap * Z->kcap);
      nb.d_leaf_off = dup(ob.d_leaf_off, ct.count());
      nb.d_rank = dup(ob.d_rank, ct.count());
    }
    const size_t nadm = Z->blocks.adm.size();
    const int32_t nr = Z->rows.count(), nc = Z->cols.count();
    Y->d_S = dup(Z->d_S, nadm * Z->kcap * Z->kcap);
    Y->d_N = dup(Z->d_N, Z->near_len);
    Y->d_row_off = dup(Z->d_row_off, nr);
    Y->d_col_off = dup(Z->d_col_off, nc);
    Y->d_row_size = dup(Z->d_row_size, nr);
    Y->d_col_size = dup(Z->d_col_size, nc);
    Y->d_subtree_r = dup(Z->d_subtree_r, nr);
    Y->d_subtree_c = dup(Z->d_subtree_c, nc);
    Y->d_father_r = dup(Z->d_father_r, nr);
    Y->d_father_c = dup(Z->d_father_c, nc);
    Y->d_blk_row = dup(Z->d_blk_row, nadm);
    Y->d_blk_col = dup(Z->d_blk_col, nadm);
    Y->d_row_ptr = dup(Z->d_row_ptr, nr + 1);
    Y->d_row_adm = dup(Z->d_row_adm, nadm);
    Y->d_col_ptr = dup(Z->d_col_ptr, nc + 1);
    Y->d_col_adm = dup(Z->d_col_adm, nadm);
    H2_CUDA(cudaStreamSynchronize(st));
    C = Y.release();
  });
  if (s == H2_OK) *out = C;
  return s;
}

extern "C" h2_status h2_tree_sizes(const h2_matrix* Z, int64_t* n, int64_t* n_clusters, int64_t* n_blocks,
                                   int64_t* n_admissible, int64_t* n_inadmissible, int* depth) {
  if (!Z) return H2_EINVAL;
  if (n) *n = Z->rows.n;
  if (n_clusters) *n_clusters = Z->rows.count();
  if (n_blocks) *n_blocks = Z->blocks.count();
  if (n_admissible) *n_admissible = (int64_t)Z->blocks.adm.size();
  if (n_inadmissible) *n_inadmissible = (int64_t)Z->blocks.near.size();
  if (depth) *depth = Z->rows.depth;
  return H2_OK;
}

extern "C" h2_status h2_stats(const h2_matrix* Z, int64_t* out, int32_t* max_rank_per_level) {
  if (!Z || !out) return H2_EINVAL;
  const ClusterTree& rt = Z->rows;
  const ClusterTree& ct = Z->cols;
  const BlockTree& bt = Z->blocks;
  const std::vector<int32_t>& rv = Z->V.rank;
  const std::vector<int32_t>& rw = Z->W.rank;
  auto rank_at = [](const std::vector<int32_t>& r, int32_t c) { return c < (int32_t)r.size() ? r[c] : 0; };
  int64_t kmax_v = 0, kmax_w = 0, ksum = 0, cap_bytes = 0, val = 0;
  const int64_t kc = Z->kcap;
  for (int s = 0; s < 2; ++s) {
    const ClusterTree& tr = s == 0 ? rt : ct;
    const std::vector<int32_t>& rk = s == 0 ? rv : rw;
    for (int32_t c = 0; c < tr.count(); ++c) {
      const int64_t k = rank_at(rk, c);
      if (s == 0) {
        kmax_v = std::max(kmax_v, k);
        ksum += k;
      } else {
        kmax_w = std::max(kmax_w, k);
      }
      if (tr.leaf(c)) {
        cap_bytes += tr.size[c] * kc;
        val += tr.size[c] * k;
      }
      cap_bytes += kc * kc;
      if (tr.father[c] >= 0) val += k * rank_at(rk, tr.father[c]);
    }
  }
  int64_t near = 0;
  for (int32_t b : bt.near) near += rt.size[bt.row[b]] * ct.size[bt.col[b]];
  for (int32_t b : bt.adm) val += (int64_t)rank_at(rv, bt.row[b]) * rank_at(rw, bt.col[b]);
  cap_bytes += (int64_t)bt.adm.size() * kc * kc + near;
  val += near;
  if (!has_storage(Z) || (!bt.near.empty() && Z->d_N == nullptr)) cap_bytes = 0;   // structure only
  out[0] = rt.n;
  out[1] = rt.count();
  out[2] = bt.count();
  out[3] = (int64_t)bt.adm.size();
  out[4] = (int64_t)bt.near.size();
  out[5] = rt.depth;
  out[6] = kc;
  out[7] = kmax_v;
  out[8] = kmax_w;
  out[9] = 8 * cap_bytes;
  out[10] = 8 * val;
  out[11] = ksum;
  if (max_rank_per_level) {
    for (int l = 0; l <= rt.depth; ++l) max_rank_per_level[l] = 0;
    for (int32_t c = 0; c < rt.count(); ++c)
      max_rank_per_level[rt.level[c]] = std::max(max_rank_per_level[rt.level[c]], rank_at(rv, c));
  }
  return H2_OK;
}

extern "C" h2_status h2_tree_clusters(const h2_matrix* Z, int64_t* offset, int64_t* size,
                                      int32_t* father, int32_t* son0, int32_t* son1, int32_t* level,
                                      int32_t* subtree) {
  if (!Z) return H2_EINVAL;
  const ClusterTree& ct = Z->rows;
  const size_t nc = ct.count();
  if (offset) std::memcpy(offset, ct.off.data(), nc * sizeof(int64_t));
  if (size) std::memcpy(size, ct.size.data(), nc * sizeof(int64_t));
  if (father) std::memcpy(father, ct.father.data(), nc * sizeof(int32_t));
  if (son0) std::memcpy(son0, ct.son0.data(), nc * sizeof(int32_t));
  if (son1) std::memcpy(son1, ct.son1.data(), nc * sizeof(int32_t));
  if (level) std::memcpy(level, ct.level.data(), nc * sizeof(int32_t));
  if (subtree) std::memcpy(subtree, ct.subtree.data(), nc * sizeof(int32_t));
  return H2_OK;
}

extern "C" h2_status h2_tree_blocks(const h2_matrix* Z, int32_t* row, int32_t* col, int32_t* kind,
                                    int32_t* father) {
  if (!Z) return H2_EINVAL;
  const BlockTree& bt = Z->blocks;
  const size_t nb = bt.count();
  if (row) std::memcpy(row, bt.row.data(), nb * sizeof(int32_t));
  if (col) std::memcpy(col, bt.col.data(), nb * sizeof(int32_t));
  if (kind) std::memcpy(kind, bt.kind.data(), nb * sizeof(int32_t));
  if (father) std::memcpy(father, bt.father.data(), nb * sizeof(int32_t));
  return H2_OK;
}

extern "C" h2_status h2_tree_permutation(const h2_matrix* Z, int64_t* perm) {
  if (!Z || !perm) return H2_EINVAL;
  std::memcpy(perm, Z->rows.perm.data(), Z->rows.perm.size() * sizeof(int64_t));
  return H2_OK;
}

// ====================================================================== data
namespace {

void basis_lengths(const h2_matrix* Z, int side, const std::vector<int32_t>& rank, int64_t& leaf,
                   int64_t& transfer) {
  const ClusterTree& ct = tree_of(Z, side);
  leaf = 0;
  transfer = 0;
  for (int32_t c = 0; c < ct.count(); ++c) {
    if (ct.leaf(c)) leaf += ct.size[c] * rank[c];
    if (ct.father[c] >= 0) transfer += (int64_t)rank[c] * rank[ct.father[c]];
  }
}

int64_t coupling_length(const h2_matrix* Z) {
  int64_t tot = 0;
  for (int32_t b : Z->blocks.adm) tot += (int64_t)Z->V.rank[Z->blocks.row[b]] * Z->W.rank[Z->blocks.col[b]];
  return tot;
}

}  // namespace

extern "C" h2_status h2_data_sizes(const h2_matrix* Z, int side, int64_t* leaf_len, int64_t* transfer_len,
                                   int64_t* coupling_len, int64_t* nearfield_len) {
  if (!Z || (side != 0 && side != 1)) return H2_EINVAL;
  int64_t l = 0, t = 0;
  basis_lengths(Z, side, basis_of(Z, side).rank, l, t);
  if (leaf_len) *leaf_len = l;
  if (transfer_len) *transfer_len = t;
  if (coupling_len) *coupling_len = coupling_length(Z);
  if (nearfield_len) {
    int64_t nl = 0;
    for (int32_t b : Z->blocks.near) nl += Z->rows.size[Z->blocks.row[b]] * Z->cols.size[Z->blocks.col[b]];
    *nearfield_len = nl;
  }
  return H2_OK;
}

extern "C" h2_status h2_get_ranks(const h2_matrix* Z, int side, int32_t* ranks) {
  if (!Z || !ranks || (side != 0 && side != 1)) return H2_EINVAL;
  const DeviceBasis& b = basis_of(Z, side);
  std::memcpy(ranks, b.rank.data(), b.rank.size() * sizeof(int32_t));
  return H2_OK;
}

extern "C" h2_status h2_set_basis(h2_ctx* ctx, h2_matrix* Z, int side, const int32_t* ranks,
                                  const double* leaf_data, const double* transfer_data) {
  if (!ctx || !Z || !ranks || (side != 0 && side != 1)) return H2_EINVAL;
  return guard(ctx, [&] {
    H2_REQUIRE(has_storage(Z), "h2_set_basis: matrix has no device storage");
    const ClusterTree& ct = tree_of(Z, side);
    std::vector<int32_t> rk(ranks, ranks + ct.count());
    int kmax = 0;
    for (int32_t c = 0; c < ct.count(); ++c) {
      H2_REQUIRE(rk[c] >= 0 && rk[c] <= kMaxCols, "h2_set_basis: rank out of 0..32");
      if (ct.leaf(c)) H2_REQUIRE(rk[c] <= ct.size[c], "h2_set_basis: leaf rank above leaf size");
      kmax = std::max(kmax, rk[c]);
    }
    int64_t ll = 0, tl = 0;
    basis_lengths(Z, side, rk, ll, tl);
    H2_REQUIRE(ll == 0 || leaf_data, "h2_set_basis: leaf_data missing");
    H2_REQUIRE(tl == 0 || transfer_data, "h2_set_basis: transfer_data missing");
    DeviceGuard g(ctx->device);
    grow_kcap(ctx, Z, kmax);
    const int kcap = Z->kcap;
    DeviceBasis& b = basis_of(Z, side);
    std::vector<double> leaf;
    int64_t tot = 0;
    for (int32_t c = 0; c < ct.count(); ++c)
      if (ct.leaf(c)) tot += ct.size[c] * kcap;
    leaf.assign(tot, 0.0);
    std::vector<double> tr((size_t)ct.count() * kcap * kcap, 0.0);
    int64_t pl = 0, pt = 0;
    for (int32_t c = 0; c < ct.count(); ++c) {
      if (ct.leaf(c)) {
        const int64_t m = ct.size[c];
        std::memcpy(leaf.data() + b.leaf_off[c], leaf_data + pl, m * rk[c] * sizeof(double));
        pl += m * rk[c];
      }
      if (ct.father[c] >= 0) {
        const int kf = rk[ct.father[c]];
        for (int j = 0; j < kf; ++j)
          for (int i = 0; i < rk[c]; ++i)
            tr[(size_t)c * kcap * kcap + i + j * kcap] = transfer_data[pt + i + (int64_t)j * rk[c]];
        pt += (int64_t)rk[c] * kf;
      }
    }
    cudaStream_t st = ctx->stream;
    if (tot) H2_CUDA(cudaMemcpyAsync(b.d_leaf, leaf.data(), tot * sizeof(double), cudaMemcpyHostToDevice, st));
    H2_CUDA(cudaMemcpyAsync(b.d_transfer, tr.data(), tr.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    b.rank = rk;
    sync_ranks(b, st);
    H2_CUDA(cudaStreamSynchronize(st));
  });
}

extern "C" h2_status h2_get_basis(h2_ctx* ctx, const h2_matrix* Z, int side, double* leaf_data,
                                  double* transfer_data) {
  if (!ctx || !Z || (side != 0 && side != 1)) return H2_EINVAL;
  return guard(ctx, [&] {
    H2_REQUIRE(has_storage(Z), "h2_get_basis: matrix has no device storage");
    DeviceGuard g(ctx->device);
    const ClusterTree& ct = tree_of(Z, side);
    const DeviceBasis& b = basis_of(Z, side);
    const int kcap = Z->kcap;
    int64_t tot = 0;
    for (int32_t c = 0; c < ct.count(); ++c)
      if (ct.leaf(c)) tot += ct.size[c] * kcap;
    std::vector<double> leaf(tot), tr((size_t)ct.count() * kcap * kcap);
    cudaStream_t st = ctx->stream;
    if (tot) H2_CUDA(cudaMemcpyAsync(leaf.data(), b.d_leaf, tot * sizeof(double), cudaMemcpyDeviceToHost, st));
    H2_CUDA(cudaMemcpyAsync(tr.data(), b.d_transfer, tr.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    H2_CUDA(cudaStreamSynchronize(st));
    int64_t pl = 0, pt = 0;
    for (int32_t c = 0; c < ct.count(); ++c) {
      if (ct.leaf(c)) {
        const int64_t m = ct.size[c];
        if (leaf_data) std::memcpy(leaf_data + pl, leaf.data() + b.leaf_off[c], m * b.rank[c] * sizeof(double));
        pl += m * b.rank[c];
      }
      if (ct.father[c] >= 0) {
        const int kf = b.rank[ct.father[c]];
        if (transfer_data)
          for (int j = 0; j < kf; ++j)
            for (int i = 0; i < b.rank[c]; ++i)
              transfer_data[pt + i + (int64_t)j * b.rank[c]] = tr[(size_t)c * kcap * kcap + i + j * kcap];
        pt += (int64_t)b.rank[c] * kf;
      }
    }
  });
}

extern "C" h2_status h2_set_couplings(h2_ctx* ctx, h2_matrix* Z, const double* data) {
  if (!ctx || !Z) return H2_EINVAL;
  return guard(ctx, [&] {
    H2_REQUIRE(has_storage(Z), "h2_set_couplings: matrix has no device storage");
    H2_REQUIRE(data || coupling_length(Z) == 0, "h2_set_couplings: data missing");
    DeviceGuard g(ctx->device);
    const int kcap = Z->kcap;
    const BlockTree& bt = Z->blocks;
    std::vector<double> S(bt.adm.size() * kcap * kcap, 0.0);
    int64_t p = 0;
    for (size_t a = 0; a < bt.adm.size(); ++a) {
      const int kt = Z->V.rank[bt.row[bt.adm[a]]], ls = Z->W.rank[bt.col[bt.adm[a]]];
      for (int j = 0; j < ls; ++j)
        for (int i = 0; i < kt; ++i) S[a * kcap * kcap + i + j * kcap] = data[p + i + (int64_t)j * kt];
      p += (int64_t)kt * ls;
    }
    if (!S.empty())
      H2_CUDA(cudaMemcpyAsync(Z->d_S, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    H2_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

extern "C" h2_status h2_get_couplings(h2_ctx* ctx, const h2_matrix* Z, double* data) {
  if (!ctx || !Z || !data) return H2_EINVAL;
  return guard(ctx, [&] {
    H2_REQUIRE(has_storage(Z), "h2_get_couplings: matrix has no device storage");
    DeviceGuard g(ctx->device);
    const int kcap = Z->kcap;
    const BlockTree& bt = Z->blocks;
    std::vector<double> S(bt.adm.size() * kcap * kcap);
    if (!S.empty())
      H2_CUDA(cudaMemcpyAsync(S.data(), Z->d_S, S.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    H2_CUDA(cudaStreamSynchronize(ctx->stream));
    int64_t p = 0;
    for (size_t a = 0; a < bt.adm.size(); ++a) {
      const int kt = Z->V.rank[bt.row[bt.adm[a]]], ls = Z->W.rank[bt.col[bt.adm[a]]];
      for (int j = 0; j < ls; ++j)
        for (int i = 0; i < kt; ++i) data[p + i + (int64_t)j * kt] = S[a * kcap * kcap + i + j * kcap];
      p += (int64_t)kt * ls;
    }
  });
}

extern "C" h2_status h2_set_nearfield(h2_ctx* ctx, h2_matrix* Z, const double* data) {
  if (!ctx || !Z) return H2_EINVAL;
  return guard(ctx, [&] {
    H2_REQUIRE(has_storage(Z), "h2_set_nearfield: matrix has no device storage");
    H2_REQUIRE(data || Z->near_len == 0, "h2_set_nearfield: data missing");
    DeviceGuard g(ctx->device);
    if (Z->near_len)
      H2_CUDA(cudaMemcpyAsync(Z->d_N, data, Z->near_len * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    H2_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

extern "C" h2_status h2_get_nearfield(h2_ctx* ctx, const h2_matrix* Z, double* data) {
  if (!ctx || !Z || !data) return H2_EINVAL;
  return guard(ctx, [&] {
    H2_REQUIRE(has_storage(Z), "h2_get_nearfield: matrix has no device storage");
    DeviceGuard g(ctx->device);
    if (Z->near_len)
      H2_CUDA(cudaMemcpyAsync(data, Z->d_N, Z->near_len * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    H2_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

extern "C" h2_status h2_get_leaf(h2_ctx* ctx, const h2_matrix* Z, int side, int64_t cluster, double* out) {
  if (!ctx || !Z || !out || (side != 0 && side != 1)) return H2_EINVAL;
  return guard(ctx, [&] {
    const ClusterTree& ct = tree_of(Z, side);
    H2_REQUIRE(has_storage(Z), "h2_get_leaf: no device storage");
    H2_REQUIRE(cluster >= 0 && cluster < ct.count() && ct.leaf((int32_t)cluster), "h2_get_leaf: not a leaf");
    DeviceGuard g(ctx->device);
    const DeviceBasis& b = basis_of(Z, side);
    const size_t len = ct.size[cluster] * b.rank[cluster];
    if (len)
      H2_CUDA(cudaMemcpyAsync(out, b.d_leaf + b.leaf_off[cluster], len * sizeof(double), cudaMemcpyDeviceToHost,
                              ctx->stream));
    H2_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

extern "C" h2_status h2_get_transfer(h2_ctx* ctx, const h2_matrix* Z, int side, int64_t cluster, double* out) {
  if (!ctx || !Z || !out || (side != 0 && side != 1)) return H2_EINVAL;
  return guard(ctx, [&] {
    const ClusterTree& ct = tree_of(Z, side);
    H2_REQUIRE(has_storage(Z), "h2_get_transfer: no device storage");
    H2_REQUIRE(cluster > 0 && cluster < ct.count(), "h2_get_transfer: cluster out of range");
    DeviceGuard g(ctx->device);
    const DeviceBasis& b = basis_of(Z, side);
    const int k = b.rank[cluster], kf = b.rank[ct.father[cluster]];
    if (k && kf)
      H2_CUDA(cudaMemcpy2DAsync(out, k * sizeof(double), b.d_transfer + cluster * Z->kcap * Z->kcap,
                                Z->kcap * sizeof(double), k * sizeof(double), kf, cudaMemcpyDeviceToHost,
                                ctx->stream));
    H2_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

extern "C" h2_status h2_get_coupling(h2_ctx* ctx, const h2_matrix* Z, int64_t block, double* out) {
  if (!ctx || !Z || !out) return H2_EINVAL;
  return guard(ctx, [&] {
    const BlockTree& bt = Z->blocks;
    H2_REQUIRE(has_storage(Z), "h2_get_coupling: no device storage");
    H2_REQUIRE(block >= 0 && block < bt.count() && bt.kind[block] == kAdm, "h2_get_coupling: not admissible");
    DeviceGuard g(ctx->device);
    const int kt = Z->V.rank[bt.row[block]], ls = Z->W.rank[bt.col[block]];
    if (kt && ls)
      H2_CUDA(cudaMemcpy2DAsync(out, kt * sizeof(double), Z->d_S + (size_t)bt.slot[block] * Z->kcap * Z->kcap,
                                Z->kcap * sizeof(double), kt * sizeof(double), ls, cudaMemcpyDeviceToHost,
                                ctx->stream));
    H2_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

// ================================================================== batches
struct h2_batch {
  const h2_matrix* Z = nullptr;
  int device = 0;
  int u = 0;
  int64_t count = 0;
  std::vector<int64_t> blocks;
  std::vector<int64_t> offA, rowsA, offB, rowsB;
  int64_t lenA = 0, lenB = 0;
  // host plan
  std::vector<Item> items;
  std::vector<Entry> ents;
  std::vector<Task> tasks;
  std::vector<NormTask> norms;
  std::vector<int64_t> upd_item, upd_task;      // per update: first item / task (+ sentinel)
  std::vector<int32_t> lvl_list;                // items sorted by level
  std::vector<int32_t> lvl_ptr;                 // per level
  std::vector<int32_t> lvl_maxrows;             // per level: bound on rows of the truncation
  std::vector<int32_t> lvl_leaves;              // per level: leaves (first in lvl_list)
  std::vector<int32_t> cl_list, cl_ptr;         // clusters of both sides by level (side << 30 | id)
  // exact path, base weights B~ only for these clusters by level (empty:
  // cl_list); the update engine computes them only where its cache of the
  // unchanged matrix's weights is stale
  std::vector<int32_t> bl_list, bl_ptr;
  int depth = 0;
  int kl = 0;                                   // max extended rank
  int max_rank = 0;                             // rank cap of the exact path's truncation (0: none)
  int64_t qlen = 0;
  // result packing (execute_host)
  std::vector<int64_t> res_task_off, res_item_off;
  int64_t res_len = 0;
  int64_t res_prefix = 0;                       // ranks, two-sided couplings, bases
  std::vector<int32_t> one;                     // one-sided coupling tasks, in result order
  std::vector<int32_t> res_chunk_of;            // per task: chunk of the one-sided region or -1
  std::vector<int64_t> res_chunk_off;           // chunk boundaries (element offsets)
  int32_t* d_one = nullptr;
  int32_t* d_chunk_of = nullptr;
  int32_t* d_flags = nullptr;                   // per chunk: re-packed after the early copy
  int32_t* h_flags = nullptr;                   // page-locked copy of d_flags
  int8_t* h_copy = nullptr;                     // page-locked copy of the copy flags (compact result)
  bool compact = false;                         // this execution writes the compact host result
  int64_t h2d_bytes = 0, d2h_bytes = 0;         // copies of the last host execution
  cudaStream_t io = nullptr;                    // stream of the early copies
  HostOutput out{};
  double* g_res = nullptr;                      // host destination the graph copies to
  // device
  Item* d_items = nullptr;
  Entry* d_ents = nullptr;
  Task* d_tasks = nullptr;
  NormTask* d_norms = nullptr;
  int32_t* d_two = nullptr;      // two-sided coupling tasks
  int32_t* d_left = nullptr;     // one-sided tasks that need products (device-built)
  int32_t* d_nleft = nullptr;
  std::vector<int32_t> two;
  int32_t* d_lvl = nullptr;
  int32_t* d_cl = nullptr;
  int32_t* d_bl = nullptr;
  ItemBuffers IB{};
  BaseWeights BW{};
  double* d_A = nullptr;   // staging for execute_host
  double* d_B = nullptr;
  double* d_res = nullptr;
  int64_t* d_res_task_off = nullptr;
  int64_t* d_res_item_off = nullptr;
  int64_t launches = 0;
  int64_t phase_launches[H2_PHASE_COUNT] = {};
  int mode = H2_MODE_AUTO;
  bool executed = false;
  int timing = 0;                            // 0 off, 1 phase events, 2 phase events, one stream
  cudaEvent_t ev[2 * H2_PHASE_COUNT] = {};   // start and end of every phase
  cudaStream_t side = nullptr;               // stream of the weights of the unchanged matrix
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaStream_t side2 = nullptr;              // stream of the basis Grams of the unchanged matrix
  cudaEvent_t join2 = nullptr;
  // CUDA graph of the launch sequence, captured when the batch is executed
  // again with the same arguments and replayed while they stay the same
  cudaGraphExec_t graph = nullptr;
  const double* g_A = nullptr;
  const double* g_B = nullptr;
  double g_eps = -1.0;
  int g_mode = -1;
  int g_timing = 0;
  bool g_compact = false;
  int g_repeats = 0;
  bool g_broken = false;                     // capture failed once: stay eager
  MatView g_view{};                          // the matrix storage the graph reads
  const h2_ctx* g_ctx = nullptr;
  cudaStream_t cap = nullptr;                // private stream for the capture (the context's
                                             // stream may be the legacy default stream)
};

namespace {

constexpr int kResChunks = 64;   // chunks of the one-sided region of a host result

void plan_batch(h2_batch& P) {
  const h2_matrix* Z = P.Z;
  const ClusterTree* tr[2] = {&Z->rows, &Z->cols};
  const BlockTree& bt = Z->blocks;
  const int u = P.u;
  std::vector<int32_t> item_of[2];
  item_of[0].assign(Z->rows.count(), -1);
  item_of[1].assign(Z->cols.count(), -1);
  std::unordered_map<int32_t, int32_t> norm_of;   // coupling slot -> norm task (per update)
  P.depth = std::max(Z->rows.depth, Z->cols.depth);
  P.upd_item.assign(P.count + 1, 0);
  P.upd_task.assign(P.count + 1, 0);
  int64_t qoff = 0;
  for (int64_t j = 0; j < P.count; ++j) {
    const int32_t b0 = (int32_t)P.blocks[j];
    const int32_t root[2] = {bt.row[b0], bt.col[b0]};
    P.upd_item[j] = (int64_t)P.items.size();
    P.upd_task[j] = (int64_t)P.tasks.size();
    std::vector<int32_t> sub[2];
    for (int sd = 0; sd < 2; ++sd) {
      const ClusterTree& ct = *tr[sd];
      const DeviceBasis& bs = basis_of(Z, sd);
      // depth-first preorder of the subtree
      std::vector<int32_t> stack{root[sd]};
      while (!stack.empty()) {
        const int32_t c = stack.back();
        stack.pop_back();
        sub[sd].push_back(c);
        if (!ct.leaf(c)) {
          stack.push_back(ct.son1[c]);
          stack.push_back(ct.son0[c]);
        }
      }
      for (int32_t c : sub[sd]) {
        Item it{};
        it.update = (int32_t)j;
        it.side = sd;
        it.cluster = c;
        it.parent = (c == root[sd]) ? -1 : item_of[sd][ct.father[c]];
        it.son0 = it.son1 = -1;
        it.flags = 0;
        if (ct.leaf(c)) it.flags |= kItemLeaf;
        if (c == root[sd]) it.flags |= kItemRoot;
        if (ct.father[c] < 0) it.flags |= kItemTreeRoot;
        it.k = bs.rank[c];
        it.kf = ct.father[c] >= 0 ? bs.rank[ct.father[c]] : 0;
        H2_REQUIRE(it.k + u <= kMaxCols, "h2_batch_create: k_t + u exceeds 32");
        it.size = (int32_t)ct.size[c];
        it.rowoff = (int32_t)(ct.off[c] - ct.off[root[sd]]);
        it.ld = (int32_t)ct.size[root[sd]];
        it.foff = sd == 0 ? P.offA[j] : P.offB[j];
        it.qoff = -1;
        if (ct.leaf(c)) {
          it.qoff = qoff;
          qoff += ct.size[c] * (it.k + u);
        }
        item_of[sd][c] = (int32_t)P.items.size();
        P.items.push_back(it);
      }
      for (int32_t c : sub[sd])
        if (!ct.leaf(c)) {
          Item& it = P.items[item_of[sd][c]];
          it.son0 = item_of[sd][ct.son0[c]];
          it.son1 = item_of[sd][ct.son1[c]];
        }
    }
    // entries and tasks
    norm_of.clear();
    for (int sd = 0; sd < 2; ++sd) {
      const std::vector<int32_t>& ptr = sd == 0 ? bt.row_ptr : bt.col_ptr;
      const std::vector<int32_t>& adm = sd == 0 ? bt.row_adm : bt.col_adm;
      for (int32_t c : sub[sd]) {
        const int32_t iid = item_of[sd][c];
        Item& it = P.items[iid];
        it.ent_begin = (int32_t)P.ents.size();
        for (int32_t e = ptr[c]; e < ptr[c + 1]; ++e) {
          const int32_t slot = adm[e];
          const int32_t blk = bt.adm[slot];
          const int32_t o = sd == 0 ? bt.col[blk] : bt.row[blk];
          const int32_t oi = item_of[1 - sd][o];
          Entry en{slot, oi, o, -1};
          if (oi >= 0) {
            auto f = norm_of.find(slot);
            if (f == norm_of.end()) {
              const int32_t nid = (int32_t)P.norms.size();
              P.norms.push_back(NormTask{slot, sd == 0 ? iid : oi, sd == 0 ? oi : iid, 0});
              norm_of.emplace(slot, nid);
              en.norm = nid;
            } else {
              en.norm = f->second;
            }
            it.flags |= kItemInside;
          }
          P.ents.push_back(en);
          const int kt = Z->V.rank[bt.row[blk]], ls = Z->W.rank[bt.col[blk]];
          if (sd == 0)
            P.tasks.push_back(Task{slot, iid, oi, kt, ls});
          else if (oi < 0)
            P.tasks.push_back(Task{slot, -1, iid, kt, ls});
        }
        it.ent_end = (int32_t)P.ents.size();
      }
    }
    for (int sd = 0; sd < 2; ++sd)
      for (int32_t c : sub[sd]) item_of[sd][c] = -1;
  }
  P.upd_item[P.count] = (int64_t)P.items.size();
  P.upd_task[P.count] = (int64_t)P.tasks.size();
  P.qlen = qoff;
  H2_REQUIRE(P.items.size() < (size_t)INT32_MAX && P.tasks.size() < (size_t)INT32_MAX,
             "h2_batch_create: batch too large");
  // level lists
  const int L = P.depth + 1;
  P.lvl_ptr.assign(L + 1, 0);
  P.lvl_maxrows.assign(L, 0);
  P.kl = 0;
  for (const Item& it : P.items) {
    const int lev = tr[it.side]->level[it.cluster];
    P.lvl_ptr[lev + 1]++;
    P.kl = std::max(P.kl, it.k + u);
  }
  for (int l = 0; l < L; ++l) P.lvl_ptr[l + 1] += P.lvl_ptr[l];
  P.lvl_list.assign(P.items.size(), 0);
  P.lvl_leaves.assign(L, 0);
  std::vector<int32_t> fill(P.lvl_ptr.begin(), P.lvl_ptr.end() - 1);
  for (int pass = 0; pass < 2; ++pass)   // leaves first within a level
    for (size_t i = 0; i < P.items.size(); ++i) {
      const Item& it = P.items[i];
      const bool leaf = it.flags & kItemLeaf;
      if (leaf != (pass == 0)) continue;
      const int lev = tr[it.side]->level[it.cluster];
      P.lvl_list[fill[lev]++] = (int32_t)i;
      if (leaf) ++P.lvl_leaves[lev];
      int rows = it.size;
      if (!leaf) rows = P.items[it.son0].k + P.items[it.son1].k + 2 * u;
      P.lvl_maxrows[lev] = std::max(P.lvl_maxrows[lev], rows);
    }
  for (int l = 0; l < L; ++l)
    H2_REQUIRE(P.lvl_maxrows[l] <= 64, "h2_batch_create: leaf clusters above 64 indices are not supported");
  // all clusters of both sides by level (weights of the unchanged matrix)
  P.cl_ptr.assign(L + 1, 0);
  for (int sd = 0; sd < 2; ++sd)
    for (int32_t c = 0; c < tr[sd]->count(); ++c) P.cl_ptr[tr[sd]->level[c] + 1]++;
  for (int l = 0; l < L; ++l) P.cl_ptr[l + 1] += P.cl_ptr[l];
  P.cl_list.assign(P.cl_ptr[L], 0);
  {
    std::vector<int32_t> f2(P.cl_ptr.begin(), P.cl_ptr.end() - 1);
    for (int sd = 0; sd < 2; ++sd)
      for (int32_t c = 0; c < tr[sd]->count(); ++c) P.cl_list[f2[tr[sd]->level[c]]++] = (sd << 30) | c;
  }
  // packed result layout: [ranks of the cluster tasks][couplings of the
  // blocks with both clusters changed][leaf bases / transfer matrices][
  // couplings of the blocks with one cluster changed], each piece at the
  // size of its largest possible rank.  The last region comes in chunks of
  // whole blocks (the unit of a repeated copy to the host).
  P.two.clear();
  P.one.clear();
  for (size_t t = 0; t < P.tasks.size(); ++t)
    (P.tasks[t].it >= 0 && P.tasks[t].is >= 0 ? P.two : P.one).push_back((int32_t)t);
  auto task_len = [&](const Task& tk) {
    const int R = tk.it >= 0 ? tk.kt + u : tk.kt;
    const int C = tk.is >= 0 ? tk.ls + u : tk.ls;
    return (int64_t)R * C;
  };
  int64_t off = (int64_t)P.items.size();
  P.res_task_off.assign(P.tasks.size(), 0);
  for (int32_t t : P.two) {
    P.res_task_off[t] = off;
    off += task_len(P.tasks[t]);
  }
  P.res_item_off.resize(P.items.size());
  for (size_t i = 0; i < P.items.size(); ++i) {
    const Item& it = P.items[i];
    P.res_item_off[i] = off;
    const int K = it.k + u;
    if (it.flags & kItemLeaf) off += (int64_t)it.size * K;
    if (!(it.flags & kItemTreeRoot)) {
      const int Kf = (it.flags & kItemRoot) ? it.kf : it.kf + u;
      off += (int64_t)K * Kf;
    }
  }
  P.res_prefix = off;
  int64_t one_len = 0;
  for (int32_t t : P.one) one_len += task_len(P.tasks[t]);
  const int64_t per_chunk = std::max<int64_t>(1, (one_len + kResChunks - 1) / kResChunks);
  P.res_chunk_of.assign(P.tasks.size(), -1);
  P.res_chunk_off.assign(1, off);
  for (int32_t t : P.one) {
    if (off - P.res_chunk_off.back() >= per_chunk) P.res_chunk_off.push_back(off);
    P.res_task_off[t] = off;
    P.res_chunk_of[t] = (int32_t)P.res_chunk_off.size() - 1;
    off += task_len(P.tasks[t]);
  }
  P.res_chunk_off.push_back(off);
  P.res_len = off;
}

// ------------------------------------------------ results to host memory
// One warp per object.  A coupling task's piece is the new coupling (rows =
// new rank of the row cluster, or its old rank when only the column cluster
// changed; column-major, ld = rows); an item's piece is its new leaf basis
// (#t x r, ld #t, leaves only) followed by its new transfer matrix (r x
// rank of the father, ld r; the committed E_t0 for the subtree root; none
// for the tree root); result[i] = new rank of item i.
// [S_b; 0] ((k_t + u) x l_s) or [S_b, 0] (k_t x (l_s + u)) from the
// unchanged coupling.
__device__ void pack_copy(const MatView& M, const Task& tk, int u, double* d, int lane) {
  const int rt = tk.it >= 0 ? tk.kt + u : tk.kt;
  const int rs = tk.it >= 0 ? tk.ls : tk.ls + u;
  const double* S = M.S + (size_t)tk.slot * M.kcap * M.kcap;
  for (int e = lane; e < rt * rs; e += 32) {
    const int i = e % rt, j = e / rt;
    d[e] = (i < tk.kt && j < tk.ls) ? S[i + (size_t)j * M.kcap] : 0.0;
  }
}

__device__ void pack_task(const MatView& M, const Task& tk, int t, int u, const ItemBuffers& IB,
                          const int64_t* task_off, double* res, int lane) {
  if (IB.copy[t]) {
    pack_copy(M, tk, u, res + task_off[t], lane);
    return;
  }
  const int rt = tk.it >= 0 ? IB.rank[tk.it] : tk.kt;
  const int rs = tk.is >= 0 ? IB.rank[tk.is] : tk.ls;
  const double* S = IB.S_out + (size_t)t * kSlot;
  double* d = res + task_off[t];
  for (int e = lane; e < rt * rs; e += 32) d[e] = S[(e % rt) + (e / rt) * 32];
}

__device__ void pack_item(const Item* items, int i, int u, const ItemBuffers& IB, const int64_t* item_off,
                          double* res, int lane) {
  const Item it = items[i];
  const int r = IB.rank[i];
  if (lane == 0) res[i] = (double)r;
  double* d = res + item_off[i];
  if (it.flags & kItemLeaf) {
    const double* Q = IB.Q + it.qoff;
    for (int e = lane; e < it.size * r; e += 32) d[e] = Q[e];
    d += (size_t)it.size * (it.k + u);
  }
  if (!(it.flags & kItemTreeRoot)) {
    const int rf = (it.flags & kItemRoot) ? it.kf : IB.rank[it.parent];
    const double* F = IB.F + (size_t)i * kSlot;
    for (int e = lane; e < r * rf; e += 32) d[e] = F[(e % r) + (e / r) * 32];
  }
}

constexpr int kPackWarps = 8;

// Everything, after the update.
__global__ void k_pack(MatView M, const Item* items, int ni, const Task* tasks, int nt, int u, ItemBuffers IB,
                       const int64_t* task_off, const int64_t* item_off, double* res) {
  const int o = blockIdx.x * kPackWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (o < nt) {
    pack_task(M, tasks[o], o, u, IB, task_off, res, lane);
  } else if (o < nt + ni) {
    pack_item(items, o - nt, u, IB, item_off, res, lane);
  }
}

// Early: a one-sided coupling task whose changed cluster has an orthonormal
// basis becomes [S_b; 0] or [S_b, 0] when the update is certified (the old
// basis stays the leading part of the new one, Section 5 with the block form
// of the certified path): packed from the unchanged coupling.
__global__ void k_pack_early(MatView M, const Item* items, const Task* tasks, const int32_t* one, int n_one,
                             int u, BaseWeights BW, const int64_t* task_off, double* res) {
  const int o = blockIdx.x * kPackWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (o >= n_one) return;
  const int t = one[o];
  const Task tk = tasks[t];
  const int side = tk.it >= 0 ? 0 : 1;
  const Item it = items[side == 0 ? tk.it : tk.is];
  if (!(side ? BW.orth[1] : BW.orth[0])[it.cluster]) return;
  pack_copy(M, tk, u, res + task_off[t], lane);
}

// Late: the two-sided couplings, the bases and ranks, and the one-sided
// couplings the early pass did not fix (all of them when it did not run;
// else those of failed updates or of clusters without an orthonormal basis,
// whose chunks are flagged for a second copy).
__global__ void k_pack_late(MatView M, const Item* items, int ni, const Task* tasks, const int32_t* two, int n_two,
                            const int32_t* one, int n_one, int u, ItemBuffers IB, BaseWeights BW,
                            const int64_t* task_off, const int64_t* item_off, const int32_t* chunk_of,
                            int32_t* flags, int early_ran, double* res) {
  const int o = blockIdx.x * kPackWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (o < n_two) {
    const int t = two[o];
    pack_task(M, tasks[t], t, u, IB, task_off, res, lane);
  } else if (o < n_two + ni) {
    pack_item(items, o - n_two, u, IB, item_off, res, lane);
  } else if (o < n_two + ni + n_one) {
    const int t = one[o - n_two - ni];
    const Task tk = tasks[t];
    if (early_ran) {
      // the early pass packed exactly the tasks that turned out copies
      if (IB.copy[t]) return;
      if (lane == 0) flags[chunk_of[t]] = 1;
    }
    pack_task(M, tk, t, u, IB, task_off, res, lane);
  }
}

int pack_blocks(int64_t n) { return (int)((n + kPackWarps - 1) / kPackWarps); }

void early_output(const Pipeline& pp, const HostOutput& O, cudaStream_t st) {
  h2_batch& P = *static_cast<h2_batch*>(O.owner);
  const int n_one = (int)P.one.size();
  if (P.compact) {
    // the couplings that turn out copies stay on the device: nothing to send early
    H2_CUDA(cudaEventRecord(O.packed, st));
    return;
  }
  if (n_one > 0)
    k_pack_early<<<pack_blocks(n_one), 32 * kPackWarps, 0, st>>>(pp.M, pp.items, pp.tasks, P.d_one, n_one, pp.u,
                                                                  pp.BW, P.d_res_task_off, P.d_res);
  H2_CUDA(cudaEventRecord(O.packed, st));
  const int64_t len = P.res_len - P.res_prefix;
  if (len > 0)
    H2_CUDA(cudaMemcpyAsync(P.g_res + P.res_prefix, P.d_res + P.res_prefix, len * sizeof(double),
                            cudaMemcpyDeviceToHost, st));
}

void late_output(const Pipeline& pp, const HostOutput& O, cudaStream_t st, bool early_ran) {
  h2_batch& P = *static_cast<h2_batch*>(O.owner);
  const int n_two = (int)P.two.size(), ni = (int)P.items.size(), n_one = (int)P.one.size();
  const int nch = (int)P.res_chunk_off.size() - 1;
  if (early_ran && nch > 0) H2_CUDA(cudaMemsetAsync(P.d_flags, 0, nch * sizeof(int32_t), st));
  const int64_t n = (int64_t)n_two + ni + n_one;
  if (n > 0)
    k_pack_late<<<pack_blocks(n), 32 * kPackWarps, 0, st>>>(pp.M, pp.items, ni, pp.tasks, P.d_two, n_two, P.d_one,
                                                            n_one,
                                                            pp.u, pp.IB, pp.BW, P.d_res_task_off, P.d_res_item_off,
                                                            P.d_chunk_of, P.d_flags, early_ran ? 1 : 0, P.d_res);
  if (P.res_prefix > 0)
    H2_CUDA(cudaMemcpyAsync(P.g_res, P.d_res, P.res_prefix * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (!early_ran) {
    const int64_t len = P.res_len - P.res_prefix;
    if (len > 0)
      H2_CUDA(cudaMemcpyAsync(P.g_res + P.res_prefix, P.d_res + P.res_prefix, len * sizeof(double),
                              cudaMemcpyDeviceToHost, st));
  } else if (nch > 0) {
    H2_CUDA(cudaMemcpyAsync(P.h_flags, P.d_flags, nch * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  }
  if (P.compact && !P.tasks.empty())
    H2_CUDA(cudaMemcpyAsync(P.h_copy, pp.IB.copy, P.tasks.size() * sizeof(int8_t), cudaMemcpyDeviceToHost, st));
}

// Buffers of the host result (first h2_batch_execute_host).
void alloc_result(h2_batch& P, cudaStream_t st) {
  if (P.d_res || !P.res_len) return;
  P.d_res = dalloc<double>(P.res_len);
  P.d_res_task_off = upload(P.res_task_off, st);
  P.d_res_item_off = upload(P.res_item_off, st);
  P.d_one = upload(P.one, st);
  P.d_chunk_of = upload(P.res_chunk_of, st);
  const size_t nch = P.res_chunk_off.size() - 1;
  P.d_flags = dalloc<int32_t>(nch);
  if (nch) H2_CUDA(cudaHostAlloc(&P.h_flags, nch * sizeof(int32_t), cudaHostAllocDefault));
  if (!P.tasks.empty()) H2_CUDA(cudaHostAlloc(&P.h_copy, P.tasks.size() * sizeof(int8_t), cudaHostAllocDefault));
  // the early copies' pack kernel runs beside the update's kernels: give its
  // stream the highest priority so that its blocks do not wait for theirs
  int lo = 0, hi = 0;
  H2_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  H2_CUDA(cudaStreamCreateWithPriority(&P.io, cudaStreamNonBlocking, hi));
  P.out.stream = P.io;
  H2_CUDA(cudaEventCreateWithFlags(&P.out.ready, cudaEventDisableTiming));
  H2_CUDA(cudaEventCreateWithFlags(&P.out.packed, cudaEventDisableTiming));
  H2_CUDA(cudaEventCreateWithFlags(&P.out.done, cudaEventDisableTiming));
  P.out.early = early_output;
  P.out.late = late_output;
  P.out.owner = &P;
}

void alloc_batch(h2_ctx* ctx, h2_batch& P) {
  cudaStream_t st = ctx->stream;
  H2_CUDA(cudaStreamCreateWithFlags(&P.side, cudaStreamNonBlocking));
  H2_CUDA(cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming));
  H2_CUDA(cudaEventCreateWithFlags(&P.join, cudaEventDisableTiming));
  H2_CUDA(cudaStreamCreateWithFlags(&P.side2, cudaStreamNonBlocking));
  H2_CUDA(cudaStreamCreateWithFlags(&P.cap, cudaStreamNonBlocking));
  H2_CUDA(cudaEventCreateWithFlags(&P.join2, cudaEventDisableTiming));
  P.d_items = upload(P.items, st);
  P.d_ents = upload(P.ents, st);
  P.d_tasks = upload(P.tasks, st);
  P.d_two = upload(P.two, st);

  P.d_left = dalloc<int32_t>(P.tasks.size());
  P.d_nleft = dalloc<int32_t>(1);
  P.d_norms = upload(P.norms, st);
  P.d_lvl = upload(P.lvl_list, st);
  P.d_cl = upload(P.cl_list, st);
  const size_t ni = P.items.size();
  P.IB.Rq = dalloc<double>(ni * kSlot);
  P.IB.Bw = dalloc<double>(ni * kSlot);
  P.IB.Gv = dalloc<double>(ni * kSlot);
  P.IB.Wg = dalloc<double>(ni * kSlot);
  P.IB.fail = dalloc<int32_t>(P.count);
  P.IB.Rt = dalloc<double>(ni * kSlot);
  P.IB.F = dalloc<double>(ni * kSlot);
  P.IB.Q = dalloc<double>(P.qlen);
  P.IB.rank = dalloc<int32_t>(ni);
  P.IB.own = dalloc<int32_t>(ni);
  P.IB.norms = dalloc<double>(P.norms.size());
  P.IB.S_out = dalloc<double>(P.tasks.size() * kSlot);
  P.IB.copy = dalloc<int8_t>(P.tasks.size());
  P.IB.jac = dalloc<unsigned long long>(4 * ni);
  if (ni) H2_CUDA(cudaMemsetAsync(P.IB.jac, 0, 4 * ni * sizeof(unsigned long long), st));
  const int32_t ncl[2] = {P.Z->rows.count(), P.Z->cols.count()};
  for (int sd = 0; sd < 2; ++sd) {
    P.BW.G[sd] = dalloc<double>((size_t)ncl[sd] * kSlot);
    P.BW.B[sd] = dalloc<double>((size_t)ncl[sd] * kSlot);
    // the certified path's Gram matrices are dead before the exact path
    // writes G and B
    P.BW.Wo[sd] = P.BW.G[sd];
    P.BW.W0[sd] = P.BW.B[sd];
    P.BW.need[sd] = dalloc<int32_t>(ncl[sd]);
    P.BW.Vg[sd] = dalloc<double>((size_t)ncl[sd] * kSlot);
    P.BW.orth[sd] = dalloc<int32_t>(ncl[sd]);
  }
  H2_CUDA(cudaStreamSynchronize(st));
}

void free_batch_device(h2_batch& P) {
  if (P.graph) cudaGraphExecDestroy(P.graph);
  P.graph = nullptr;
  if (P.side) cudaStreamSynchronize(P.side);
  if (P.side2) cudaStreamSynchronize(P.side2);
  if (P.cap) cudaStreamDestroy(P.cap);
  P.cap = nullptr;
  if (P.io) {
    cudaStreamSynchronize(P.io);
    cudaStreamDestroy(P.io);
  }
  P.io = nullptr;
  for (cudaEvent_t* e : {&P.out.ready, &P.out.packed, &P.out.done}) {
    if (*e) cudaEventDestroy(*e);
    *e = nullptr;
  }
  if (P.h_flags) cudaFreeHost(P.h_flags);
  P.h_flags = nullptr;
  if (P.h_copy) cudaFreeHost(P.h_copy);
  P.h_copy = nullptr;
  dfree(P.d_one);
  dfree(P.d_chunk_of);
  dfree(P.d_flags);
  if (P.join2) cudaEventDestroy(P.join2);
  if (P.side2) cudaStreamDestroy(P.side2);
  P.join2 = nullptr;
  P.side2 = nullptr;
  if (P.fork) cudaEventDestroy(P.fork);
  if (P.join) cudaEventDestroy(P.join);
  if (P.side) cudaStreamDestroy(P.side);
  P.fork = P.join = nullptr;
  P.side = nullptr;
  dfree(P.d_items);
  dfree(P.d_ents);
  dfree(P.d_tasks);
  dfree(P.d_two);
  dfree(P.d_left);
  dfree(P.d_nleft);
  dfree(P.d_norms);
  dfree(P.d_lvl);
  dfree(P.d_cl);
  dfree(P.d_bl);
  for (int sd = 0; sd < 2; ++sd) {
    dfree(P.BW.G[sd]);
    dfree(P.BW.B[sd]);
    dfree(P.BW.need[sd]);
    dfree(P.BW.Vg[sd]);
    dfree(P.BW.orth[sd]);
    P.BW.Wo[sd] = P.BW.W0[sd] = nullptr;
  }
  dfree(P.IB.Rq);
  dfree(P.IB.Bw);
  dfree(P.IB.Gv);
  dfree(P.IB.Wg);
  dfree(P.IB.fail);
  dfree(P.IB.Rt);
  dfree(P.IB.F);
  dfree(P.IB.Q);
  dfree(P.IB.rank);
  dfree(P.IB.own);
  dfree(P.IB.norms);
  dfree(P.IB.S_out);
  dfree(P.IB.copy);
  dfree(P.IB.jac);
  dfree(P.d_A);
  dfree(P.d_B);
  dfree(P.d_res);
  dfree(P.d_res_task_off);
  dfree(P.d_res_item_off);
}

bool same_view(const MatView& a, const MatView& b) {
  for (int sd = 0; sd < 2; ++sd)
    if (a.leaf[sd] != b.leaf[sd] || a.transfer[sd] != b.transfer[sd] || a.leaf_off[sd] != b.leaf_off[sd] ||
        a.rank[sd] != b.rank[sd] || a.father[sd] != b.father[sd] || a.subtree[sd] != b.subtree[sd] ||
        a.size[sd] != b.size[sd])
      return false;
  return a.S == b.S && a.kcap == b.kcap;
}

// h_res: page-locked host destination of the packed result (its copies are
// part of the launch sequence), or nullptr.
void execute(h2_ctx* ctx, h2_batch& P, const double* A, const double* B, double eps, double* h_res = nullptr) {
  const h2_matrix* Z = P.Z;
  Pipeline pp{};
  pp.M = view_of(Z);
  pp.BL.ptr[0] = Z->d_row_ptr;
  pp.BL.ptr[1] = Z->d_col_ptr;
  pp.BL.adm[0] = Z->d_row_adm;
  pp.BL.adm[1] = Z->d_col_adm;
  pp.BL.other[0] = Z->d_blk_col;
  pp.BL.other[1] = Z->d_blk_row;
  pp.BW = P.BW;
  pp.IB = P.IB;
  pp.items = P.d_items;
  pp.ents = P.d_ents;
  pp.tasks = P.d_tasks;
  pp.norms = P.d_norms;
  pp.lvl_list = P.d_lvl;
  pp.lvl_ptr = P.lvl_ptr.data();
  pp.lvl_rows = P.lvl_maxrows.data();
  pp.lvl_leaves = P.lvl_leaves.data();
  pp.cl_list = P.d_cl;
  pp.cl_ptr = P.cl_ptr.data();
  pp.bl_list = P.bl_ptr.empty() ? nullptr : P.d_bl;
  pp.bl_ptr = P.bl_ptr.empty() ? nullptr : P.bl_ptr.data();
  pp.levels = P.depth + 1;
  pp.n_updates = (int)P.count;
  pp.ncl[0] = Z->rows.count();
  pp.ncl[1] = Z->cols.count();
  pp.exact_only = P.mode == H2_MODE_EXACT ? 1 : 0;
  pp.n_tasks = (int)P.tasks.size();
  pp.two = P.d_two;
  pp.n_two = (int)P.two.size();
  pp.left = P.d_left;
  pp.n_left = P.d_nleft;
  pp.n_norms = (int)P.norms.size();
  pp.u = P.u;
  pp.kl = P.kl;
  pp.max_rank = P.max_rank;
  pp.eps = eps;
  pp.A = A;
  pp.B = B;
  pp.err = ctx->d_error;
  pp.stream = ctx->stream;
  // timing mode 2 runs every phase on the context's stream (no overlap), so
  // that each phase's events time its kernels alone
  const bool one_stream = P.timing == 2;
  pp.side = one_stream ? nullptr : P.side;
  pp.fork = P.fork;
  pp.join = P.join;
  pp.side2 = one_stream ? nullptr : P.side2;
  pp.join2 = P.join2;
  pp.events = P.timing ? P.ev : nullptr;
  pp.phase_launches = P.phase_launches;
  // the first execution with given arguments runs eagerly (it also sets the
  // kernels' attributes); a repeat is captured once into a graph and the
  // graph is replayed while the arguments stay the same
  // (the graph holds the matrix's storage pointers, which change when its
  // rank capacity grows, and the context's error word)
  pp.out = h_res ? &P.out : nullptr;
  const bool same = A == P.g_A && B == P.g_B && eps == P.g_eps && P.mode == P.g_mode && P.timing == P.g_timing &&
                    ctx == P.g_ctx && same_view(pp.M, P.g_view) && h_res == P.g_res &&
                    P.compact == P.g_compact;
  if (!same) {
    P.g_res = h_res;
    P.g_view = pp.M;
    P.g_ctx = ctx;
    if (P.graph) cudaGraphExecDestroy(P.graph);
    P.graph = nullptr;
    P.g_A = A;
    P.g_B = B;
    P.g_eps = eps;
    P.g_mode = P.mode;
    P.g_timing = P.timing;
    P.g_compact = P.compact;
    P.g_repeats = 0;
  } else {
    ++P.g_repeats;
  }
  bool done = false;
  if (P.g_repeats >= 1 && !P.g_broken && P.side) {
    if (!P.graph) {
      cudaGraph_t g = nullptr;
      Pipeline pc = pp;
      pc.stream = P.cap;
      pc.capturing = true;
      bool ok = cudaStreamBeginCapture(P.cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        try {
          run_pipeline(pc);
        } catch (...) {
          ok = false;
        }
        ok = cudaStreamEndCapture(P.cap, &g) == cudaSuccess && ok;
        ok = ok && cudaGraphInstantiate(&P.graph, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
      }
      if (!ok) {
        (void)cudaGetLastError();
        if (P.graph) cudaGraphExecDestroy(P.graph);
        P.graph = nullptr;
        P.g_broken = true;
      }
    }
    if (P.graph) {
      H2_CUDA(cudaGraphLaunch(P.graph, ctx->stream));
      done = true;
    }
  }
  if (!done) run_pipeline(pp);
  int64_t launches = 0;
  for (int ph = 0; ph < H2_PHASE_COUNT; ++ph) launches += P.phase_launches[ph];
  P.launches = launches;
  P.executed = true;
}

}  // namespace

namespace {
// A batch over `blocks`; the factors of update j start at offA[j], offB[j]
// of the concatenated arrays when given (else they are packed in order).
h2_status create_batch(h2_ctx* ctx, const h2_matrix* Z, int64_t count, const int64_t* blocks, int u,
                       const int64_t* offA, const int64_t* offB, h2_batch** out) {
  if (!Z || !out || count < 0 || (count > 0 && !blocks)) return H2_EINVAL;
  *out = nullptr;
  auto P = std::make_unique<h2_batch>();
  h2_status s = guard(ctx, [&] {
    H2_REQUIRE(u >= 1 && u < kMaxCols, "h2_batch_create: update rank must be in 1..31");
    const BlockTree& bt = Z->blocks;
    P->Z = Z;
    P->u = u;
    P->count = count;
    P->blocks.assign(blocks, blocks + count);
    P->offA.resize(count);
    P->offB.resize(count);
    P->rowsA.resize(count);
    P->rowsB.resize(count);
    for (int64_t j = 0; j < count; ++j) {
      H2_REQUIRE(blocks[j] >= 0 && blocks[j] < bt.count(), "h2_batch_create: block id out of range");
      P->rowsA[j] = Z->rows.size[bt.row[blocks[j]]];
      P->rowsB[j] = Z->cols.size[bt.col[blocks[j]]];
      P->offA[j] = offA ? offA[j] : P->lenA;
      P->offB[j] = offB ? offB[j] : P->lenB;
      P->lenA = std::max(P->lenA, P->offA[j] + P->rowsA[j] * u);
      P->lenB = std::max(P->lenB, P->offB[j] + P->rowsB[j] * u);
    }
    plan_batch(*P);
    if (!ctx) return;   // host-only plan
    H2_REQUIRE(has_storage(Z), "h2_batch_create: matrix has no device storage");
    DeviceGuard g(ctx->device);
    P->device = ctx->device;
    alloc_batch(ctx, *P);
  });
  if (s == H2_OK) *out = P.release();
  else if (ctx) free_batch_device(*P);   // partial allocations
  return s;
}
}  // namespace

extern "C" h2_status h2_batch_create(h2_ctx* ctx, const h2_matrix* Z, int64_t count, const int64_t* blocks,
                                     int u, h2_batch** out) {
  return create_batch(ctx, Z, count, blocks, u, nullptr, nullptr, out);
}

extern "C" void h2_batch_free(h2_batch* P) {
  if (!P) return;
  for (cudaEvent_t& e : P->ev)
    if (e) cudaEventDestroy(e);
  free_batch_device(*P);
  delete P;
}

extern "C" h2_status h2_batch_factor_layout(const h2_batch* P, int64_t j, int64_t* rows_A, int64_t* off_A,
                                            int64_t* rows_B, int64_t* off_B) {
  if (!P || j < 0 || j >= P->count) return H2_EINVAL;
  if (rows_A) *rows_A = P->rowsA[j];
  if (off_A) *off_A = P->offA[j];
  if (rows_B) *rows_B = P->rowsB[j];
  if (off_B) *off_B = P->offB[j];
  return H2_OK;
}

extern "C" h2_status h2_batch_factor_sizes(const h2_batch* P, int64_t* len_A, int64_t* len_B) {
  if (!P) return H2_EINVAL;
  if (len_A) *len_A = P->lenA;
  if (len_B) *len_B = P->lenB;
  return H2_OK;
}

extern "C" h2_status h2_batch_execute(h2_ctx* ctx, h2_batch* P, const double* A, const double* B, double eps) {
  if (!ctx || !P) return H2_EINVAL;
  return guard(ctx, [&] {
    H2_REQUIRE(P->d_items || P->items.empty(), "h2_batch_execute: plan has no device buffers");
    H2_REQUIRE((A || P->lenA == 0) && (B || P->lenB == 0), "h2_batch_execute: factors missing");
    H2_REQUIRE(std::isfinite(eps) && eps >= 0, "h2_batch_execute: eps must be finite and >= 0");
    DeviceGuard g(ctx->device);
    P->compact = false;
    execute(ctx, *P, A, B, eps);
  });
}


extern "C" h2_status h2_batch_result_size(const h2_batch* P, int64_t* len) {
  if (!P || !len) return H2_EINVAL;
  *len = P->res_len;
  return H2_OK;
}

extern "C" h2_status h2_batch_result_offsets(const h2_batch* P, int64_t* item_off, int64_t* task_off) {
  if (!P || (!item_off && !P->items.empty()) || (!task_off && !P->tasks.empty())) return H2_EINVAL;
  std::copy(P->res_item_off.begin(), P->res_item_off.end(), item_off);
  std::copy(P->res_task_off.begin(), P->res_task_off.end(), task_off);
  return H2_OK;
}

extern "C" h2_status h2_batch_task_info(const h2_batch* P, int64_t task, int32_t* info) {
  if (!P || !info || task < 0 || task >= (int64_t)P->tasks.size()) return H2_EINVAL;
  const Task& tk = P->tasks[task];
  info[0] = (int32_t)(std::upper_bound(P->upd_task.begin(), P->upd_task.end(), task) - P->upd_task.begin() - 1);
  info[1] = P->Z->blocks.adm[tk.slot];
  info[2] = tk.it;
  info[3] = tk.is;
  info[4] = tk.kt;
  info[5] = tk.ls;
  return H2_OK;
}

// Both host-result entry points; copied == nullptr: the full result.
static h2_status execute_host(h2_ctx* ctx, h2_batch* P, const double* A_host, const double* B_host, double eps,
                              double* result, int8_t* copied) {
  if (!ctx || !P || !result) return H2_EINVAL;
  return guard(ctx, [&] {
    H2_REQUIRE((A_host || P->lenA == 0) && (B_host || P->lenB == 0), "h2_batch_execute_host: factors missing");
    H2_REQUIRE(std::isfinite(eps) && eps >= 0, "h2_batch_execute_host: eps must be finite and >= 0");
    DeviceGuard g(ctx->device);
    P->compact = copied != nullptr;
    const int64_t n_tasks = (int64_t)P->tasks.size();
    P->h2d_bytes = (P->lenA + P->lenB) * (int64_t)sizeof(double);
    P->d2h_bytes = copied ? n_tasks : 0;
    cudaStream_t st = ctx->stream;
    if (!P->d_A && P->lenA) P->d_A = dalloc<double>(P->lenA);
    if (!P->d_B && P->lenB) P->d_B = dalloc<double>(P->lenB);
    alloc_result(*P, st);
    if (P->lenA) H2_CUDA(cudaMemcpyAsync(P->d_A, A_host, P->lenA * sizeof(double), cudaMemcpyHostToDevice, st));
    if (P->lenB) H2_CUDA(cudaMemcpyAsync(P->d_B, B_host, P->lenB * sizeof(double), cudaMemcpyHostToDevice, st));
    // a page-locked destination receives the result in copies that overlap
    // the update (part of the launch sequence); any other after it
    cudaPointerAttributes pa{};
    const bool pinned = P->res_len > 0 && cudaPointerGetAttributes(&pa, result) == cudaSuccess &&
                        pa.type == cudaMemoryTypeHost;
    (void)cudaGetLastError();
    if (pinned) {
      execute(ctx, *P, P->d_A, P->d_B, eps, result);
      P->launches += (P->mode != H2_MODE_EXACT && !P->compact) ? 2 : 1;   // the pack kernels
      H2_CUDA(cudaStreamSynchronize(st));
      check_device_error(ctx);
      if (P->mode != H2_MODE_EXACT) {
        // chunks of the early region that the late pass packed again
        const int64_t nch = (int64_t)P->res_chunk_off.size() - 1;
        P->d2h_bytes += nch * (int64_t)sizeof(int32_t) +
                        (P->compact ? P->res_prefix : P->res_len) * (int64_t)sizeof(double);
        bool again = false;
        for (int64_t c = 0; c < nch; ++c) {
          if (!P->h_flags[c]) continue;
          const int64_t a = P->res_chunk_off[c], b = P->res_chunk_off[c + 1];
          H2_CUDA(cudaMemcpyAsync(result + a, P->d_res + a, (b - a) * sizeof(double), cudaMemcpyDeviceToHost, st));
          P->d2h_bytes += (b - a) * (int64_t)sizeof(double);
          again = true;
        }
        if (again) H2_CUDA(cudaStreamSynchronize(st));
      } else {
        P->d2h_bytes += P->res_len * (int64_t)sizeof(double);
      }
      if (copied && !P->tasks.empty()) std::memcpy(copied, P->h_copy, P->tasks.size() * sizeof(int8_t));
    } else {
      execute(ctx, *P, P->d_A, P->d_B, eps);
      const int64_t n = (int64_t)P->tasks.size() + (int64_t)P->items.size();
      if (n > 0) {
        k_pack<<<pack_blocks(n), 32 * kPackWarps, 0, st>>>(view_of(P->Z), P->d_items, (int)P->items.size(),
                                                            P->d_tasks,
                                                            (int)P->tasks.size(), P->u, P->IB, P->d_res_task_off,
                                                            P->d_res_item_off, P->d_res);
        H2_CUDA(cudaGetLastError());
        P->launches += 1;
      }
      if (P->res_len)
        H2_CUDA(cudaMemcpyAsync(result, P->d_res, P->res_len * sizeof(double), cudaMemcpyDeviceToHost, st));
      P->d2h_bytes += P->res_len * (int64_t)sizeof(double);
      // a pageable destination receives every piece; the flags say which
      // pieces are copies all the same
      if (copied && !P->tasks.empty())
        H2_CUDA(cudaMemcpyAsync(copied, P->IB.copy, P->tasks.size() * sizeof(int8_t), cudaMemcpyDeviceToHost, st));
      H2_CUDA(cudaStreamSynchronize(st));
    }
    check_device_error(ctx);
  });
}

extern "C" h2_status h2_batch_execute_host(h2_ctx* ctx, h2_batch* P, const double* A_host, const double* B_host,
                                           double eps, double* result) {
  return execute_host(ctx, P, A_host, B_host, eps, result, nullptr);
}

extern "C" h2_status h2_batch_host_bytes(const h2_batch* P, int64_t* h2d, int64_t* d2h) {
  if (!P || !h2d || !d2h) return H2_EINVAL;
  *h2d = P->h2d_bytes;
  *d2h = P->d2h_bytes;
  return H2_OK;
}

extern "C" h2_status h2_batch_execute_host_compact(h2_ctx* ctx, h2_batch* P, const double* A_host,
                                                   const double* B_host, double eps, double* result, int8_t* copied) {
  if (!copied && P && !P->tasks.empty()) return H2_EINVAL;
  static int8_t none = 0;   // a batch without coupling tasks needs no flags
  return execute_host(ctx, P, A_host, B_host, eps, result, copied ? copied : &none);
}

namespace {
// Persistent device buffers of the commit's copy lists (the update engine);
// without them the lists are uploaded into fresh allocations.
struct CommitScratch {
  double wait_s = 0.0;    // time spent waiting for the ranks (the GPU work before them)
  CopyDesc* cd = nullptr;
  size_t c_cd = 0;
  NearDesc* nd = nullptr;
  size_t c_nd = 0;
  int* err = nullptr;     // page-locked copy of the device error word
};

void commit_update(h2_ctx* ctx, const h2_batch* P, int64_t j, const double* A, const double* B, h2_matrix* dst,
                   CommitScratch* sc) {
  H2_REQUIRE(P->executed, "h2_batch_apply: batch not executed");
  H2_REQUIRE(has_storage(dst), "h2_batch_apply: destination has no device storage");
  const h2_matrix* Z = P->Z;
  H2_REQUIRE(dst->rows.count() == Z->rows.count() && dst->blocks.count() == Z->blocks.count(),
             "h2_batch_apply: destination has another structure");
  DeviceGuard g(ctx->device);
  cudaStream_t st = ctx->stream;
  const int64_t i0 = P->upd_item[j], i1 = P->upd_item[j + 1];
  const int64_t t0 = P->upd_task[j], t1 = P->upd_task[j + 1];
  std::vector<int32_t> rk(i1 - i0);
  std::vector<int8_t> copy(t1 - t0);
  if (i1 > i0)
    H2_CUDA(cudaMemcpyAsync(rk.data(), P->IB.rank + i0, (i1 - i0) * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (t1 > t0)
    H2_CUDA(cudaMemcpyAsync(copy.data(), P->IB.copy + t0, (t1 - t0) * sizeof(int8_t), cudaMemcpyDeviceToHost, st));
  if (sc) {
    // one synchronisation: the error word comes back with the ranks
    H2_CUDA(cudaMemcpyAsync(sc->err, ctx->d_error, sizeof(int), cudaMemcpyDeviceToHost, st));
    const auto w0 = std::chrono::steady_clock::now();
    H2_CUDA(cudaStreamSynchronize(st));
    sc->wait_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - w0).count();
    if (*sc->err) check_device_error(ctx);
  } else {
    H2_CUDA(cudaStreamSynchronize(st));
    check_device_error(ctx);
  }
  int kmax = 0;
  for (int32_t r : rk) kmax = std::max(kmax, r);
  grow_kcap(ctx, dst, kmax);
  const int kcap = dst->kcap;
  std::vector<CopyDesc> cd;
  auto rank_of_item = [&](int32_t id) { return rk[id - i0]; };
  for (int64_t i = i0; i < i1; ++i) {
    const Item& it = P->items[i];
    DeviceBasis& db = basis_of(dst, it.side);
    const ClusterTree& ct = tree_of(dst, it.side);
    const int r = rank_of_item((int32_t)i);
    if ((it.flags & kItemLeaf) && r > 0)
      cd.push_back({P->IB.Q + it.qoff, db.d_leaf + db.leaf_off[it.cluster], it.size, r, it.size, it.size});
    if (!(it.flags & kItemTreeRoot)) {
      const int rf = (it.flags & kItemRoot) ? db.rank[ct.father[it.cluster]] : rank_of_item(it.parent);
      if (r > 0 && rf > 0)
        cd.push_back({P->IB.F + (size_t)i * kSlot, db.d_transfer + (size_t)it.cluster * kcap * kcap, r, rf, 32,
                      kcap});
    }
  }
  for (int64_t t = t0; t < t1; ++t) {
    const Task& tk = P->tasks[t];
    const int rt = tk.it >= 0 ? rank_of_item(tk.it) : tk.kt;
    const int rs = tk.is >= 0 ? rank_of_item(tk.is) : tk.ls;
    if (rt <= 0 || rs <= 0) continue;
    double* d = dst->d_S + (size_t)tk.slot * kcap * kcap;
    if (copy[t - t0]) {
      // [S_b; 0] or [S_b, 0]: the coupling of the planned matrix (the same
      // storage when dst is that matrix) and the zero rows or columns
      if (dst != Z && tk.kt > 0 && tk.ls > 0)
        cd.push_back({Z->d_S + (size_t)tk.slot * Z->kcap * Z->kcap, d, tk.kt, tk.ls, Z->kcap, kcap});
      if (tk.it >= 0)
        cd.push_back({nullptr, d + tk.kt, rt - tk.kt, rs, 0, kcap});
      else
        cd.push_back({nullptr, d + (size_t)tk.ls * kcap, rt, rs - tk.ls, 0, kcap});
      continue;
    }
    cd.push_back({P->IB.S_out + (size_t)t * kSlot, d, rt, rs, 32, kcap});
  }
  // nearfield leaves inside the block
  std::vector<NearDesc> nd;
  const BlockTree& bt = Z->blocks;
  const int32_t b0 = (int32_t)P->blocks[j];
  std::vector<int32_t> stack{b0};
  while (!stack.empty()) {
    const int32_t b = stack.back();
    stack.pop_back();
    if (bt.kind[b] == kSub) {
      for (int i = 3; i >= 0; --i)
        if (bt.son4[4 * b + i] >= 0) stack.push_back(bt.son4[4 * b + i]);
    } else if (bt.kind[b] == kNear) {
      const int32_t t = bt.row[b], s = bt.col[b];
      const int64_t ro = Z->rows.off[t] - Z->rows.off[bt.row[b0]];
      const int64_t co = Z->cols.off[s] - Z->cols.off[bt.col[b0]];
      NearDesc d{};
      d.N = dst->d_N + dst->near_off[bt.slot[b]];
      d.A = A + P->offA[j] + ro;
      d.B = B + P->offB[j] + co;
      d.rows = (int)Z->rows.size[t];
      d.cols = (int)Z->cols.size[s];
      d.ldn = d.rows;
      d.lda = (int)P->rowsA[j];
      d.ldb = (int)P->rowsB[j];
      nd.push_back(d);
    }
  }
  H2_REQUIRE(nd.empty() || (A && B), "h2_batch_apply: factors needed for the nearfield part");
  CopyDesc* dcd = nullptr;
  NearDesc* dnd = nullptr;
  if (sc) {
    // persistent lists; pageable sources are staged before the calls return
    if (cd.size() > sc->c_cd) {
      dfree(sc->cd);
      sc->c_cd = std::max(cd.size(), 2 * sc->c_cd);
      sc->cd = dalloc<CopyDesc>(sc->c_cd);
    }
    if (nd.size() > sc->c_nd) {
      dfree(sc->nd);
      sc->c_nd = std::max(nd.size(), 2 * sc->c_nd);
      sc->nd = dalloc<NearDesc>(sc->c_nd);
    }
    dcd = sc->cd;
    dnd = sc->nd;
    if (!cd.empty())
      H2_CUDA(cudaMemcpyAsync(dcd, cd.data(), cd.size() * sizeof(CopyDesc), cudaMemcpyHostToDevice, st));
    if (!nd.empty())
      H2_CUDA(cudaMemcpyAsync(dnd, nd.data(), nd.size() * sizeof(NearDesc), cudaMemcpyHostToDevice, st));
  } else {
    dcd = upload(cd, st);
    try {
      dnd = upload(nd, st);
    } catch (...) {
      dfree(dcd);
      throw;
    }
  }
  launch_copy(dcd, (int)cd.size(), st);
  launch_near_add(dnd, (int)nd.size(), P->u, st);
  H2_CUDA(cudaGetLastError());
  for (int64_t i = i0; i < i1; ++i) {
    const Item& it = P->items[i];
    basis_of(dst, it.side).rank[it.cluster] = rank_of_item((int32_t)i);
  }
  sync_ranks(dst->V, st);
  sync_ranks(dst->W, st);
  if (!sc) {
    H2_CUDA(cudaStreamSynchronize(st));
    dfree(dcd);
    dfree(dnd);
  }
}
}  // namespace

extern "C" h2_status h2_batch_apply(h2_ctx* ctx, const h2_batch* P, int64_t j, const double* A, const double* B,
                                    h2_matrix* dst) {
  if (!ctx || !P || !dst || j < 0 || j >= P->count) return H2_EINVAL;
  return guard(ctx, [&] { commit_update(ctx, P, j, A, B, dst, nullptr); });
}

namespace {

// Algorithmic float64 flops per phase of the last execution (standard
// counts: Householder QR 2mn^2 - 2n^3/3, products 2mnk with triangular
// factors halved, symmetric products on their lower triangle, one-sided
// Jacobi 6m per pair checked plus 6m per rotation as counted on the device).
// The certified path counts for every update (it runs for all of them), the
// exact path for the updates it recomputed and the clusters it marked.
void phase_flops(h2_ctx* ctx, const h2_batch* P, double f[H2_PHASE_COUNT]) {
  for (int ph = 0; ph < H2_PHASE_COUNT; ++ph) f[ph] = 0.0;
  const size_t ni = P->items.size();
  std::vector<unsigned long long> jac(4 * ni);
  std::vector<int32_t> rk(ni);
  std::vector<int32_t> fail(P->count, 1);
  if (ni) {
    H2_CUDA(cudaMemcpyAsync(jac.data(), P->IB.jac, 4 * ni * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                            ctx->stream));
    H2_CUDA(cudaMemcpyAsync(rk.data(), P->IB.rank, ni * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (P->count)
    H2_CUDA(cudaMemcpyAsync(fail.data(), P->IB.fail, P->count * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            ctx->stream));
  std::vector<int32_t> orth[2];
  const bool gram = P->mode != H2_MODE_EXACT;
  for (int sd = 0; sd < 2; ++sd) {
    orth[sd].assign(tree_of(P->Z, sd).count(), 0);
    if (gram && !orth[sd].empty())
      H2_CUDA(cudaMemcpyAsync(orth[sd].data(), P->BW.orth[sd], orth[sd].size() * sizeof(int32_t),
                              cudaMemcpyDeviceToHost, ctx->stream));
  }
  H2_CUDA(cudaStreamSynchronize(ctx->stream));
  const double u = P->u;
  auto qr = [](double m, double n) {
    return m >= n ? 2 * m * n * n - 2.0 / 3.0 * n * n * n : 2 * n * m * m - 2.0 / 3.0 * m * m * m;
  };
  auto tri = [](double n) { return n * (n + 1) / 2; };
  // LDL^*: per pivot the scaled column and the symmetric trailing update
  auto ldl = [&](double n) {
    double x = 0;
    for (double m = n - 1; m >= 0; m -= 1) x += m + 2 * tri(m);
    return x;
  };
  const h2_matrix* Z = P->Z;
  // fold of ch rows into an upper n x n factor: 2 ch n^2 (Householder)
  auto fold = [](double ch, double n) { return 2.0 * ch * n * n; };
  // clusters whose weights of the unchanged matrix the exact path computed
  std::vector<char> need[2];
  for (int sd = 0; sd < 2; ++sd) need[sd].assign(tree_of(Z, sd).count(), gram ? 0 : 1);
  if (gram)
    for (size_t i = 0; i < ni; ++i) {
      const Item& it = P->items[i];
      if (!fail[it.update]) continue;
      for (int32_t c = it.cluster; c >= 0; c = tree_of(Z, it.side).father[c]) need[it.side][c] = 1;
    }
  for (int sd = 0; sd < 2; ++sd) {
    const ClusterTree& ct = tree_of(Z, sd);
    const DeviceBasis& bs = basis_of(Z, sd);
    const DeviceBasis& o = basis_of(Z, 1 - sd);
    const std::vector<int32_t>& ptr = sd == 0 ? Z->blocks.row_ptr : Z->blocks.col_ptr;
    const std::vector<int32_t>& adm = sd == 0 ? Z->blocks.row_adm : Z->blocks.col_adm;
    for (int32_t c = 0; c < ct.count(); ++c) {
      const double k = bs.rank[c];
      if (gram) {
        // local orthonormality test (V_c^* V_c or sum E_s^* E_s), and
        // V_c^* V_c by the recursion for clusters that are not orthonormal
        const bool oc = orth[sd][c] != 0;
        if (ct.leaf(c)) {
          f[H2_PHASE_BASE_WEIGHTS] += (oc ? 2 : 4) * tri(k) * (double)ct.size[c];
        } else {
          for (int32_t sn : {ct.son0[c], ct.son1[c]}) {
            const double ks = bs.rank[sn];
            f[H2_PHASE_BASE_WEIGHTS] += 2 * tri(k) * ks;
            if (!oc) f[H2_PHASE_BASE_WEIGHTS] += orth[sd][sn] ? 2 * tri(k) * ks : 2 * ks * ks * k + 2 * tri(k) * ks;
          }
        }
      }
      for (int32_t e = ptr[c]; e < ptr[c + 1]; ++e) {
        const int32_t blk = Z->blocks.adm[adm[e]];
        const double l = o.rank[sd == 0 ? Z->blocks.col[blk] : Z->blocks.row[blk]];
        if (gram) f[H2_PHASE_BASE_WEIGHTS] += 2 * k * l + 2 * tri(k) * l + 2 * tri(k);
        if (need[sd][c]) f[H2_PHASE_EXACT] += 2 * k * l + fold(l, k);   // norm, fold
      }
      if (ct.father[c] >= 0) {
        const double kf = bs.rank[ct.father[c]];
        if (gram) f[H2_PHASE_BASE_WEIGHTS] += 2 * k * kf * kf + 2 * tri(k) * kf;
        if (need[sd][c]) f[H2_PHASE_EXACT] += kf * kf * k + fold(kf, k);
      }
    }
  }
  for (const NormTask& nt : P->norms) {
    const double kt = P->items[nt.it].k, ls = P->items[nt.is].k;
    const double Kt = kt + u, Ks = ls + u;
    if (gram) {
      if (orth[0][P->items[nt.it].cluster] && orth[1][P->items[nt.is].cluster])
        f[H2_PHASE_NORMS] += 2 * kt * ls + 2 * kt * u * ls + 2 * kt * u + 2 * u * u;   // ||S||, <C_t, S C_s>, <N_t, N_s>
      else
        f[H2_PHASE_NORMS] += 2 * Kt * ls * kt + 2 * kt * Ks * ls + 2 * Kt * Ks;
    }
    if (fail[P->items[nt.it].update]) f[H2_PHASE_EXACT] += 2 * kt * ls * Ks + Kt * Kt * Ks + 2 * Kt * Ks;
  }
  for (size_t i = 0; i < ni; ++i) {
    const Item& it = P->items[i];
    const double k = it.k, K = it.k + u;
    const bool leaf = it.flags & kItemLeaf;
    const bool root = it.flags & kItemRoot;
    const bool troot = it.flags & kItemTreeRoot;
    const double kf = it.kf;
    if (gram) {
      // step 2: C_t and N_t of the basis Gram matrices
      if (leaf) {
        f[H2_PHASE_RFACTOR] += 2 * (k * u + tri(u)) * it.size;
      } else {
        for (int32_t sid : {it.son0, it.son1}) {
          const double ks = P->items[sid].k;
          f[H2_PHASE_RFACTOR] += 2 * k * u * ks + tri(u);
        }
      }
      // step 3: weight Gram matrices (jac[3] = 1: V_t not orthonormal)
      const bool orth_w = jac[4 * i + 3] == 0;
      for (int32_t e = it.ent_begin; e < it.ent_end; ++e) {
        const Entry& en = P->ents[e];
        const double l = basis_of(Z, 1 - it.side).rank[en.other_cluster];
        if (en.other >= 0) {
          if (orth_w) f[H2_PHASE_WEIGHTS] += 2 * k * l;   // ||S_b|| for the base term
          if (orth[1 - it.side][P->items[en.other].cluster]) {
            // S' S'^* (shared with the base term), C_o^* S'^*, N_o
            f[H2_PHASE_WEIGHTS] += 2 * tri(k) * l + 2 * tri(k) + 2 * u * k * l + 2 * tri(u);
          } else {
            if (orth_w) f[H2_PHASE_WEIGHTS] += 2 * tri(k) * l + 2 * tri(k);
            f[H2_PHASE_WEIGHTS] += 2 * k * (l + u) * l + 2 * (k * K - tri(k - 1)) * l + 2 * tri(K);
          }
        } else if (!orth_w) {
          f[H2_PHASE_WEIGHTS] += 2 * k * k * l + 2 * k * l + 2 * tri(k) * l + 2 * tri(k);
        }
      }
      if (root && !troot) {
        f[H2_PHASE_WEIGHTS] += 2 * k * kf * kf + 2 * tri(k) * kf;
      } else if (!root) {
        f[H2_PHASE_WEIGHTS] += 2 * k * (kf + u) * kf + 2 * (k * K - tri(k - 1)) * kf;
      }
      // step 4: certificate (LDL^* of G_t, W L, L^* (W L), LDL^* of the
      // certificate matrix) and new bases; block formulas for an orthonormal V_t
      const bool ob = orth[it.side][it.cluster] != 0;
      if (ob) {
        // S = N - C^* C, LDL^*(S); Y = W21 + W22 C^*, Z = W22 L_S; C2_11 =
        // W11 + W12 C^* + C Y, C2_21 = L_S^* Y, C2_22 = L_S^* Z; LDL^*(C2)
        double c2 = 4 * tri(k) * u;
        for (double a = 0; a < u; a += 1) c2 += 2 * (k + a + 1) * (u - a);
        f[H2_PHASE_TRUNCATE] += 2 * tri(u) * k + ldl(u) + 2 * u * k * u + 2 * u * tri(u) + c2;
      } else {
        f[H2_PHASE_TRUNCATE] += ldl(K) + 2 * K * tri(K) + (K * K * K + 3 * K * K + 2 * K) / 3;
      }
      // certificate: float64 shift and scaling of the lower triangle for the
      // float32 factorisation (float32 flops not counted), plus the float64
      // factorisation where the float32 one did not prove it (jac[0] = 1)
      f[H2_PHASE_TRUNCATE] += 2 * tri(K) + (!fail[it.update] && jac[4 * i] ? ldl(K) : 0.0);
      if (!fail[it.update]) {
        if (leaf) f[H2_PHASE_BASES] += ob ? 2.0 * it.size * (k * u + tri(u)) : (double)it.size * K * K;
        if (!troot && !(root && ob)) {
          const bool op = orth[it.side][tree_of(Z, it.side).father[it.cluster]] != 0;
          if (root)
            f[H2_PHASE_BASES] += 2 * tri(k) * kf;
          else if (ob && op)
            f[H2_PHASE_BASES] += 2 * k * kf * u + K * u * u;
          else
            f[H2_PHASE_BASES] += 2 * tri(k) * kf + K * (kf + u) * (kf + u);
        }
      }
    }
    if (!fail[it.update]) continue;
    // exact path
    if (leaf) {
      f[H2_PHASE_EXACT] += qr(it.size, K);
    } else {
      const double k0 = P->items[it.son0].k, k1 = P->items[it.son1].k;
      f[H2_PHASE_EXACT] += (k0 + u) * k0 * k + (k1 + u) * k1 * k + qr(k0 + k1 + 2 * u, K);
    }
    // weights: outside blocks folded into k columns by the task itself when
    // some block lies inside the update (otherwise the precomputed G_t), then
    // the inside blocks and the father's part folded into K columns
    if (it.flags & kItemInside) {
      for (int32_t e = it.ent_begin; e < it.ent_end; ++e) {
        const Entry& en = P->ents[e];
        if (en.other < 0) {
          const double l = basis_of(Z, 1 - it.side).rank[en.other_cluster];
          f[H2_PHASE_EXACT] += 2 * k * l + fold(l, k);
        } else {
          const double l = P->items[en.other].k;
          f[H2_PHASE_EXACT] += (l + u) * l * k + fold(l + u, K);
        }
      }
    }
    if (!troot) {
      const double kfx = root ? kf : kf + u;
      f[H2_PHASE_EXACT] += kfx * kf * k + fold(kfx, K);
    }
    // truncation
    const double m = leaf ? it.size : rk[it.son0] + rk[it.son1];
    double ft = 0;
    if (!leaf) {
      const double k0 = P->items[it.son0].k, k1 = P->items[it.son1].k;
      ft += 2 * rk[it.son0] * k0 * k + 2 * rk[it.son1] * k1 * k;
    }
    ft += m * K * K;                                               // V^ times triangular B~^*
    if (jac[4 * i + 2]) {
      // certificate factorisation used as the first Cholesky-QR pass, then a
      // polish: 2 Grams, 1 factorisation, 1 triangular inverse, 1
      // triangular product, 1 product
      ft += 2 * (2 * m * K * K) + (K * K * K / 3) + (K * K * K / 3) + (m * K * K) + 2 * m * K * K;
    } else {
      if (K >= 2 && m > 0) ft += 2 * (4 * K * K * K) + 2 * m * K * K;  // Newton-Schulz (2 steps), M V
      ft += 6.0 * m * (double)jac[4 * i] + 6.0 * m * (double)jac[4 * i + 1];
    }
    ft += 2 * m * K * rk[i];                                       // R_t = Q^* V^
    if (root && !troot) ft += 2 * rk[i] * k * kf;
    f[H2_PHASE_EXACT] += ft;
  }
  for (const Task& tk : P->tasks) {
    const double kt = tk.kt, ls = tk.ls;
    if (!fail[P->items[tk.it >= 0 ? tk.it : tk.is].update]) {
      // certified update: R_t = L_t^* upper triangular, products over the
      // triangle; one-sided blocks of an orthonormal basis are copies
      if (tk.it >= 0 && tk.is >= 0) {
        f[H2_PHASE_REPROJECT] += 2.0 * kt * tri(ls) + 2.0 * tri(kt + u) * (ls + u);
      } else if (tk.it >= 0) {
        if (!orth[0][P->items[tk.it].cluster]) f[H2_PHASE_REPROJECT] += 2.0 * tri(kt) * ls;
      } else {
        if (!orth[1][P->items[tk.is].cluster]) f[H2_PHASE_REPROJECT] += 2.0 * kt * tri(ls);
      }
      continue;
    }
    if (tk.it >= 0 && tk.is >= 0)
      f[H2_PHASE_REPROJECT] += 2.0 * (kt + u) * ls * rk[tk.is] + 2.0 * rk[tk.it] * (kt + u) * rk[tk.is];
    else if (tk.it >= 0)
      f[H2_PHASE_REPROJECT] += 2.0 * rk[tk.it] * kt * ls;
    else
      f[H2_PHASE_REPROJECT] += 2.0 * kt * ls * rk[tk.is];
  }
}

}  // namespace

extern "C" h2_status h2_batch_stats(h2_ctx* ctx, const h2_batch* P, int64_t* n_cluster_tasks,
                                    int64_t* n_block_tasks, int64_t* n_launches, double* flops) {
  if (!P) return H2_EINVAL;
  return guard(ctx, [&] {
    if (n_cluster_tasks) *n_cluster_tasks = (int64_t)P->items.size();
    if (n_block_tasks) *n_block_tasks = (int64_t)P->tasks.size();
    if (n_launches) *n_launches = P->launches;
    if (!flops) return;
    H2_REQUIRE(ctx && P->executed, "h2_batch_stats: flops need an executed batch and a context");
    DeviceGuard g(ctx->device);
    double f[H2_PHASE_COUNT];
    phase_flops(ctx, P, f);
    double tot = 0;
    for (double x : f) tot += x;
    *flops = tot;
  });
}

extern "C" h2_status h2_batch_set_timing(h2_batch* P, int on) {
  if (!P) return H2_EINVAL;
  return guard(nullptr, [&] {
    if (on && !P->ev[0]) {
      DeviceGuard g(P->device);
      for (cudaEvent_t& e : P->ev) H2_CUDA(cudaEventCreate(&e));
    }
    P->timing = on == 2 ? 2 : (on != 0 ? 1 : 0);
  });
}

extern "C" h2_status h2_batch_set_mode(h2_batch* P, int mode) {
  if (!P || (mode != H2_MODE_AUTO && mode != H2_MODE_EXACT)) return H2_EINVAL;
  P->mode = mode;
  return H2_OK;
}

extern "C" h2_status h2_batch_paths(h2_ctx* ctx, const h2_batch* P, int32_t* exact) {
  if (!ctx || !P || (P->count > 0 && !exact)) return H2_EINVAL;
  return guard(ctx, [&] {
    H2_REQUIRE(P->executed, "h2_batch_paths: batch not executed");
    DeviceGuard g(ctx->device);
    if (P->count)
      H2_CUDA(cudaMemcpyAsync(exact, P->IB.fail, P->count * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    H2_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int64_t j = 0; j < P->count; ++j) exact[j] = exact[j] != 0;
  });
}

extern "C" h2_status h2_batch_phase_stats(h2_ctx* ctx, const h2_batch* P, int phase, int64_t* launches,
                                          double* ms, double* flops) {
  if (!ctx || !P || phase < 0 || phase >= H2_PHASE_COUNT) return H2_EINVAL;
  return guard(ctx, [&] {
    H2_REQUIRE(P->executed, "h2_batch_phase_stats: batch not executed");
    DeviceGuard g(ctx->device);
    if (launches) *launches = P->phase_launches[phase];
    if (ms) {
      *ms = -1.0;
      const bool gram_phase = phase != H2_PHASE_EXACT && phase != H2_PHASE_REPROJECT;
      if (P->timing && P->ev[0] && gram_phase && P->mode == H2_MODE_EXACT) {
        *ms = 0.0;   // the certified path did not run
      } else if (P->timing && P->ev[0]) {
        H2_CUDA(cudaEventSynchronize(P->ev[2 * phase + 1]));
        float t = 0;
        H2_CUDA(cudaEventElapsedTime(&t, P->ev[2 * phase], P->ev[2 * phase + 1]));
        *ms = t;
      }
    }
    if (flops) {
      double f[H2_PHASE_COUNT];
      phase_flops(ctx, P, f);
      *flops = f[phase];
    }
  });
}

extern "C" h2_status h2_batch_item_info(const h2_batch* P, int64_t item, int32_t* info) {
  if (!P || !info || item < 0 || item >= (int64_t)P->items.size()) return H2_EINVAL;
  const Item& it = P->items[item];
  int64_t j = std::upper_bound(P->upd_item.begin(), P->upd_item.end(), item) - P->upd_item.begin() - 1;
  info[0] = (int32_t)j;
  info[1] = it.side;
  info[2] = it.cluster;
  info[3] = it.k;
  info[4] = -1;
  if (P->executed) {
    int32_t r = -1;
    if (cudaMemcpy(&r, P->IB.rank + item, sizeof(int32_t), cudaMemcpyDeviceToHost) == cudaSuccess) info[4] = r;
  }
  info[5] = it.flags;
  info[6] = 0;
  info[7] = 0;
  return H2_OK;
}

extern "C" h2_status h2_batch_item_tile(h2_ctx* ctx, const h2_batch* P, int64_t item, int which, double* out) {
  if (!ctx || !P || !out || item < 0 || item >= (int64_t)P->items.size() || which < 0 || which > 2)
    return H2_EINVAL;
  return guard(ctx, [&] {
    H2_REQUIRE(P->executed, "h2_batch_item_tile: batch not executed");
    DeviceGuard g(ctx->device);
    const Item& it = P->items[item];
    int32_t exact = 1;
    if (P->count)
      H2_CUDA(cudaMemcpyAsync(&exact, P->IB.fail + it.update, sizeof(int32_t), cudaMemcpyDeviceToHost,
                              ctx->stream));
    H2_CUDA(cudaStreamSynchronize(ctx->stream));
    // which 0, 1: the certified path stores the Gram matrices themselves, the
    // exact path R-factors (returned as R^* R)
    const double* src = which == 2 ? P->IB.Rt
                        : exact    ? (which == 0 ? P->IB.Rq : P->IB.Bw)
                                   : (which == 0 ? P->IB.Gv : P->IB.Wg);
    src += (size_t)item * kSlot;
    std::vector<double> tile(kSlot);
    H2_CUDA(cudaMemcpyAsync(tile.data(), src, kSlot * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    H2_CUDA(cudaStreamSynchronize(ctx->stream));
    if (which == 2 || (which == 1 && !exact)) {
      // only the (k+u) x (k+u) part (R_t: its first k+u columns) is written
      const int K = it.k + P->u;
      for (int j = 0; j < 32; ++j)
        for (int i = 0; i < 32; ++i)
          out[i + j * 32] = (j >= K || (which == 1 && i >= K)) ? 0.0 : tile[i + j * 32];
      return;
    }
    if (!exact) {
      // basis Gram: the V_t^* V_t block comes from the unchanged basis (the
      // identity where the basis is orthonormal; only the others have a slot)
      std::vector<double> vg(kSlot, 0.0);
      int32_t orth = 0;
      H2_CUDA(cudaMemcpyAsync(&orth, P->BW.orth[it.side] + it.cluster, sizeof(int32_t), cudaMemcpyDeviceToHost,
                              ctx->stream));
      H2_CUDA(cudaStreamSynchronize(ctx->stream));
      if (orth) {
        for (int i = 0; i < 32; ++i) vg[i * 33] = 1.0;
      } else {
        H2_CUDA(cudaMemcpyAsync(vg.data(), P->BW.Vg[it.side] + (size_t)it.cluster * kSlot, kSlot * sizeof(double),
                                cudaMemcpyDeviceToHost, ctx->stream));
        H2_CUDA(cudaStreamSynchronize(ctx->stream));
      }
      const int K = it.k + P->u;
      for (int j = 0; j < 32; ++j)
        for (int i = 0; i < 32; ++i)
          out[i + j * 32] = (i >= K || j >= K) ? 0.0 : (i < it.k && j < it.k) ? vg[i + j * 32] : tile[i + j * 32];
      return;
    }
    const int K = it.k + P->u;
    for (int j = 0; j < 32; ++j)
      for (int i = 0; i < 32; ++i) {
        double g = 0.0;
        if (i < K && j < K)
          for (int q = 0; q < 32; ++q) g += tile[q + i * 32] * tile[q + j * 32];
        out[i + j * 32] = g;
      }
  });
}

extern "C" h2_status h2_batch_update_items(const h2_batch* P, int64_t j, int64_t* first, int64_t* last) {
  if (!P || j < 0 || j >= P->count) return H2_EINVAL;
  if (first) *first = P->upd_item[j];
  if (last) *last = P->upd_item[j + 1];
  return H2_OK;
}

// ============================================================ single update
// ========================================== reusable single-update engine
// In-place local low-rank updates one at a time on persistent device
// buffers (grown on demand, never shrunk), through the exact path (every
// update of a factorisation truncates), with the weights of the unchanged
// matrix computed only for the clusters the update reads: the subtrees
// T_t0, T_s0 and their ancestors.  The work of one update is then
// proportional to #T_t0 + #T_s0 plus the depth (Section 5), instead of
// the whole tree of an isolated batch.  Used by the H^2-LR driver.
namespace h2 {

struct UpdateEngine {
  h2_batch* P = nullptr;
  CommitScratch cs;
  size_t c_items = 0, c_ents = 0, c_tasks = 0, c_two = 0, c_norms = 0, c_lvl = 0, c_cl = 0, c_bl = 0, c_q = 0;
  // The weights of the unchanged matrix kept between updates: G_t (the
  // R-factor of the weighted blocks of t's block row) and B~_t (of the
  // whole weight stack) of matrix wz stay in the device buffers and are
  // valid where g_ok / b_ok is set.
  const h2_matrix* wz = nullptr;
  std::vector<uint8_t> g_ok[2], b_ok[2];
  size_t c_A = 0, c_B = 0;
  int32_t c_ncl[2] = {0, 0};
  int64_t updates = 0;
  double plan_s = 0.0, launch_s = 0.0, total_s = 0.0;   // host planning, enqueue of the kernels, whole call
};

template <typename T>
static void ensure(T*& p, size_t& cap, size_t need) {
  if (p && need <= cap) return;
  if (p) cudaFree(p);
  p = nullptr;
  cap = std::max<size_t>(std::max<size_t>(need, 1), cap + cap / 2);
  p = dalloc<T>(cap);
}

template <typename T>
static void put(T* dst, const std::vector<T>& v, cudaStream_t st) {
  // pageable source: staged before the call returns
  if (!v.empty()) H2_CUDA(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
}


void zero_matrix(h2_ctx* ctx, h2_matrix* Z) {
  H2_REQUIRE(has_storage(Z), "zero_matrix: matrix has no device storage");
  DeviceGuard g(ctx->device);
  cudaStream_t st = ctx->stream;
  for (int sd = 0; sd < 2; ++sd) {
    const ClusterTree& ct = tree_of(Z, sd);
    DeviceBasis& b = basis_of(Z, sd);
    int64_t tot = 0;
    for (int32_t c = 0; c < ct.count(); ++c)
      if (ct.leaf(c)) tot += ct.size[c] * Z->kcap;
    if (tot) H2_CUDA(cudaMemsetAsync(b.d_leaf, 0, tot * sizeof(double), st));
    H2_CUDA(cudaMemsetAsync(b.d_transfer, 0, (size_t)ct.count() * Z->kcap * Z->kcap * sizeof(double), st));
    b.rank.assign(ct.count(), 0);
    sync_ranks(b, st);
  }
  const size_t nadm = Z->blocks.adm.size();
  if (nadm) H2_CUDA(cudaMemsetAsync(Z->d_S, 0, nadm * Z->kcap * Z->kcap * sizeof(double), st));
  if (Z->near_len) H2_CUDA(cudaMemsetAsync(Z->d_N, 0, Z->near_len * sizeof(double), st));
  // the host ranks are the source of the device copy: keep them alive until
  // the copy ran
  H2_CUDA(cudaStreamSynchronize(st));
}

UpdateEngine* engine_new() { return new UpdateEngine(); }

void engine_touch(UpdateEngine* E, const h2_matrix* Z, int32_t b0) {
  if (!E || E->wz != Z || E->g_ok[0].empty()) return;
  const BlockTree& bt = Z->blocks;
  const ClusterTree* tr[2] = {&Z->rows, &Z->cols};
  const int32_t c0[2] = {bt.row[b0], bt.col[b0]};
  std::vector<int32_t> dirty[2];
  for (int sd = 0; sd < 2; ++sd) {
    const ClusterTree& ct = *tr[sd];
    // the subtree: its bases, transfers and every coupling of its block
    // rows (columns) change
    for (int32_t c = c0[sd]; c < c0[sd] + ct.subtree[c0[sd]]; ++c) dirty[sd].push_back(c);
    // the other side's clusters of the blocks whose row (column) lies in
    // the subtree: their couplings are reprojected
    const std::vector<int32_t>& ptr = sd == 0 ? bt.row_ptr : bt.col_ptr;
    const std::vector<int32_t>& adm = sd == 0 ? bt.row_adm : bt.col_adm;
    for (int32_t c = c0[sd]; c < c0[sd] + ct.subtree[c0[sd]]; ++c)
      for (int32_t e = ptr[c]; e < ptr[c + 1]; ++e) {
        const int32_t b = bt.adm[adm[e]];
        dirty[1 - sd].push_back(sd == 0 ? bt.col[b] : bt.row[b]);
      }
  }
  for (int sd = 0; sd < 2; ++sd) {
    const ClusterTree& ct = *tr[sd];
    for (int32_t c : dirty[sd]) {
      E->g_ok[sd][c] = 0;
      // B~ of c and of everything below it depends on G_c
      for (int32_t d = c; d < c + ct.subtree[c]; ++d) E->b_ok[sd][d] = 0;
    }
  }
}

void engine_delete(UpdateEngine* E) {
  if (!E) return;
  if (E->P) h2_batch_free(E->P);   // synchronizes its streams
  dfree(E->cs.cd);
  dfree(E->cs.nd);
  if (E->cs.err) cudaFreeHost(E->cs.err);
  delete E;
}

int64_t engine_updates(const UpdateEngine* E) { return E ? E->updates : 0; }

void engine_times(const UpdateEngine* E, double* plan, double* launch, double* wait, double* total) {
  *plan = E ? E->plan_s : 0.0;
  *launch = E ? E->launch_s : 0.0;
  *wait = E ? E->cs.wait_s : 0.0;
  *total = E ? E->total_s : 0.0;
}

void engine_update(h2_ctx* ctx, h2_matrix* Z, UpdateEngine* E, int32_t block, int u, const double* A, int64_t lda,
                   const double* B, int64_t ldb, double eps, int max_rank) {
  H2_REQUIRE(u >= 1 && u < kMaxCols, "update rank must be in 1..31");
  using clk = std::chrono::steady_clock;
  const auto c0 = clk::now();
  cudaStream_t st = ctx->stream;
  if (!E->P) {
    E->P = new h2_batch();
    h2_batch& P = *E->P;
    P.device = ctx->device;
    H2_CUDA(cudaStreamCreateWithFlags(&P.side, cudaStreamNonBlocking));
    H2_CUDA(cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming));
    H2_CUDA(cudaEventCreateWithFlags(&P.join, cudaEventDisableTiming));
    H2_CUDA(cudaStreamCreateWithFlags(&P.side2, cudaStreamNonBlocking));
    H2_CUDA(cudaStreamCreateWithFlags(&P.cap, cudaStreamNonBlocking));
    H2_CUDA(cudaEventCreateWithFlags(&P.join2, cudaEventDisableTiming));
  }
  h2_batch& P = *E->P;
  const BlockTree& bt = Z->blocks;
  const ClusterTree* tr[2] = {&Z->rows, &Z->cols};
  // host plan of one update (the planner appends to these lists)
  P.Z = Z;
  P.u = u;
  P.count = 1;
  P.blocks.assign(1, block);
  P.rowsA.assign(1, Z->rows.size[bt.row[block]]);
  P.rowsB.assign(1, Z->cols.size[bt.col[block]]);
  P.offA.assign(1, 0);
  P.offB.assign(1, 0);
  P.lenA = P.rowsA[0] * u;
  P.lenB = P.rowsB[0] * u;
  P.items.clear();
  P.ents.clear();
  P.tasks.clear();
  P.norms.clear();
  plan_batch(P);
  P.mode = H2_MODE_EXACT;
  P.max_rank = max_rank;
  const auto c1 = clk::now();
  E->plan_s += std::chrono::duration<double>(c1 - c0).count();
  // the weights of the unchanged matrix the update reads, only where the
  // cache lacks them: G_t of the subtrees' clusters, B~ of the ancestors
  // (the subtree root's father and up), and G of an ancestor whose B~ is
  // recomputed
  {
    if (E->wz != Z || E->g_ok[0].size() != (size_t)tr[0]->count() ||
        E->g_ok[1].size() != (size_t)tr[1]->count()) {
      for (int sd = 0; sd < 2; ++sd) {
        E->g_ok[sd].assign(tr[sd]->count(), 0);
        E->b_ok[sd].assign(tr[sd]->count(), 0);
      }
      E->wz = Z;
    }
    const int L = P.depth + 1;
    std::vector<std::vector<int32_t>> gby(L), bby(L);
    for (int sd = 0; sd < 2; ++sd) {
      const ClusterTree& ct = *tr[sd];
      const int32_t root = sd == 0 ? bt.row[block] : bt.col[block];
      for (int32_t c = root; c < root + ct.subtree[root]; ++c)
        if (!E->g_ok[sd][c]) gby[ct.level[c]].push_back((sd << 30) | c);
      for (int32_t a = ct.father[root]; a >= 0; a = ct.father[a])
        if (!E->b_ok[sd][a]) {
          bby[ct.level[a]].push_back((sd << 30) | a);
          if (!E->g_ok[sd][a]) gby[ct.level[a]].push_back((sd << 30) | a);
        }
    }
    auto flatten = [&](std::vector<std::vector<int32_t>>& by, std::vector<int32_t>& list, std::vector<int32_t>& ptr) {
      ptr.assign(L + 1, 0);
      list.clear();
      for (int l = 0; l < L; ++l) {
        list.insert(list.end(), by[l].begin(), by[l].end());
        ptr[l + 1] = (int32_t)list.size();
      }
    };
    flatten(gby, P.cl_list, P.cl_ptr);
    flatten(bby, P.bl_list, P.bl_ptr);
  }
  // device buffers
  const size_t ni = P.items.size(), nt = P.tasks.size();
  const size_t prev_items = E->c_items, prev_tasks = E->c_tasks;
  ensure(P.d_items, E->c_items, ni);
  if (E->c_items != prev_items) {   // the per-item buffers follow the item capacity
    const size_t c = E->c_items;
    for (double** b : {&P.IB.Rq, &P.IB.Bw, &P.IB.Gv, &P.IB.Wg, &P.IB.Rt, &P.IB.F}) {
      dfree(*b);
      *b = dalloc<double>(c * kSlot);
    }
    dfree(P.IB.rank);
    dfree(P.IB.own);
    dfree(P.IB.jac);
    P.IB.rank = dalloc<int32_t>(c);
    P.IB.own = dalloc<int32_t>(c);
    P.IB.jac = dalloc<unsigned long long>(4 * c);
  }
  ensure(P.d_ents, E->c_ents, P.ents.size());
  ensure(P.d_tasks, E->c_tasks, nt);
  if (E->c_tasks != prev_tasks) {
    const size_t c = E->c_tasks;
    dfree(P.d_left);
    dfree(P.IB.S_out);
    dfree(P.IB.copy);
    P.d_left = dalloc<int32_t>(c);
    P.IB.S_out = dalloc<double>(c * kSlot);
    P.IB.copy = dalloc<int8_t>(c);
  }
  if (!P.d_nleft) P.d_nleft = dalloc<int32_t>(1);
  if (!P.IB.fail) P.IB.fail = dalloc<int32_t>(1);
  ensure(P.d_two, E->c_two, P.two.size());
  {
    const size_t prev = E->c_norms;
    ensure(P.d_norms, E->c_norms, P.norms.size());
    if (E->c_norms != prev || !P.IB.norms) {
      dfree(P.IB.norms);
      P.IB.norms = dalloc<double>(E->c_norms);
    }
  }
  ensure(P.d_lvl, E->c_lvl, P.lvl_list.size());
  ensure(P.d_cl, E->c_cl, P.cl_list.size());
  ensure(P.d_bl, E->c_bl, P.bl_list.size());
  ensure(P.IB.Q, E->c_q, (size_t)P.qlen);
  for (int sd = 0; sd < 2; ++sd) {
    const int32_t ncl = tr[sd]->count();
    if (E->c_ncl[sd] != ncl) {
      dfree(P.BW.G[sd]);
      dfree(P.BW.B[sd]);
      dfree(P.BW.need[sd]);
      dfree(P.BW.Vg[sd]);
      dfree(P.BW.orth[sd]);
      P.BW.G[sd] = dalloc<double>((size_t)ncl * kSlot);
      P.BW.B[sd] = dalloc<double>((size_t)ncl * kSlot);
      P.BW.Wo[sd] = P.BW.G[sd];
      P.BW.W0[sd] = P.BW.B[sd];
      P.BW.need[sd] = dalloc<int32_t>(ncl);
      P.BW.Vg[sd] = dalloc<double>((size_t)ncl * kSlot);
      P.BW.orth[sd] = dalloc<int32_t>(ncl);
      E->c_ncl[sd] = ncl;
    }
  }
  put(P.d_items, P.items, st);
  put(P.d_ents, P.ents, st);
  put(P.d_tasks, P.tasks, st);
  put(P.d_two, P.two, st);
  put(P.d_norms, P.norms, st);
  put(P.d_lvl, P.lvl_list, st);
  put(P.d_cl, P.cl_list, st);
  put(P.d_bl, P.bl_list, st);
  if (ni) H2_CUDA(cudaMemsetAsync(P.IB.jac, 0, 4 * ni * sizeof(unsigned long long), st));
  // the factors with leading dimension = rows
  ensure(P.d_A, E->c_A, (size_t)P.lenA);
  ensure(P.d_B, E->c_B, (size_t)P.lenB);
  H2_CUDA(cudaMemcpy2DAsync(P.d_A, P.rowsA[0] * sizeof(double), A, lda * sizeof(double), P.rowsA[0] * sizeof(double),
                            u, cudaMemcpyDeviceToDevice, st));
  H2_CUDA(cudaMemcpy2DAsync(P.d_B, P.rowsB[0] * sizeof(double), B, ldb * sizeof(double), P.rowsB[0] * sizeof(double),
                            u, cudaMemcpyDeviceToDevice, st));
  // a new plan every call: never replay a captured graph
  if (P.graph) cudaGraphExecDestroy(P.graph);
  P.graph = nullptr;
  P.g_A = nullptr;
  P.g_repeats = 0;
  if (!E->cs.err) H2_CUDA(cudaMallocHost(&E->cs.err, sizeof(int)));
  const auto c2 = clk::now();
  execute(ctx, P, P.d_A, P.d_B, eps);
  E->launch_s += std::chrono::duration<double>(clk::now() - c2).count();
  // the commit reads the new ranks back (one synchronisation); its copies
  // stay in flight on the context's stream
  commit_update(ctx, &P, 0, P.d_A, P.d_B, Z, &E->cs);
  // what this update computed is cached; what it changed is stale
  for (int32_t e : P.cl_list) E->g_ok[e >> 30][e & 0x3fffffff] = 1;
  for (int32_t e : P.bl_list) E->b_ok[e >> 30][e & 0x3fffffff] = 1;
  engine_touch(E, Z, block);
  ++E->updates;
  E->total_s += std::chrono::duration<double>(clk::now() - c0).count();
}

}  // namespace h2

extern "C" h2_status h2_lowrank_update(h2_ctx* ctx, h2_matrix* Z, int64_t block, int u, const double* A,
                                       int64_t lda, const double* B, int64_t ldb, double eps) {
  if (!ctx || !Z || !A || !B) return H2_EINVAL;
  return guard(ctx, [&] {
    H2_REQUIRE(block >= 0 && block < Z->blocks.count(), "h2_lowrank_update: block out of range");
    const int64_t rows = Z->rows.size[Z->blocks.row[block]];
    const int64_t cols = Z->cols.size[Z->blocks.col[block]];
    H2_REQUIRE(lda >= rows && ldb >= cols, "h2_lowrank_update: leading dimension too small");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    h2_batch* P = nullptr;
    h2_status s = h2_batch_create(ctx, Z, 1, &block, u, &P);
    if (s != H2_OK) throw Error(s, ctx->last_error);
    std::unique_ptr<h2_batch, void (*)(h2_batch*)> hold(P, h2_batch_free);
    double* dA = nullptr;
    double* dB = nullptr;
    try {
      dA = dalloc<double>(rows * u);
      dB = dalloc<double>(cols * u);
      H2_CUDA(cudaMemcpy2DAsync(dA, rows * sizeof(double), A, lda * sizeof(double), rows * sizeof(double), u,
                                cudaMemcpyDeviceToDevice, st));
      H2_CUDA(cudaMemcpy2DAsync(dB, cols * sizeof(double), B, ldb * sizeof(double), cols * sizeof(double), u,
                                cudaMemcpyDeviceToDevice, st));
      execute(ctx, *P, dA, dB, eps);
      s = h2_batch_apply(ctx, P, 0, dA, dB, Z);
      if (s != H2_OK) throw Error(s, ctx->last_error);
    } catch (...) {
      cudaStreamSynchronize(st);
      dfree(dA);
      dfree(dB);
      throw;
    }
    H2_CUDA(cudaStreamSynchronize(st));
    dfree(dA);
    dfree(dB);
  });
}

namespace {
// Waves of a sequence of updates (sequential semantics, Section 5 applied in
// order).  What update j reads: the bases (leaf matrices, transfer matrices,
// ranks) of the clusters of T_t0 and of the ancestors of t0, likewise on the
// column side, and the couplings of every block in the rows of those row
// clusters and in the columns of those column clusters (the weights of
// Section 4 over the whole block rows and the ancestor paths, the
// reprojection).  What it writes: the bases of T_t0 and T_s0 (the commit of
// E_t0 included) and the couplings of the blocks with row in T_t0 or column
// in T_s0 (and the nearfield inside b0, which no update reads).  Update j
// goes into the first wave after every earlier update whose writes it reads,
// and not before any earlier update that reads what j writes; inside a wave
// all updates read the matrix as it was before the wave and commit in order.
int32_t sequence_waves(const h2_matrix* Z, int64_t count, const int64_t* blocks, std::vector<int32_t>& wave) {
  const BlockTree& bt = Z->blocks;
  const ClusterTree* tr[2] = {&Z->rows, &Z->cols};
  const int32_t nc0 = tr[0]->count();
  const int32_t ncl = nc0 + tr[1]->count();
  const int32_t nslot = (int32_t)bt.adm.size();
  std::vector<int32_t> wr_cl(ncl, -1), rd_cl(ncl, -1), wr_s(nslot, -1), rd_s(nslot, -1);
  std::vector<int32_t> rcl, wcl, rs, ws;
  int32_t waves = 0;
  wave.assign(count, 0);
  for (int64_t j = 0; j < count; ++j) {
    rcl.clear();
    wcl.clear();
    rs.clear();
    ws.clear();
    for (int sd = 0; sd < 2; ++sd) {
      const ClusterTree& ct = *tr[sd];
      const int32_t c0 = sd == 0 ? bt.row[blocks[j]] : bt.col[blocks[j]];
      const int32_t base = sd == 0 ? 0 : nc0;
      const std::vector<int32_t>& ptr = sd == 0 ? bt.row_ptr : bt.col_ptr;
      const std::vector<int32_t>& adm = sd == 0 ? bt.row_adm : bt.col_adm;
      auto blocks_of = [&](int32_t c, std::vector<int32_t>& out) {
        for (int32_t e = ptr[c]; e < ptr[c + 1]; ++e) out.push_back(adm[e]);
      };
      for (int32_t c = c0; c < c0 + ct.subtree[c0]; ++c) {   // T_c0 (preorder)
        wcl.push_back(base + c);
        rcl.push_back(base + c);
        blocks_of(c, ws);
        blocks_of(c, rs);
      }
      for (int32_t a = ct.father[c0]; a >= 0; a = ct.father[a]) {
        rcl.push_back(base + a);
        blocks_of(a, rs);
      }
    }
    int32_t w = 0;
    for (int32_t r : rcl) w = std::max(w, wr_cl[r] + 1);
    for (int32_t r : rs) w = std::max(w, wr_s[r] + 1);
    for (int32_t r : wcl) w = std::max(w, rd_cl[r]);
    for (int32_t r : ws) w = std::max(w, rd_s[r]);
    wave[j] = w;
    waves = std::max(waves, w + 1);
    for (int32_t r : wcl) wr_cl[r] = std::max(wr_cl[r], w);
    for (int32_t r : ws) wr_s[r] = std::max(wr_s[r], w);
    for (int32_t r : rcl) rd_cl[r] = std::max(rd_cl[r], w);
    for (int32_t r : rs) rd_s[r] = std::max(rd_s[r], w);
  }
  return waves;
}
}  // namespace

extern "C" h2_status h2_sequence_waves(const h2_matrix* Z, int64_t count, const int64_t* blocks, int32_t* wave,
                                       int64_t* n_waves) {
  if (!Z || count < 0 || (count > 0 && (!blocks || !wave))) return H2_EINVAL;
  return guard(nullptr, [&] {
    for (int64_t j = 0; j < count; ++j)
      H2_REQUIRE(blocks[j] >= 0 && blocks[j] < Z->blocks.count(), "h2_sequence_waves: block id out of range");
    std::vector<int32_t> wv;
    const int32_t waves = sequence_waves(Z, count, blocks, wv);
    std::copy(wv.begin(), wv.end(), wave);
    if (n_waves) *n_waves = waves;
  });
}

extern "C" h2_status h2_lowrank_update_sequence(h2_ctx* ctx, h2_matrix* Z, int64_t count, const int64_t* blocks,
                                                int u, const double* A, const double* B, double eps,
                                                int64_t* waves_out) {
  if (!ctx || !Z || count < 0 || (count > 0 && (!blocks || !A || !B))) return H2_EINVAL;
  return guard(ctx, [&] {
    H2_REQUIRE(std::isfinite(eps) && eps >= 0, "h2_lowrank_update_sequence: eps must be finite and >= 0");
    H2_REQUIRE(has_storage(Z), "h2_lowrank_update_sequence: matrix has no device storage");
    const BlockTree& bt = Z->blocks;
    std::vector<int64_t> offA(count), offB(count);
    int64_t la = 0, lb = 0;
    for (int64_t j = 0; j < count; ++j) {
      H2_REQUIRE(blocks[j] >= 0 && blocks[j] < bt.count(), "h2_lowrank_update_sequence: block id out of range");
      offA[j] = la;
      offB[j] = lb;
      la += Z->rows.size[bt.row[blocks[j]]] * u;
      lb += Z->cols.size[bt.col[blocks[j]]] * u;
    }
    std::vector<int32_t> wave;
    const int32_t waves = sequence_waves(Z, count, blocks, wave);
    DeviceGuard g(ctx->device);
    std::vector<int64_t> wb, wa, wbo;
    std::vector<int64_t> members;
    for (int32_t w = 0; w < waves; ++w) {
      members.clear();
      for (int64_t j = 0; j < count; ++j)
        if (wave[j] == w) members.push_back(j);
      wb.clear();
      wa.clear();
      wbo.clear();
      for (int64_t j : members) {
        wb.push_back(blocks[j]);
        wa.push_back(offA[j]);
        wbo.push_back(offB[j]);
      }
      // the wave as one isolated batch on the current matrix (its factors
      // addressed in place in the caller's arrays), then its commits in order
      h2_batch* P = nullptr;
      h2_status s = create_batch(ctx, Z, (int64_t)wb.size(), wb.data(), u, wa.data(), wbo.data(), &P);
      if (s != H2_OK) throw Error(s, ctx->last_error);
      std::unique_ptr<h2_batch, void (*)(h2_batch*)> hold(P, h2_batch_free);
      execute(ctx, *P, A, B, eps);
      for (int64_t i = 0; i < (int64_t)wb.size(); ++i) {
        s = h2_batch_apply(ctx, P, i, A, B, Z);
        if (s != H2_OK) throw Error(s, ctx->last_error);
      }
    }
    H2_CUDA(cudaStreamSynchronize(ctx->stream));
    if (waves_out) *waves_out = waves;
  });
}

namespace {
void ensure_matvec_plan(h2_matrix* Z, cudaStream_t st) {
  if (Z->mv_ready) return;
  const ClusterTree* tr[2] = {&Z->rows, &Z->cols};
  for (int sd = 0; sd < 2; ++sd) {
    const ClusterTree& ct = *tr[sd];
    const int L = ct.depth + 1;
    std::vector<int32_t>& ptr = Z->mv_lvl_ptr[sd];
    ptr.assign(L + 1, 0);
    for (int32_t c = 0; c < ct.count(); ++c) ptr[ct.level[c] + 1]++;
    for (int l = 0; l < L; ++l) ptr[l + 1] += ptr[l];
    std::vector<int32_t> list(ct.count()), fill(ptr.begin(), ptr.end() - 1);
    for (int32_t c = 0; c < ct.count(); ++c) list[fill[ct.level[c]]++] = c;
    dfree(Z->d_mv_lvl[sd]);   // a retry after a failed allocation
    Z->d_mv_lvl[sd] = upload(list, st);
  }
  std::vector<int32_t> leaves;
  for (int32_t c = 0; c < Z->rows.count(); ++c)
    if (Z->rows.leaf(c)) leaves.push_back(c);
  Z->mv_n_leaves = (int32_t)leaves.size();
  dfree(Z->d_mv_leaves);
  Z->d_mv_leaves = upload(leaves, st);
  const BlockTree& bt = Z->blocks;
  std::vector<int32_t> nptr(Z->rows.count() + 1, 0), ncol(bt.near.size());
  std::vector<int64_t> noff(bt.near.size());
  for (int32_t b : bt.near) nptr[bt.row[b] + 1]++;
  for (int32_t c = 0; c < Z->rows.count(); ++c) nptr[c + 1] += nptr[c];
  std::vector<int32_t> nf(nptr.begin(), nptr.end() - 1);
  for (size_t i = 0; i < bt.near.size(); ++i) {
    const int32_t b = bt.near[i];
    const int32_t x = nf[bt.row[b]]++;
    ncol[x] = bt.col[b];
    noff[x] = Z->near_off[bt.slot[b]];
  }
  dfree(Z->d_near_ptr);
  dfree(Z->d_near_col);
  dfree(Z->d_near_off);
  Z->d_near_ptr = upload(nptr, st);
  Z->d_near_col = upload(ncol, st);
  Z->d_near_off = upload(noff, st);
  Z->mv_ready = true;
}
}  // namespace

extern "C" h2_status h2_matvec(h2_ctx* ctx, const h2_matrix* Zc, int64_t nrhs, double alpha, const double* X,
                               int64_t ldx, double beta, double* Y, int64_t ldy) {
  if (!ctx || !Zc || nrhs < 0) return H2_EINVAL;
  return guard(ctx, [&] {
    h2_matrix* Z = const_cast<h2_matrix*>(Zc);   // the plan is cached on the matrix
    H2_REQUIRE(has_storage(Z), "h2_matvec: matrix has no device storage");
    if (nrhs == 0) return;
    const int64_t nr = Z->rows.count() ? Z->rows.size[0] : 0;
    const int64_t nc = Z->cols.count() ? Z->cols.size[0] : 0;
    H2_REQUIRE(X && Y, "h2_matvec: operands missing");
    H2_REQUIRE(ldx >= nc && ldy >= nr, "h2_matvec: leading dimension too small");
    H2_REQUIRE(nrhs <= (int64_t)1 << 20, "h2_matvec: too many right-hand sides");
    const double* Xe = X + (size_t)(nrhs - 1) * ldx + nc;
    const double* Ye = Y + (size_t)(nrhs - 1) * ldy + nr;
    H2_REQUIRE(Xe <= Y || Ye <= X, "h2_matvec: X and Y overlap");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    ensure_matvec_plan(Z, st);
    MatvecArgs a{};
    const int64_t* offs[2] = {Z->d_row_off, Z->d_col_off};
    const int32_t* sizes[2] = {Z->d_row_size, Z->d_col_size};
    const int32_t* subs[2] = {Z->d_subtree_r, Z->d_subtree_c};
    const int32_t* fath[2] = {Z->d_father_r, Z->d_father_c};
    for (int sd = 0; sd < 2; ++sd) {
      const DeviceBasis& bs = basis_of(Z, sd);
      a.off[sd] = offs[sd];
      a.size[sd] = sizes[sd];
      a.rank[sd] = bs.d_rank;
      a.subtree[sd] = subs[sd];
      a.father[sd] = fath[sd];
      a.leaf[sd] = bs.d_leaf;
      a.leaf_off[sd] = bs.d_leaf_off;
      a.transfer[sd] = bs.d_transfer;
      a.lvl_ptr[sd] = Z->mv_lvl_ptr[sd].data();
      a.lvl_list[sd] = Z->d_mv_lvl[sd];
      a.levels[sd] = (int)Z->mv_lvl_ptr[sd].size() - 1;
      a.n_clusters[sd] = tree_of(Z, sd).count();
    }
    a.S = Z->d_S;
    a.kcap = Z->kcap;
    a.row_ptr = Z->d_row_ptr;
    a.row_adm = Z->d_row_adm;
    a.blk_col = Z->d_blk_col;
    a.N = Z->d_N;
    a.near_ptr = Z->d_near_ptr;
    a.near_col = Z->d_near_col;
    a.near_off = Z->d_near_off;
    a.leaves = Z->d_mv_leaves;
    a.n_leaves = Z->mv_n_leaves;
    a.nrhs = (int)nrhs;
    a.alpha = alpha;
    a.beta = beta;
    a.X = X;
    a.ldx = ldx;
    a.Y = Y;
    a.ldy = ldy;
    // per-cluster workspace, stream-ordered
    const size_t wx = (size_t)a.n_clusters[1] * Z->kcap * nrhs, wy = (size_t)a.n_clusters[0] * Z->kcap * nrhs;
    void* w = device_alloc_async((wx + wy) * sizeof(double), st);
    a.xh = static_cast<double*>(w);
    a.yh = a.xh ? a.xh + wx : nullptr;
    launch_matvec(a, st);
    const cudaError_t e = cudaGetLastError();
    if (w) H2_CUDA(cudaFreeAsync(w, st));
    H2_CUDA(e);
  });
}

namespace {
__global__ void k_unit_columns(double* X, int64_t n, int64_t s_off, int64_t ns) {
  // X (n x ns, ld n) = columns s_off .. s_off + ns - 1 of the identity
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * ns) return;
  const int64_t i = e % n, j = e / n;
  X[e] = i == s_off + j ? 1.0 : 0.0;
}

__global__ void k_rows_out(const double* Y, int64_t n, int64_t t_off, int64_t nt, int64_t ns, double* out,
                           int64_t ld) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nt * ns) return;
  const int64_t i = e % nt, j = e / nt;
  out[i + j * ld] = Y[t_off + i + j * n];
}
}  // namespace

extern "C" h2_status h2_block_to_dense(h2_ctx* ctx, const h2_matrix* Z, int64_t block, double* out, int64_t ld) {
  if (!ctx || !Z || !out) return H2_EINVAL;
  return guard(ctx, [&] {
    const BlockTree& bt = Z->blocks;
    H2_REQUIRE(block >= 0 && block < bt.count(), "h2_block_to_dense: block out of range");
    H2_REQUIRE(has_storage(Z), "h2_block_to_dense: matrix has no device storage");
    const int32_t t = bt.row[block], sc = bt.col[block];
    const int64_t nt = Z->rows.size[t], ns = Z->cols.size[sc];
    H2_REQUIRE(ld >= nt, "h2_block_to_dense: leading dimension too small");
    const int64_t n_r = Z->rows.size[0], n_c = Z->cols.size[0];
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    // Z|_{t x s} = rows t of Z times the unit columns of s (the whole matrix
    // product h2_matvec with #s right-hand sides)
    void* w = device_alloc_async((size_t)(n_c + n_r) * ns * sizeof(double), st);
    double* X = static_cast<double*>(w);
    double* Y = X + (size_t)n_c * ns;
    const int th = 256;
    k_unit_columns<<<(unsigned)((n_c * ns + th - 1) / th), th, 0, st>>>(X, n_c, Z->cols.off[sc], ns);
    h2_status s = h2_matvec(ctx, Z, ns, 1.0, X, n_c, 0.0, Y, n_r);
    if (s == H2_OK && nt * ns > 0)
      k_rows_out<<<(unsigned)((nt * ns + th - 1) / th), th, 0, st>>>(Y, n_r, Z->rows.off[t], nt, ns, out, ld);
    const cudaError_t e = cudaGetLastError();
    H2_CUDA(cudaFreeAsync(w, st));
    if (s != H2_OK) throw Error(s, ctx->last_error);
    H2_CUDA(e);
  });
}

extern "C" h2_status h2_check_reciprocal(h2_ctx* ctx, const double* d, int64_t n, double* out) {
  using namespace h2;
  if (!ctx || n < 0 || (n > 0 && (!d || !out))) return H2_EINVAL;
  return guard(ctx, [&] {
    DeviceGuard g(ctx->device);
    launch_recip_check(d, n, out, ctx->stream);
    H2_CUDA(cudaGetLastError());
  });
}
