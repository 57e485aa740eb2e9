// Internal declarations of libh2gb (host C++ and CUDA).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/h2gb.h"

namespace h2 {

// Largest supported extended rank k_t + u (one warp lane per column).
constexpr int kMaxCols = 32;

struct Error : std::runtime_error {
  h2_status code;
  Error(h2_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define H2_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      throw ::h2::Error(H2_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define H2_REQUIRE(cond, msg) \
  do {                        \
    if (!(cond)) throw ::h2::Error(H2_EINVAL, msg); \
  } while (0)

// Every device allocation of the library goes through these two calls.
// They throw Error(H2_ENOMEM) when the allocation fails, or when the
// failure hook (h2_debug_fail_allocation) says this allocation is the one
// to fail.
void* device_alloc(size_t bytes);
void* device_alloc_async(size_t bytes, cudaStream_t st);

// Raise a kernel's dynamic shared memory limit once per device: `done` holds
// one bit per device ordinal below 64 (above, the attribute is set on every
// call).  Host threads with contexts of their own may call it at once; the
// attribute is idempotent.
template <class Kern>
inline void smem_limit(Kern kern, size_t bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  H2_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return;
  H2_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  done.fetch_or(bit, std::memory_order_release);
}

// ----------------------------------------------------------------- trees
struct ClusterTree {
  int64_t n = 0;
  int dim = 0;
  std::vector<int64_t> perm;            // tree position -> original index
  std::vector<int64_t> off, size;       // per cluster, tree order
  std::vector<int32_t> father, son0, son1, level, subtree;
  std::vector<double> lo, hi;           // dim per cluster (padded boxes)
  int depth = 0;
  int max_leaf = 0;
  int32_t count() const { return (int32_t)off.size(); }
  bool leaf(int32_t c) const { return son0[c] < 0; }
};

enum BlockKind : int32_t { kSub = 0, kAdm = 1, kNear = 2 };

struct BlockTree {
  std::vector<int32_t> row, col, kind, father;
  std::vector<int32_t> son4;       // 4 entries per block (-1 where absent), order (t1,s1),(t1,s2),(t2,s1),(t2,s2)
  std::vector<int32_t> slot;       // admissible: coupling slot; near: nearfield slot; sub: -1
  std::vector<int32_t> adm, near;  // block ids of the leaves, in block order
  // admissible slots by row cluster and by column cluster (CSR)
  std::vector<int32_t> row_ptr, row_adm, col_ptr, col_adm;
  int32_t count() const { return (int32_t)row.size(); }
};

void build_cluster_tree(const double* pts, int64_t n, int dim, int leaf_size, double pad,
                        ClusterTree& ct);
void build_block_tree(const ClusterTree& rt, const ClusterTree& ct, double eta, BlockTree& bt);

// --------------------------------------------------------------- storage
// One cluster basis on the device.  Leaf matrices: size_t x kcap slots with
// leading dimension size_t; transfers: kcap x kcap slots (ld kcap).
struct DeviceBasis {
  std::vector<int32_t> rank;       // host copy of the ranks
  int32_t* d_rank = nullptr;
  double* d_leaf = nullptr;        // concatenated leaf slots
  double* d_transfer = nullptr;    // n_clusters slots of kcap*kcap
  std::vector<int64_t> leaf_off;   // per cluster (leaves), element offset
  int64_t* d_leaf_off = nullptr;
};

// Z <- the zero matrix on Z's trees: every rank 0, couplings, nearfield
// and basis storage zero (asynchronous on the context's stream).
void zero_matrix(h2_ctx* ctx, h2_matrix* Z);

// Reusable engine of in-place single updates (api.cu): persistent device
// buffers, the exact path, base weights only for the clusters an update
// reads.  Not thread-safe; one per driver.
struct UpdateEngine;
UpdateEngine* engine_new();
void engine_delete(UpdateEngine* E);
int64_t engine_updates(const UpdateEngine* E);
// seconds spent planning on the host, enqueueing the kernels, waiting for
// the GPU before the commit, and in the whole calls
void engine_times(const UpdateEngine* E, double* plan, double* launch, double* wait, double* total);
// Z's block b0 is about to change, or has changed (an update of b0, or a
// coupling written outside the engine): the engine's cached weights of the
// clusters it affects are stale.  No effect for another matrix or a null E.
void engine_touch(UpdateEngine* E, const h2_matrix* Z, int32_t b0);
// Z|_b <- trunc_eps(Z|_b + A B^*) in place (A: #t x u, ld lda; B: #s x u,
// ld ldb; device); the new ranks are on the host on return, the device
// work of the commit may still run on the context's stream.  max_rank > 0:
// every new basis keeps at most max_rank columns (0: the rank rule alone).
// Throws h2::Error.
void engine_update(h2_ctx* ctx, h2_matrix* Z, UpdateEngine* E, int32_t block, int u, const double* A, int64_t lda,
                   const double* B, int64_t ldb, double eps, int max_rank = 0);

}  // namespace h2

struct h2_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string last_error;
  int* d_error = nullptr;          // device error word (0 = fine)
};

struct h2_matrix {
  h2::ClusterTree rows, cols;      // row and column trees (identical index sets here)
  h2::BlockTree blocks;
  int kcap = 0;
  int device = 0;
  h2::DeviceBasis V, W;
  double* d_S = nullptr;           // n_adm slots of kcap*kcap (ld kcap)
  double* d_N = nullptr;           // nearfield, concatenated size_t x size_s
  std::vector<int64_t> near_off;   // per nearfield slot
  int64_t near_len = 0;
  // device copies of the structure needed by kernels
  int64_t* d_row_off = nullptr;    // cluster offsets (tree order), row tree
  int64_t* d_col_off = nullptr;
  int32_t* d_row_size = nullptr;
  int32_t* d_col_size = nullptr;
  int32_t* d_subtree_r = nullptr;
  int32_t* d_subtree_c = nullptr;
  int32_t* d_blk_row = nullptr;    // per admissible slot: row / col cluster
  int32_t* d_blk_col = nullptr;
  int32_t* d_row_ptr = nullptr;    // CSR admissible slots by row cluster
  int32_t* d_row_adm = nullptr;
  int32_t* d_col_ptr = nullptr;
  int32_t* d_col_adm = nullptr;
  int32_t* d_father_r = nullptr;
  int32_t* d_father_c = nullptr;
  // plan of h2_matvec (built on first use; the trees never change): clusters
  // of each tree by level, the leaves of the row tree, the nearfield blocks
  // by row cluster (CSR: column cluster, offset in d_N)
  bool mv_ready = false;
  std::vector<int32_t> mv_lvl_ptr[2];
  int32_t* d_mv_lvl[2] = {nullptr, nullptr};
  int32_t* d_mv_leaves = nullptr;
  int32_t mv_n_leaves = 0;
  int32_t* d_near_ptr = nullptr;
  int32_t* d_near_col = nullptr;
  int64_t* d_near_off = nullptr;
};
