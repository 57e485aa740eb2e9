// Launchers of the update kernels (called by the host planner).
#pragma once

#include <cuda_runtime.h>

#include "update_plan.h"

namespace h2 {

struct CopyDesc {
  const double* src;
  double* dst;
  int rows, cols;
  int lds, ldd;
};

struct NearDesc {
  double* N;
  const double* A;
  const double* B;
  int rows, cols;
  int ldn, lda, ldb;
  int pad;
};

// Admissible-block lists of the matrix, for the weights of the unchanged matrix.
struct BlockLists {
  const int32_t* ptr[2];     // CSR of admissible slots by row / column cluster
  const int32_t* adm[2];
  const int32_t* other[2];   // per slot: the cluster on the other side
};

// Everything one execution of the update kernels needs (device pointers
// unless marked host).
struct Pipeline {
  MatView M;
  BlockLists BL;
  BaseWeights BW;
  ItemBuffers IB;
  const Item* items;
  const Entry* ents;
  const Task* tasks;
  const NormTask* norms;
  const int32_t* lvl_list;      // items sorted by level
  const int32_t* lvl_ptr;       // host, levels + 1 entries
  const int32_t* lvl_rows;      // host, per level: bound on the truncation rows
  const int32_t* lvl_leaves;    // host, per level: number of leaves (they come first in lvl_list)
  const int32_t* cl_list;       // all clusters of both sides sorted by level (side << 30 | id)
  const int32_t* cl_ptr;        // host, levels + 1 entries
  // exact path: base weights only for these clusters by level (null: cl_list)
  const int32_t* bl_list = nullptr;
  const int32_t* bl_ptr = nullptr;   // host, levels + 1 entries
  int max_rank = 0;                  // exact path: rank cap of the truncation (0: none)
  int levels;
  int n_updates;
  int ncl[2];                   // clusters per side
  int exact_only;               // 1: every update takes the exact path
  int n_tasks, n_norms;
  const int32_t* two;           // the two-sided coupling tasks (both clusters inside)
  int n_two;
  int32_t* left;                // one-sided tasks that are not copies (filled on the device)
  int32_t* n_left;              // their number (device)
  int u, kl;
  double eps;
  const double* A;
  const double* B;
  int* err;
  cudaStream_t stream;
  // optional second stream for the weights of the unchanged matrix, which
  // overlap steps 2 and the outside folds of step 3; fork/join events
  // required when side != nullptr
  cudaStream_t side;
  cudaEvent_t fork, join;
  // optional third stream for the basis Grams V_t^* V_t of the unchanged
  // matrix, which run beside the weights on `side` (join2 required with it)
  cudaStream_t side2;
  cudaEvent_t join2;
  cudaEvent_t* events;          // 2 * H2_PHASE_COUNT events (start, end per phase) or nullptr
  int64_t* phase_launches;      // host, H2_PHASE_COUNT entries or nullptr
  bool capturing;               // the launches are being captured into a graph
  const struct HostOutput* out; // copy of the results to host memory, or nullptr
};

// Copy of the results to page-locked host memory, overlapped with the
// update: `early` is launched on `stream` once the orthonormality flags of
// the unchanged matrix exist (certified path only; `packed` is recorded
// after its kernels, `done` after its copies), `late` on the main stream
// after the reprojection (after waiting for `packed` when early ran); the
// main stream then waits for `done`.
struct HostOutput {
  cudaStream_t stream;
  cudaEvent_t ready, packed, done;
  void (*early)(const Pipeline& P, const HostOutput& O, cudaStream_t st);
  void (*late)(const Pipeline& P, const HostOutput& O, cudaStream_t st, bool early_ran);
  void* owner;
};

// Launch the whole update (weights of the unchanged matrix, steps 2-5) on
// P.stream: the certified Gram path for every update, the exact path for the
// updates whose certificate failed (all of them when P.exact_only), then the
// reprojection.
void run_pipeline(const Pipeline& P);

// Certified Gram path (gram_kernels.cu).
void launch_gram_orth(const Pipeline& P, cudaStream_t st);                // orthonormality flags (2 launches)
void launch_gram_vbasis_level(const Pipeline& P, int level, cudaStream_t st);  // V_t^* V_t, one level
void launch_gram_base(const Pipeline& P, cudaStream_t st);               // Wo, all clusters
void launch_gram_base_level(const Pipeline& P, int level, cudaStream_t st);  // W0, one level
int launch_gram_basis(const Pipeline& P, int level);                     // G_t, one level (returns launches)
void launch_gram_norms(const Pipeline& P);                               // ||Z~|_b||_F inside
void launch_gram_weights(const Pipeline& P, int level);                  // W_t, one level
void launch_gram_certify(const Pipeline& P);                             // certificate, R_t
void launch_gram_outputs(const Pipeline& P);                             // new bases, marks
void launch_copy(const CopyDesc* d, int n, cudaStream_t st);
void launch_recip_check(const double* d, int64_t n, double* out, cudaStream_t st);
void launch_near_add(const NearDesc* d, int n, int u, cudaStream_t st);

}  // namespace h2
