// H^2-matrix times a block of vectors: launch sequence (matvec.cu).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace h2 {

struct MatvecArgs {
  // row tree (Y side) and column tree (X side), tree order, device
  const int64_t* off[2];
  const int32_t* size[2];
  const int32_t* rank[2];
  const int32_t* subtree[2];     // sons of c: c + 1 and c + 1 + subtree[c + 1]
  const int32_t* father[2];
  const double* leaf[2];         // leaf bases V (side 0), W (side 1)
  const int64_t* leaf_off[2];
  const double* transfer[2];     // kcap x kcap slots per cluster
  const double* S;               // couplings, kcap x kcap slots
  int kcap;
  const int32_t* row_ptr;        // admissible slots by row cluster (CSR)
  const int32_t* row_adm;
  const int32_t* blk_col;        // column cluster of a slot
  const double* N;               // nearfield blocks (column-major #t x #s)
  const int32_t* near_ptr;       // nearfield blocks by row cluster (CSR)
  const int32_t* near_col;       // their column clusters
  const int64_t* near_off;       // their offsets in N
  // levels: clusters of each tree by level (host pointers to the CSR, device list)
  const int32_t* lvl_ptr[2];
  const int32_t* lvl_list[2];
  int levels[2];
  const int32_t* leaves;         // leaves of the row tree (device)
  int n_leaves;
  int n_clusters[2];
  // operands
  int nrhs;
  double alpha, beta;
  const double* X;
  int64_t ldx;
  double* Y;
  int64_t ldy;
  double* xh;                    // per column cluster kcap x nrhs (ld kcap)
  double* yh;                    // per row cluster kcap x nrhs
};

// Launch Y <- alpha Z X + beta Y on st; returns the number of launches.
int launch_matvec(const MatvecArgs& a, cudaStream_t st);

}  // namespace h2
