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

void launch_prepass(const MatView& M, int side, const int32_t* clusters, int n, const int32_t* ptr,
                    const int32_t* adm, const int32_t* other_cl, const BaseWeights& BW, int* err,
                    cudaStream_t st);
void launch_rfactor(const MatView& M, const Item* items, const int32_t* list, int n, int u,
                    const double* A, const double* B, const ItemBuffers& IB, int* err, cudaStream_t st);
void launch_norms(const MatView& M, const Item* items, const NormTask* tasks, int n, int u,
                  const ItemBuffers& IB, cudaStream_t st);
void launch_weights(const MatView& M, const Item* items, const Entry* ents, const int32_t* list, int n,
                    int u, const BaseWeights& BW, const ItemBuffers& IB, int* err, cudaStream_t st);
void launch_truncate(const MatView& M, const Item* items, const int32_t* list, int n, int u, int kl,
                     int max_rows, double eps, const double* A, const double* B, const ItemBuffers& IB,
                     int* err, cudaStream_t st);
void launch_reproject(const MatView& M, const Item* items, const Task* tasks, int n, int u,
                      const ItemBuffers& IB, cudaStream_t st);
void launch_copy(const CopyDesc* d, int n, cudaStream_t st);
void launch_near_add(const NearDesc* d, int n, int u, cudaStream_t st);

}  // namespace h2
