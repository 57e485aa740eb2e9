// Internal declarations of the H^2-LR factorisation path (lr.cu, lr_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace h2 {

// One cluster basis seen from a kernel (device pointers; tree order).
struct BasisView {
  const int64_t* off;        // cluster offsets
  const int32_t* size;       // cluster sizes
  const int32_t* rank;       // ranks
  const int32_t* subtree;    // #T_c; the sons of c are c + 1 and c + 1 + subtree[c + 1]
  const double* leaf;        // leaf slots (size_t x kcap, ld size_t)
  const int64_t* leaf_off;   // per cluster, element offset of its leaf slot
  const double* transfer;    // kcap x kcap slots per cluster
};

// Y += alpha op(Z|_b) X for one block b of the block tree, op = identity
// (trans = 0: X on the columns of b, Y on its rows) or transpose (trans = 1).
// "in" is the side of X, "out" the side of Y.
struct BlockProd {
  BasisView in, out;
  int kcap;
  int trans;
  int64_t in_off0, out_off0;  // tree offsets of b's X-side and Y-side clusters
  const double* S;            // couplings, kcap x kcap slots
  const double* N;            // nearfield blocks
  const int64_t* near_off;    // per nearfield slot
  int m;                      // columns of X and Y
  double alpha;
  const double* X;
  int64_t ldx;
  double* Y;
  int64_t ldy;
  double* xh;                 // per X-side cluster kcap x m (ld kcap)
  double* yh;                 // per Y-side cluster kcap x m
};

// forward transformation: xh_c for the X-side clusters of `list`
void launch_bp_forward(const BlockProd& a, const int32_t* list, int n, cudaStream_t st);
// couplings: yh_c = sum_e S_e xh_{in_e} (or S_e^* xh) for the Y-side clusters
// of `list` with entries ptr[i]..ptr[i+1] (pairs slot, X-side cluster)
void launch_bp_coupling(const BlockProd& a, const int32_t* list, int n, const int32_t* ptr,
                        const int32_t* ent, cudaStream_t st);
// backward transformation: yh_c += E_c yh_father for the clusters of `list`
void launch_bp_backward(const BlockProd& a, const int32_t* list, const int32_t* fathers, int n,
                        cudaStream_t st);
// leaves of the Y side: Y|_l += alpha (V_l yh_l + nearfield rows), near
// entries ptr[i]..ptr[i+1] of (nearfield slot, X-side cluster, Y-side cluster)
void launch_bp_leaves(const BlockProd& a, const int32_t* leaves, int n, const int32_t* ptr, const int32_t* ent,
                      cudaStream_t st);
// yh_c = identity (k x k, ld kcap), for the expansion of a basis
void launch_identity(double* yh, int k, int kcap, cudaStream_t st);

// C = alpha op(A) op(B) + beta C (C is m x n; C not read when beta = 0)
void launch_gemm(int m, int n, int k, double alpha, const double* A, int64_t lda, int ta, const double* B,
                 int64_t ldb, int tb, double beta, double* C, int64_t ldc, cudaStream_t st);
// B (n x m) = alpha A^* (A m x n); A = identity (n x n)
void launch_transpose(int m, int n, double alpha, const double* A, int64_t lda, double* B, int64_t ldb,
                      cudaStream_t st);
void launch_eye(double* A, int n, int64_t lda, cudaStream_t st);
// in-place LU without pivoting (Doolittle) of the m x m block A (ld lda);
// a zero pivot sets bit 8 of *err
void launch_leaf_lu(double* A, int m, int64_t lda, int* err, cudaStream_t st);
// Cholesky factor (lower, strictly upper part zeroed) of a dense leaf in
// place; a pivot that is not positive sets bit 512 of *err
void launch_leaf_chol(double* A, int m, int64_t lda, int* err, cudaStream_t st);
// triangular solves with the factor F (m x m, ld ldf):
//   kind 0: X <- L^-1 X  (L unit lower in F, X m x n)
//   kind 1: X <- R^-1 X  (R upper with the diagonal in F, X m x n)
//   kind 2: X <- X R^-1  (X n x m)
void launch_trsm(int kind, const double* F, int m, int64_t ldf, double* X, int n, int64_t ldx, cudaStream_t st);
// Truncation of a factor pair (A mt x m, B mr x m, m <= kCompressMax): Householder
// QR of both in place, the SVD of the core R_A R_B^* by one-sided Jacobi
// and the rank rule, then A' = Q_A [U_r Sigma_r; 0], B' = Q_B [W_r; 0].
// One temporary to truncate (device pointers): the factors A (ld mt) and B
// (ld mr); ka = min(mt, m), kb = min(mr, m); scratch tauA, tauB (m), C, W
// (m x m), TA, TB (m x m, first r columns: U_r Sigma_r and W_r); flags[0]
// receives the rank, flags[1..2] whether A and B have a nonzero entry (a
// zero product has rank 0 at once).
struct Compress {
  double* A;
  double* B;
  int mt, mr, m, ka, kb;
  double* tauA;
  double* tauB;
  double* C;
  double* W;
  double* TA;
  double* TB;
  int* flags;
};
// QR and core SVD of n temporaries at once (one block per temporary and
// side); max_core_doubles = the largest ka kb + kb kb
void launch_compress_batch(const Compress* d, int n, int max_core_doubles, double eps, cudaStream_t st);
void launch_apply_q(const double* A, int64_t lda, int rows_a, const double* tau_a, const double* TA, double* OA,
                    const double* B, int64_t ldb, int rows_b, const double* tau_b, const double* TB, double* OB,
                    int m, int r, cudaStream_t st);
// most columns a temporary may stack (the truncation kernels' per-column
// shared arrays)
constexpr int kCompressMax = 1024;
// vectors of the conjugate gradients
void launch_dot(const double* x, const double* y, int64_t n, double* partial, double* out, cudaStream_t st);
void launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st);
constexpr int kDotBlocks = 608;

}  // namespace h2
