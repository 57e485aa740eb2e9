// Kernels of the H^2-LR factorisation path (Section 3): products of one
// block of an H^2 matrix with dense columns, dense leaf factorisations and
// triangular solves, small dense products, and the vector operations of
// the preconditioned conjugate gradients.  All float64.
//
// Block products follow Eq. (vsw) with the nested bases of Eq. (nested)
// restricted to the block's subtrees: forward transformation over the
// X-side subtree, the couplings of the admissible leaves below the block,
// backward transformation over the Y-side subtree, and at the Y-side leaves
// the basis rows plus the rows of the inadmissible leaves below the block.
// One warp per cluster (lanes over the k x m entries or over the rows), one
// launch per tree level, as in the whole-matrix product.
#include <algorithm>

#include "h2_internal.h"
#include "lr.h"

namespace h2 {
namespace {

constexpr int kWarps = 4;

// sons of cluster c in depth-first preorder
__device__ __forceinline__ int sons0(int c) { return c + 1; }
__device__ __forceinline__ int sons1(const int32_t* subtree, int c) { return c + 1 + subtree[c + 1]; }

__global__ void k_bp_forward(BlockProd a, const int32_t* __restrict__ list, int n) {
  const int w = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const int c = list[w];
  const int kc = a.in.rank[c];
  const int kcap = a.kcap;
  double* out = a.xh + (size_t)c * kcap * a.m;
  const int ne = kc * a.m;
  if (a.in.subtree[c] == 1) {
    const int mc = a.in.size[c];
    const double* B = a.in.leaf + a.in.leaf_off[c];
    const double* X = a.X + (a.in.off[c] - a.in_off0);
    for (int e = lane; e < ne; e += 32) {
      const int i = e % kc, r = e / kc;
      double v = 0.0;
      for (int p = 0; p < mc; ++p) v = fma(B[p + (size_t)i * mc], X[p + r * a.ldx], v);
      out[i + r * kcap] = v;
    }
  } else {
    const int s0 = sons0(c), s1 = sons1(a.in.subtree, c);
    const int k0 = a.in.rank[s0], k1 = a.in.rank[s1];
    const double* E0 = a.in.transfer + (size_t)s0 * kcap * kcap;
    const double* E1 = a.in.transfer + (size_t)s1 * kcap * kcap;
    const double* x0 = a.xh + (size_t)s0 * kcap * a.m;
    const double* x1 = a.xh + (size_t)s1 * kcap * a.m;
    for (int e = lane; e < ne; e += 32) {
      const int i = e % kc, r = e / kc;
      double v = 0.0;
      for (int q = 0; q < k0; ++q) v = fma(E0[q + i * kcap], x0[q + r * kcap], v);
      for (int q = 0; q < k1; ++q) v = fma(E1[q + i * kcap], x1[q + r * kcap], v);
      out[i + r * kcap] = v;
    }
  }
}

__global__ void k_bp_coupling(BlockProd a, const int32_t* __restrict__ list, int n, const int32_t* __restrict__ ptr,
                              const int32_t* __restrict__ ent) {
  const int w = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const int c = list[w];
  const int kc = a.out.rank[c];
  const int kcap = a.kcap;
  double* out = a.yh + (size_t)c * kcap * a.m;
  const int ne = kc * a.m;
  for (int e = lane; e < ne; e += 32) {
    const int i = e % kc, r = e / kc;
    double v = 0.0;
    for (int x = ptr[w]; x < ptr[w + 1]; ++x) {
      const int slot = ent[2 * x], ci = ent[2 * x + 1];
      const int ki = a.in.rank[ci];
      const double* S = a.S + (size_t)slot * kcap * kcap;
      const double* xs = a.xh + (size_t)ci * kcap * a.m + (size_t)r * kcap;
      if (a.trans)
        for (int q = 0; q < ki; ++q) v = fma(S[q + i * kcap], xs[q], v);
      else
        for (int q = 0; q < ki; ++q) v = fma(S[i + q * kcap], xs[q], v);
    }
    out[i + r * kcap] = v;
  }
}

__global__ void k_bp_backward(BlockProd a, const int32_t* __restrict__ list, const int32_t* __restrict__ fathers,
                              int n) {
  const int w = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const int c = list[w], f = fathers[w];
  const int kc = a.out.rank[c], kf = a.out.rank[f];
  const int kcap = a.kcap;
  const double* E = a.out.transfer + (size_t)c * kcap * kcap;
  const double* yf = a.yh + (size_t)f * kcap * a.m;
  double* out = a.yh + (size_t)c * kcap * a.m;
  const int ne = kc * a.m;
  for (int e = lane; e < ne; e += 32) {
    const int i = e % kc, r = e / kc;
    double v = out[i + r * kcap];
    for (int q = 0; q < kf; ++q) v = fma(E[i + q * kcap], yf[q + r * kcap], v);
    out[i + r * kcap] = v;
  }
}

__global__ void k_bp_leaves(BlockProd a, const int32_t* __restrict__ leaves, int n, const int32_t* __restrict__ ptr,
                            const int32_t* __restrict__ ent) {
  const int w = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const int l = leaves[w];
  const int ml = a.out.size[l];
  const int kl = a.out.rank[l];
  const int kcap = a.kcap;
  const double* V = a.out.leaf + a.out.leaf_off[l];
  const double* yl = a.yh + (size_t)l * kcap * a.m;
  const int64_t loff = a.out.off[l];
  double* Y = a.Y + (loff - a.out_off0);
  const int ne = ml * a.m;
  for (int e = lane; e < ne; e += 32) {
    const int p = e % ml, r = e / ml;
    double v = 0.0;
    for (int i = 0; i < kl; ++i) v = fma(V[p + (size_t)i * ml], yl[i + r * kcap], v);
    for (int x = ptr[w]; x < ptr[w + 1]; ++x) {
      const int slot = ent[3 * x], ci = ent[3 * x + 1], co = ent[3 * x + 2];
      const double* N = a.N + a.near_off[slot];
      const int mi = a.in.size[ci], mo = a.out.size[co];
      const int po = (int)(loff - a.out.off[co]) + p;       // row of the leaf inside the Y-side cluster
      const double* X = a.X + (a.in.off[ci] - a.in_off0) + r * a.ldx;
      if (a.trans)   // N is mi x mo (ld mi): rows of N^* are its columns
        for (int j = 0; j < mi; ++j) v = fma(N[j + (size_t)po * mi], X[j], v);
      else           // N is mo x mi (ld mo)
        for (int j = 0; j < mi; ++j) v = fma(N[po + (size_t)j * mo], X[j], v);
    }
    Y[p + r * a.ldy] += a.alpha * v;
  }
}

__global__ void k_identity(double* yh, int k, int kcap) {
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;
    yh[i + j * kcap] = i == j ? 1.0 : 0.0;
  }
}

// C = alpha op(A) op(B) + beta C, one thread per entry of C
__global__ void k_gemm(int m, int n, int k, double alpha, const double* A, int64_t lda, int ta, const double* B,
                       int64_t ldb, int tb, double beta, double* C, int64_t ldc) {
  const int i = blockIdx.x * 16 + threadIdx.x;
  const int j = blockIdx.y * 16 + threadIdx.y;
  if (i >= m || j >= n) return;
  double v = 0.0;
  for (int q = 0; q < k; ++q) {
    const double x = ta ? A[q + i * lda] : A[i + q * lda];
    const double y = tb ? B[j + q * ldb] : B[q + j * ldb];
    v = fma(x, y, v);
  }
  double* c = C + i + j * ldc;
  *c = beta == 0.0 ? alpha * v : fma(beta, *c, alpha * v);
}

// B (n x m) = alpha A^* (A m x n)
__global__ void k_transpose(int m, int n, double alpha, const double* A, int64_t lda, double* B, int64_t ldb) {
  const int i = blockIdx.x * 16 + threadIdx.x;   // row of A
  const int j = blockIdx.y * 16 + threadIdx.y;   // column of A
  if (i < m && j < n) B[j + i * ldb] = alpha * A[i + j * lda];
}

__global__ void k_eye(double* A, int n, int64_t lda) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n; e += (int64_t)blockDim.x * gridDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    A[i + j * lda] = i == j ? 1.0 : 0.0;
  }
}

// Doolittle LU without pivoting of one m x m block (m <= 64), one warp:
// lane i owns rows i and i + 32; step k scales column k below the pivot and
// updates the trailing rows (the same order of operations as the textbook
// loop, so the same rounding)
__global__ void k_leaf_lu(double* A, int m, int64_t lda, int* err) {
  const int lane = threadIdx.x;
  for (int k = 0; k < m; ++k) {
    const double piv = A[k + k * lda];
    if (piv == 0.0 && lane == 0) atomicOr(err, 256);   // zero pivot
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      if (i > k && i < m) {
        const double l = A[i + k * lda] / piv;
        A[i + k * lda] = l;
        for (int j = k + 1; j < m; ++j) A[i + j * lda] = fma(-l, A[k + j * lda], A[i + j * lda]);
      }
    }
    __syncwarp();
  }
}

// Cholesky factor of a dense m x m leaf (m <= 64) in place, one warp, lane
// i holding rows i and i + 32: right-looking, column k scaled by the root
// of its pivot, then the lower triangle of the trailing block updated; the
// strictly upper part is set to zero.  A pivot that is not positive sets
// bit 512 of err (the matrix is not positive definite).
__global__ void k_leaf_chol(double* A, int m, int64_t lda, int* err) {
  const int lane = threadIdx.x;
  for (int k = 0; k < m; ++k) {
    const double piv = A[k + k * lda];
    if (!(piv > 0.0) && lane == 0) atomicOr(err, 512);
    const double rt = sqrt(piv);
    __syncwarp();
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      if (i > k && i < m) A[i + k * lda] = A[i + k * lda] / rt;
      if (i == k) A[k + k * lda] = rt;
    }
    __syncwarp();
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      if (i > k && i < m) {
        const double l = A[i + k * lda];
        for (int j = k + 1; j <= i; ++j) A[i + j * lda] = fma(-l, A[j + k * lda], A[i + j * lda]);
      }
    }
    __syncwarp();
  }
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    if (i < m)
      for (int j = i + 1; j < m; ++j) A[i + j * lda] = 0.0;
  }
}

// Triangular solves with an m x m factor (m <= 64), one warp per
// right-hand side, lane i holding entries i and i + 32; the solved entry of
// each step is broadcast and the others updated column by column
//   kind 0: column j of X, L x = y (unit lower)
//   kind 1: column j of X, R x = y (upper)
//   kind 2: row j of X, x R = y
//   kind 3: column j of X, L x = y (lower with its diagonal)
//   kind 4: column j of X, L^* x = y (L lower with its diagonal)
__global__ void k_trsm(int kind, const double* F, int m, int64_t ldf, double* X, int n, int64_t ldx) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= n) return;
  const int64_t stride = kind == 2 ? ldx : 1;
  double* x = kind == 2 ? X + j : X + j * ldx;
  double r[2];
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    r[h] = i < m ? x[i * stride] : 0.0;
  }
  if (kind == 3) {
    for (int k = 0; k < m; ++k) {
      const int hk = k >> 5;
      if ((k & 31) == lane) r[hk] = r[hk] / F[k + k * ldf];
      const double xk = __shfl_sync(0xffffffffu, hk ? r[1] : r[0], k & 31);
      for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        if (i > k && i < m) r[h] = fma(-F[i + k * ldf], xk, r[h]);
      }
    }
  } else if (kind == 4) {
    for (int k = m - 1; k >= 0; --k) {
      const int hk = k >> 5;
      if ((k & 31) == lane) r[hk] = r[hk] / F[k + k * ldf];
      const double xk = __shfl_sync(0xffffffffu, hk ? r[1] : r[0], k & 31);
      for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        if (i < k) r[h] = fma(-F[k + i * ldf], xk, r[h]);
      }
    }
  } else if (kind == 0) {
    for (int k = 0; k < m; ++k) {
      const double xk = __shfl_sync(0xffffffffu, k < 32 ? r[0] : r[1], k & 31);
      for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        if (i > k && i < m) r[h] = fma(-F[i + k * ldf], xk, r[h]);
      }
    }
  } else if (kind == 1) {
    for (int k = m - 1; k >= 0; --k) {
      const int hk = k >> 5;
      if ((k & 31) == lane) r[hk] = r[hk] / F[k + k * ldf];
      const double xk = __shfl_sync(0xffffffffu, hk ? r[1] : r[0], k & 31);
      for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        if (i < k) r[h] = fma(-F[i + k * ldf], xk, r[h]);
      }
    }
  } else {
    for (int q = 0; q < m; ++q) {
      const int hq = q >> 5;
      if ((q & 31) == lane) r[hq] = r[hq] / F[q + q * ldf];
      const double xq = __shfl_sync(0xffffffffu, hq ? r[1] : r[0], q & 31);
      for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        if (i > q && i < m) r[h] = fma(-xq, F[q + i * ldf], r[h]);
      }
    }
  }
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    if (i < m) x[i * stride] = r[h];
  }
}

// deterministic dot product: fixed grid, per-block tree sums, one final sum
__global__ void k_dot_partial(const double* x, const double* y, int64_t n, double* partial) {
  __shared__ double sh[256];
  double v = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)blockDim.x * gridDim.x)
    v = fma(x[i], y[i], v);
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_dot_final(const double* partial, int np, double* out) {
  __shared__ double sh[256];
  double v = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) v += partial[i];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_axpby(int64_t n, double a, const double* x, double b, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)blockDim.x * gridDim.x)
    y[i] = b == 0.0 ? a * x[i] : fma(a, x[i], b * y[i]);
}

// ------------------------------------------------ factor-pair compression
// Truncation of a factor pair (A, B) with m columns (m <= kCompressMax):
//  1. Householder QR of A (rows_a x m) and of B, in place, one thread block
//     per factor: reflection j maps column j below the diagonal to zero
//     (H = I - tau v v^*, v_j = 1, beta = -sign(alpha) ||x||, the form of
//     LAPACK's dlarfg); R in the upper triangle, v below it;
//  2. the core C = R_A R_B^* (ka x kb, ka = min(rows_a, m)), its SVD by
//     one-sided Jacobi on the columns (C W = U Sigma), the rank r = the
//     smallest with sum_{i>r} sigma_i^2 <= (eps/2)^2 sum sigma_i^2;
//  3. A' = Q_A [U_r Sigma_r; 0], B' = Q_B [W_r; 0] by the reflections in
//     reverse order.
// A' B'^* is the truncated A B^* (B' has orthonormal columns).

// QR of the rows x m matrix X (ld ldx) in place; tau (m entries).  One block.
__device__ __forceinline__ void house_qr_one(double* X, int64_t ldx, int rows, int m, double* tau, int* nonzero) {
  __shared__ double red[32];
  __shared__ double sh_beta, sh_tau, sh_scale;
  __shared__ int any;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  // an all-zero factor (most temporaries of the factorisation have one):
  // the product is zero and the core SVD returns rank 0 at once
  if (tid == 0) any = 0;
  __syncthreads();
  int mine = 0;
  for (int64_t e = tid; e < (int64_t)rows * m; e += nt)
    if (X[e % rows + (e / rows) * ldx] != 0.0) mine = 1;
  if (__any_sync(0xffffffffu, mine) && lane == 0) any = 1;
  __syncthreads();
  if (tid == 0) *nonzero = any;
  if (!any) {
    for (int j = tid; j < m; j += nt) tau[j] = 0.0;
    return;
  }
  const int kk = min(rows, m);
  for (int j = 0; j < kk; ++j) {
    double* x = X + j + (int64_t)j * ldx;       // column j from the diagonal down
    const int len = rows - j;
    double s = 0.0;
    for (int i = 1 + tid; i < len; i += nt) s = fma(x[i], x[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (tid == 0) {
      double sig = 0.0;
      for (int w = 0; w < nw; ++w) sig += red[w];
      const double alpha = x[0];
      if (sig == 0.0) {
        sh_tau = 0.0;
        sh_beta = alpha;
        sh_scale = 0.0;
      } else {
        const double nrm = sqrt(fma(alpha, alpha, sig));
        const double beta = alpha >= 0.0 ? -nrm : nrm;
        sh_tau = (beta - alpha) / beta;
        sh_scale = 1.0 / (alpha - beta);
        sh_beta = beta;
      }
      tau[j] = sh_tau;
    }
    __syncthreads();
    const double t = sh_tau;
    if (t != 0.0)
      for (int i = 1 + tid; i < len; i += nt) x[i] *= sh_scale;
    __syncthreads();
    if (tid == 0) x[0] = sh_beta;
    // apply H to the columns j+1..m-1: one warp per column
    if (t != 0.0)
      for (int c = j + 1 + warp; c < m; c += nw) {
        double* y = X + j + (int64_t)c * ldx;
        double w = lane == 0 ? y[0] : 0.0;
        for (int i = 1 + lane; i < len; i += 32) w = fma(x[i], y[i], w);
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        w *= t;
        if (lane == 0) y[0] -= w;
        for (int i = 1 + lane; i < len; i += 32) y[i] = fma(-w, x[i], y[i]);
      }
    __syncthreads();
  }
}

// every temporary of a product at once: block (side, temporary)
__global__ void __launch_bounds__(512) k_house_qr_batch(const Compress* __restrict__ d, int n) {
  const Compress c = d[blockIdx.y];
  if (blockIdx.x == 0) house_qr_one(c.A, c.mt, c.mt, c.m, c.tauA, c.flags + 1);
  else house_qr_one(c.B, c.mr, c.mr, c.m, c.tauB, c.flags + 2);
  (void)n;
}

__device__ __forceinline__ int rr_partner(int i, int r, int n2, int& p, int& q) {
  if (i == 0) { p = r; q = n2 - 1; }
  else { p = (r + i) % (n2 - 1); q = (r - i + (n2 - 1)) % (n2 - 1); }
  if (p > q) { const int t = p; p = q; q = t; }
  return 0;
}

// One-sided Jacobi on the cols columns of X (rows x cols, ld ldx): X V = U
// Sigma, the rotations accumulated into V (cols x cols, ld ldv).  Round-
// robin pairs, one warp a pair.  Columns whose squared norm is below 1e-28
// of the largest are at the rounding level of the product: they are not
// rotated (rotating them need not converge, and they lie far below any
// truncation threshold).  Rotate while |gamma| > 64 u sqrt(alpha beta): a
// smaller threshold lies below the rounding of the dot products (up to 1024
// terms) and the sweeps would not end.  nrm2 (cols) is scratch.
__device__ __forceinline__ void jacobi_cols(double* X, int ldx, int rows, int cols, double* V, int ldv,
                                            double* nrm2) {
  __shared__ int any_rot;
  __shared__ double tiny;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int j = tid; j < cols; j += nt) {
    double v = 0.0;
    for (int k = 0; k < rows; ++k) v = fma(X[k + j * ldx], X[k + j * ldx], v);
    nrm2[j] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    for (int j = 0; j < cols; ++j) mx = fmax(mx, nrm2[j]);
    tiny = 1e-28 * mx;
  }
  __syncthreads();
  const int n2 = cols + (cols & 1);
  const double tol2 = (64.0 * 2.220446049250313e-16) * (64.0 * 2.220446049250313e-16);
  for (int sweep = 0; sweep < 40 && cols > 1; ++sweep) {
    if (tid == 0) any_rot = 0;
    __syncthreads();
    for (int r = 0; r < n2 - 1; ++r) {
      for (int i = warp; i < n2 / 2; i += nw) {
        int p, q;
        rr_partner(i, r, n2, p, q);
        if (q >= cols) continue;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int k = lane; k < rows; k += 32) {
          const double x = X[k + p * ldx], y = X[k + q * ldx];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (ga * ga > tol2 * al * be && ga != 0.0 && al > tiny && be > tiny) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
          const double c = 1.0 / sqrt(fma(t, t, 1.0)), s = c * t;
          for (int k = lane; k < rows; k += 32) {
            const double x = X[k + p * ldx], y = X[k + q * ldx];
            X[k + p * ldx] = c * x - s * y;
            X[k + q * ldx] = s * x + c * y;
          }
          for (int k = lane; k < cols; k += 32) {
            const double x = V[k + p * ldv], y = V[k + q * ldv];
            V[k + p * ldv] = c * x - s * y;
            V[k + q * ldv] = s * x + c * y;
          }
          if (lane == 0) any_rot = 1;
        }
      }
      __syncthreads();
    }
    if (!any_rot) break;
    __syncthreads();
  }
  // squared column norms = sigma^2
  for (int j = tid; j < cols; j += nt) {
    double v = 0.0;
    for (int k = 0; k < rows; ++k) v = fma(X[k + j * ldx], X[k + j * ldx], v);
    nrm2[j] = v;
  }
  __syncthreads();
}

// Descending order of the squared singular values nrm2 (cols) and the rank
// rule: the smallest r with sum_{i>r} sigma_i^2 <= (eps/2)^2 sum sigma_i^2.
// Thread 0 writes order and *rank; every thread returns the rank.
__device__ __forceinline__ int rank_rule(const double* nrm2, int* order, int cols, double eps, int* rank) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < cols; ++i) order[i] = i;
    for (int i = 1; i < cols; ++i) {
      const int k = order[i];
      int j = i - 1;
      while (j >= 0 && nrm2[order[j]] < nrm2[k]) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = k;
    }
    double total = 0.0;
    for (int i = 0; i < cols; ++i) total += nrm2[i];
    int r = cols;
    if (total == 0.0) {
      r = 0;
    } else {
      const double thr = 0.25 * eps * eps * total;
      double tail = 0.0;
      while (r > 0 && tail + nrm2[order[r - 1]] <= thr) {
        tail += nrm2[order[r - 1]];
        --r;
      }
    }
    *rank = r;
  }
  __syncthreads();
  return *rank;
}

// Core SVD and rank.  C (ka x kb, ld m, scratch), W (kb x kb, ld m,
// scratch); writes T = U_r Sigma_r (ka x r, ld m) into TA and the right
// singular vectors W_r (kb x r, ld m) into TB, the rank into *rank.  One
// block.  With in_smem, C and W live in dynamic shared memory instead (ld ka
// and kb).
//
// Up to 32 columns the one-sided Jacobi runs on C itself.  Wider cores (a
// temporary stacking many terms) first go through a Householder QR with
// column pivoting, C P = Q R, stopped once the trailing columns' norm is at
// the rounding level of C (below 1e-15 ||C||_F): C = Q_p R_p P^* up to that
// remainder, p the numerical rank.  The Jacobi then runs on the p columns of
// M = R_p^* (kb x p): M V = U_M Sigma, so C = (Q_p V) Sigma (P U_M)^* -- the
// same singular values and vectors as a Jacobi on all kb columns, with p^2
// instead of kb^2 pairs.
__device__ __forceinline__ void core_svd_one(const double* XA, int64_t lda, int ka, const double* XB, int64_t ldb,
                                             int kb, int m, double eps, const int* nonzero, double* Cg, double* Wg,
                                             double* TA, double* TB, int* rank, int in_smem) {
  extern __shared__ double csm[];
  __shared__ int order[kCompressMax];
  __shared__ double nrm2[kCompressMax];
  __shared__ int perm[kCompressMax];
  __shared__ double tauc[kCompressMax];
  __shared__ int sh_p, sh_piv;
  __shared__ double sh_beta, sh_tau, sh_scale, sh_delta2;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  if (!nonzero[0] || !nonzero[1]) {   // A B^* = 0
    if (tid == 0) *rank = 0;
    return;
  }
  double* C = in_smem ? csm : Cg;
  double* W = in_smem ? csm + ka * kb : Wg;
  const int lc = in_smem ? ka : m;   // leading dimensions of C and W
  const int lw = in_smem ? kb : m;
  // C = R_A R_B^* (upper triangles)
  for (int e = tid; e < ka * kb; e += nt) {
    const int i = e % ka, j = e / ka;
    double v = 0.0;
    for (int q = max(i, j); q < m; ++q) v = fma(XA[i + (int64_t)q * lda], XB[j + (int64_t)q * ldb], v);
    C[i + j * lc] = v;
  }
  if (kb <= 32) {
    for (int e = tid; e < kb * kb; e += nt) W[e % kb + (e / kb) * lw] = (e % kb == e / kb) ? 1.0 : 0.0;
    __syncthreads();
    jacobi_cols(C, lc, ka, kb, W, lw, nrm2);
    const int r = rank_rule(nrm2, order, kb, eps, rank);
    for (int e = tid; e < ka * r; e += nt) TA[e % ka + (e / ka) * m] = C[e % ka + order[e / ka] * lc];
    for (int e = tid; e < kb * r; e += nt) TB[e % kb + (e / kb) * m] = W[e % kb + order[e / kb] * lw];
    return;
  }
  // Householder QR with column pivoting, stopped at the rounding level
  for (int c = tid; c < kb; c += nt) perm[c] = c;
  __syncthreads();
  const int kk = min(ka, kb);
  if (tid == 0) sh_p = kk;
  for (int j = 0; j < kk; ++j) {
    // norms of the trailing columns over the rows j..ka-1
    for (int c = j + warp; c < kb; c += nw) {
      double v = 0.0;
      for (int i = j + lane; i < ka; i += 32) v = fma(C[i + c * lc], C[i + c * lc], v);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) nrm2[c] = v;
    }
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0, best = -1.0;
      int piv = j;
      for (int c = j; c < kb; ++c) {
        tot += nrm2[c];
        if (nrm2[c] > best) {
          best = nrm2[c];
          piv = c;
        }
      }
      if (j == 0) sh_delta2 = 1e-30 * tot;
      if (tot <= sh_delta2) {
        sh_p = j;
        piv = -1;
      } else {
        const int t = perm[j];
        perm[j] = perm[piv];
        perm[piv] = t;
      }
      sh_piv = piv;
    }
    __syncthreads();
    const int piv = sh_piv;
    if (piv < 0) break;
    if (piv != j)
      for (int i = tid; i < ka; i += nt) {
        const double t = C[i + j * lc];
        C[i + j * lc] = C[i + piv * lc];
        C[i + piv * lc] = t;
      }
    __syncthreads();
    // reflection of column j (rows j..ka-1), the form of LAPACK's dlarfg
    double* x = C + j + j * lc;
    const int len = ka - j;
    if (tid < 32) {
      double sv = 0.0;
      for (int i = 1 + lane; i < len; i += 32) sv = fma(x[i], x[i], sv);
      for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
      if (lane == 0) {
        const double alpha = x[0];
        if (sv == 0.0) {
          sh_tau = 0.0;
          sh_beta = alpha;
          sh_scale = 0.0;
        } else {
          const double nrm = sqrt(fma(alpha, alpha, sv));
          const double beta = alpha >= 0.0 ? -nrm : nrm;
          sh_tau = (beta - alpha) / beta;
          sh_scale = 1.0 / (alpha - beta);
          sh_beta = beta;
        }
        tauc[j] = sh_tau;
      }
    }
    __syncthreads();
    const double t = sh_tau;
    if (t != 0.0)
      for (int i = 1 + tid; i < len; i += nt) x[i] *= sh_scale;
    __syncthreads();
    if (tid == 0) x[0] = sh_beta;
    // apply H to the columns j+1..kb-1: one warp per column
    if (t != 0.0)
      for (int c = j + 1 + warp; c < kb; c += nw) {
        double* y = C + j + c * lc;
        double w = lane == 0 ? y[0] : 0.0;
        for (int i = 1 + lane; i < len; i += 32) w = fma(x[i], y[i], w);
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        w *= t;
        if (lane == 0) y[0] -= w;
        for (int i = 1 + lane; i < len; i += 32) y[i] = fma(-w, x[i], y[i]);
      }
    __syncthreads();
  }
  __syncthreads();
  const int p = sh_p;
  if (p == 0) {
    if (tid == 0) *rank = 0;
    return;
  }
  // M = R_p^* (kb x p) in W, V = I (p x p) in TB
  for (int e = tid; e < kb * p; e += nt) {
    const int c = e % kb, j = e / kb;
    W[c + j * lw] = c >= j ? C[j + c * lc] : 0.0;
  }
  for (int e = tid; e < p * p; e += nt) TB[e % p + (e / p) * m] = (e % p == e / p) ? 1.0 : 0.0;
  __syncthreads();
  jacobi_cols(W, lw, kb, p, TB, m, nrm2);
  const int r = rank_rule(nrm2, order, p, eps, rank);
  // TA = Q_p [V_r Sigma_r; 0]: one warp per column, the reflections in
  // reverse order
  for (int i = warp; i < r; i += nw) {
    const int jc = order[i];
    const double sg = sqrt(nrm2[jc]);
    double* y = TA + (int64_t)i * m;
    for (int k = lane; k < ka; k += 32) y[k] = k < p ? TB[k + jc * m] * sg : 0.0;
    __syncwarp();
    for (int j = p - 1; j >= 0; --j) {
      const double t = tauc[j];
      if (t == 0.0) continue;
      const double* v = C + j + j * lc;   // v_0 = 1 implied
      const int len = ka - j;
      double w = lane == 0 ? y[j] : 0.0;
      for (int k = 1 + lane; k < len; k += 32) w = fma(v[k], y[j + k], w);
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      w *= t;
      __syncwarp();
      if (lane == 0) y[j] -= w;
      for (int k = 1 + lane; k < len; k += 32) y[j + k] = fma(-w, v[k], y[j + k]);
      __syncwarp();
    }
  }
  __syncthreads();   // V (in TB) is read; TB now receives P U_M
  for (int e = tid; e < kb * r; e += nt) {
    const int c = e % kb, i = e / kb;
    const int jc = order[i];
    TB[perm[c] + (int64_t)i * m] = W[c + jc * lw] / sqrt(nrm2[jc]);
  }
}

// every temporary of a product at once, one block each; C and W in shared
// memory when ka kb + kb kb <= smem_doubles
__global__ void __launch_bounds__(1024) k_core_svd_batch(const Compress* __restrict__ d, int n, double eps,
                                                         int smem_doubles) {
  const Compress c = d[blockIdx.x];
  const int in_smem = c.ka * c.kb + c.kb * c.kb <= smem_doubles ? 1 : 0;
  core_svd_one(c.A, c.mt, c.ka, c.B, c.mr, c.kb, c.m, eps, c.flags + 1, c.C, c.W, c.TA, c.TB, c.flags, in_smem);
  (void)n;
}

// out (rows x r, ld ldo) = Q [T; 0] with Q = H_0 H_1 ... H_{k-1} stored in X
// (reflections below the diagonal, tau); T is k x r (ld ldt).  One block
// per factor (blockIdx 0: A side, 1: B side).
__global__ void __launch_bounds__(512) k_apply_q(const double* XA, int64_t lda, int rows_a, const double* tau_a, const double* TA,
                          double* OA, const double* XB, int64_t ldb, int rows_b, const double* tau_b,
                          const double* TB, double* OB, int m, int r) {
  const bool sa = blockIdx.x == 0;
  const double* X = sa ? XA : XB;
  const int64_t ldx = sa ? lda : ldb;
  const int rows = sa ? rows_a : rows_b;
  const double* tau = sa ? tau_a : tau_b;
  const double* T = sa ? TA : TB;
  double* O = sa ? OA : OB;
  const int k = min(rows, m);
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int e = tid; e < rows * r; e += nt) {
    const int i = e % rows, c = e / rows;
    O[i + (int64_t)c * rows] = i < k ? T[i + c * m] : 0.0;
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const double t = tau[j];
    if (t == 0.0) continue;
    const double* v = X + j + (int64_t)j * ldx;   // v_0 = 1 implied
    const int len = rows - j;
    for (int c = warp; c < r; c += nw) {
      double* y = O + j + (int64_t)c * rows;
      double w = lane == 0 ? y[0] : 0.0;
      for (int i = 1 + lane; i < len; i += 32) w = fma(v[i], y[i], w);
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      w *= t;
      if (lane == 0) y[0] -= w;
      for (int i = 1 + lane; i < len; i += 32) y[i] = fma(-w, v[i], y[i]);
    }
    __syncthreads();
  }
}

inline unsigned warps_grid(int n) { return (unsigned)((n + kWarps - 1) / kWarps); }

}  // namespace

void launch_bp_forward(const BlockProd& a, const int32_t* list, int n, cudaStream_t st) {
  if (n > 0) k_bp_forward<<<warps_grid(n), 32 * kWarps, 0, st>>>(a, list, n);
}

void launch_bp_coupling(const BlockProd& a, const int32_t* list, int n, const int32_t* ptr, const int32_t* ent,
                        cudaStream_t st) {
  if (n > 0) k_bp_coupling<<<warps_grid(n), 32 * kWarps, 0, st>>>(a, list, n, ptr, ent);
}

void launch_bp_backward(const BlockProd& a, const int32_t* list, const int32_t* fathers, int n, cudaStream_t st) {
  if (n > 0) k_bp_backward<<<warps_grid(n), 32 * kWarps, 0, st>>>(a, list, fathers, n);
}

void launch_bp_leaves(const BlockProd& a, const int32_t* leaves, int n, const int32_t* ptr, const int32_t* ent,
                      cudaStream_t st) {
  if (n > 0) k_bp_leaves<<<warps_grid(n), 32 * kWarps, 0, st>>>(a, leaves, n, ptr, ent);
}

void launch_identity(double* yh, int k, int kcap, cudaStream_t st) {
  if (k > 0) k_identity<<<1, 256, 0, st>>>(yh, k, kcap);
}

void launch_gemm(int m, int n, int k, double alpha, const double* A, int64_t lda, int ta, const double* B,
                 int64_t ldb, int tb, double beta, double* C, int64_t ldc, cudaStream_t st) {
  if (m <= 0 || n <= 0) return;
  dim3 grid((m + 15) / 16, (n + 15) / 16);
  k_gemm<<<grid, dim3(16, 16), 0, st>>>(m, n, k, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc);
}

void launch_transpose(int m, int n, double alpha, const double* A, int64_t lda, double* B, int64_t ldb,
                      cudaStream_t st) {
  if (m <= 0 || n <= 0) return;
  dim3 grid((m + 15) / 16, (n + 15) / 16);
  k_transpose<<<grid, dim3(16, 16), 0, st>>>(m, n, alpha, A, lda, B, ldb);
}

void launch_eye(double* A, int n, int64_t lda, cudaStream_t st) {
  if (n > 0) k_eye<<<(unsigned)std::min<int64_t>(((int64_t)n * n + 255) / 256, 1024), 256, 0, st>>>(A, n, lda);
}

void launch_leaf_lu(double* A, int m, int64_t lda, int* err, cudaStream_t st) {
  if (m > 0) k_leaf_lu<<<1, 32, 0, st>>>(A, m, lda, err);
}

void launch_leaf_chol(double* A, int m, int64_t lda, int* err, cudaStream_t st) {
  if (m > 0) k_leaf_chol<<<1, 32, 0, st>>>(A, m, lda, err);
}

void launch_trsm(int kind, const double* F, int m, int64_t ldf, double* X, int n, int64_t ldx, cudaStream_t st) {
  if (m <= 0 || n <= 0) return;
  const int warps = 4;
  k_trsm<<<(unsigned)((n + warps - 1) / warps), 32 * warps, 0, st>>>(kind, F, m, ldf, X, n, ldx);
}

void launch_compress_batch(const Compress* d, int n, int max_core_doubles, double eps, cudaStream_t st) {
  if (n <= 0) return;
  k_house_qr_batch<<<dim3(2, n), 512, 0, st>>>(d, n);
  constexpr size_t kMax = 160 * 1024;
  static std::atomic<unsigned long long> attr{0};
  const size_t bytes = (size_t)max_core_doubles * sizeof(double);
  const int fit = bytes <= kMax ? max_core_doubles : 0;
  if (fit) smem_limit(k_core_svd_batch, kMax, attr);
  k_core_svd_batch<<<n, 1024, (size_t)fit * sizeof(double), st>>>(d, n, eps, fit);
}

void launch_apply_q(const double* A, int64_t lda, int rows_a, const double* tau_a, const double* TA, double* OA,
                    const double* B, int64_t ldb, int rows_b, const double* tau_b, const double* TB, double* OB,
                    int m, int r, cudaStream_t st) {
  if (r > 0) k_apply_q<<<2, 512, 0, st>>>(A, lda, rows_a, tau_a, TA, OA, B, ldb, rows_b, tau_b, TB, OB, m, r);
}

void launch_dot(const double* x, const double* y, int64_t n, double* partial, double* out, cudaStream_t st) {
  k_dot_partial<<<kDotBlocks, 256, 0, st>>>(x, y, n, partial);
  k_dot_final<<<1, 256, 0, st>>>(partial, kDotBlocks, out);
}

void launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st) {
  if (n > 0) k_axpby<<<kDotBlocks, 256, 0, st>>>(n, a, x, b, y);
}

}  // namespace h2
