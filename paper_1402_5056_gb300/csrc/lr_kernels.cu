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

// Doolittle LU without pivoting of one m x m block, one thread block
__global__ void k_leaf_lu(double* A, int m, int64_t lda, int* err) {
  for (int k = 0; k < m; ++k) {
    const double piv = A[k + k * lda];
    if (piv == 0.0 && threadIdx.x == 0) atomicOr(err, 256);   // zero pivot
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) A[i + k * lda] = A[i + k * lda] / piv;
    __syncthreads();
    const int mt = m - k - 1;
    for (int e = threadIdx.x; e < mt * mt; e += blockDim.x) {
      const int i = k + 1 + e % mt, j = k + 1 + e / mt;
      A[i + j * lda] = fma(-A[i + k * lda], A[k + j * lda], A[i + j * lda]);
    }
    __syncthreads();
  }
}

__global__ void k_trsm(int kind, const double* F, int m, int64_t ldf, double* X, int n, int64_t ldx) {
  for (int j = threadIdx.x + blockIdx.x * blockDim.x; j < n; j += blockDim.x * gridDim.x) {
    if (kind == 0) {          // column j of X: L x = y, unit lower
      double* x = X + j * ldx;
      for (int i = 0; i < m; ++i) {
        double v = x[i];
        for (int q = 0; q < i; ++q) v = fma(-F[i + q * ldf], x[q], v);
        x[i] = v;
      }
    } else if (kind == 1) {   // column j of X: R x = y, upper
      double* x = X + j * ldx;
      for (int i = m - 1; i >= 0; --i) {
        double v = x[i];
        for (int q = i + 1; q < m; ++q) v = fma(-F[i + q * ldf], x[q], v);
        x[i] = v / F[i + i * ldf];
      }
    } else {                  // row j of X: x R = y
      double* x = X + j;
      for (int i = 0; i < m; ++i) {
        double v = x[i * ldx];
        for (int q = 0; q < i; ++q) v = fma(-x[q * ldx], F[q + i * ldf], v);
        x[i * ldx] = v / F[i + i * ldf];
      }
    }
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
// Symmetric eigendecomposition A = V diag(w) V^* of an n x n matrix (global
// scratch, ld n, destroyed: its diagonal ends up as w) by two-sided Jacobi
// rotations (Golub and Van Loan, the symmetric Schur step) in a round-robin
// parallel ordering: each step rotates n/2 disjoint pairs at once, which
// commute.  One thread block; sweeps until the off-diagonal mass is below
// 1e-30 of the diagonal mass (at most 40 sweeps).
__device__ void jacobi_eig(double* A, double* V, int n, double* cs, double* sn, int* pp, int* qq) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n * n; e += nt) V[e] = (e % n == e / n) ? 1.0 : 0.0;
  __syncthreads();
  if (n < 2) return;
  const int n2 = n + (n & 1);
  __shared__ double red[2];
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) {
      double off = 0.0, dia = 0.0;
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          const double v = A[i + j * n];
          if (i == j) dia = fma(v, v, dia); else off = fma(v, v, off);
        }
      red[0] = off;
      red[1] = dia;
    }
    __syncthreads();
    if (!(red[0] > 1e-30 * red[1])) break;
    __syncthreads();
    for (int r = 0; r < n2 - 1; ++r) {
      // pairs of this round: player n2-1 meets r, player i meets (2r - i) mod (n2-1)
      for (int i = tid; i < n2 / 2; i += nt) {
        int p, q;
        if (i == 0) { p = r; q = n2 - 1; }
        else { p = (r + i) % (n2 - 1); q = (r - i + (n2 - 1)) % (n2 - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = A[p + q * n];
          if (apq != 0.0) {
            const double tau = (A[q + q * n] - A[p + p * n]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(fma(tau, tau, 1.0)));
            c = 1.0 / sqrt(fma(t, t, 1.0));
            s = t * c;
          }
        }
        pp[i] = p; qq[i] = q; cs[i] = c; sn[i] = s;
      }
      __syncthreads();
      const int np = n2 / 2;
      for (int e = tid; e < np * n; e += nt) {          // rows p, q: A <- J^* A
        const int i = e % np, j = e / np;
        const int p = pp[i], q = qq[i];
        if (q >= n) continue;
        const double a = A[p + j * n], b = A[q + j * n];
        A[p + j * n] = cs[i] * a - sn[i] * b;
        A[q + j * n] = sn[i] * a + cs[i] * b;
      }
      __syncthreads();
      for (int e = tid; e < np * n; e += nt) {          // columns p, q: A <- A J, V <- V J
        const int i = e % np, j = e / np;
        const int p = pp[i], q = qq[i];
        if (q >= n) continue;
        const double a = A[j + p * n], b = A[j + q * n];
        A[j + p * n] = cs[i] * a - sn[i] * b;
        A[j + q * n] = sn[i] * a + cs[i] * b;
        const double va = V[j + p * n], vb = V[j + q * n];
        V[j + p * n] = cs[i] * va - sn[i] * vb;
        V[j + q * n] = sn[i] * va + cs[i] * vb;
      }
      __syncthreads();
    }
  }
}

// Truncation of the factor pair (A, B), A B^* of rank <= m, from the Gram
// matrices GA = A^* A and GB = B^* B (m x m): with GA = VA diag(a) VA^*
// and GB = VB diag(b) VB^* (directions with a_i <= m 2^-52 max a dropped),
// Q_A = A VA a^-1/2 and Q_B = B VB b^-1/2 are orthonormal and
// A B^* = Q_A C Q_B^*, C = a^1/2 VA^* VB b^1/2.  The right singular vectors
// of C are the eigenvectors of C^* C; the rank r is the smallest with
// sum_{i>r} sigma_i^2 <= (eps/2)^2 sum sigma_i^2, and the truncated pair is
// A' = A TA, B' = B TB with TA = VA a^-1/2 C VC_r, TB = VB b^-1/2 VC_r (so
// B' has orthonormal columns and A' = Q_A U_r Sigma_r).  Scratch: 6 m*m
// doubles.  Writes TA, TB (m x m, ld m; first r columns) and *rank.
__global__ void k_compress(const double* GA, const double* GB, int m, double eps, double* scratch, double* TA,
                           double* TB, int* rank) {
  extern __shared__ double sm[];
  double* cs = sm;
  double* sn = sm + 128;
  int* pp = reinterpret_cast<int*>(sm + 256);
  int* qq = pp + 128;
  __shared__ int ka[256], kb[256], order[256];
  __shared__ int na, nb;
  double* EA = scratch;
  double* VA = scratch + m * m;
  double* EB = scratch + 2 * m * m;
  double* VB = scratch + 3 * m * m;
  double* C = scratch + 4 * m * m;
  double* VC = scratch + 5 * m * m;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < m * m; e += nt) {
    EA[e] = GA[e];
    EB[e] = GB[e];
  }
  __syncthreads();
  jacobi_eig(EA, VA, m, cs, sn, pp, qq);
  jacobi_eig(EB, VB, m, cs, sn, pp, qq);
  if (tid == 0) {
    double amax = 0.0, bmax = 0.0;
    for (int i = 0; i < m; ++i) {
      amax = fmax(amax, EA[i + i * m]);
      bmax = fmax(bmax, EB[i + i * m]);
    }
    const double tol = m * 2.220446049250313e-16;
    int x = 0, y = 0;
    for (int i = 0; i < m; ++i) {
      if (EA[i + i * m] > tol * amax) ka[x++] = i;
      if (EB[i + i * m] > tol * bmax) kb[y++] = i;
    }
    na = x;
    nb = y;
  }
  __syncthreads();
  // C (na x nb, ld m) = a^1/2 VA^* VB b^1/2 on the kept directions
  for (int e = tid; e < na * nb; e += nt) {
    const int i = e % na, j = e / na;
    const int ia = ka[i], jb = kb[j];
    double v = 0.0;
    for (int q = 0; q < m; ++q) v = fma(VA[q + ia * m], VB[q + jb * m], v);
    C[i + j * m] = sqrt(EA[ia + ia * m]) * v * sqrt(EB[jb + jb * m]);
  }
  __syncthreads();
  // CtC (nb x nb, ld nb) in the EA scratch, no longer needed past the diagonal
  double* wa = TA;   // diagonal of EA kept in TA's first column while EA is reused
  for (int i = tid; i < na; i += nt) wa[i] = EA[ka[i] + ka[i] * m];
  __syncthreads();
  double* M = EA;
  for (int e = tid; e < nb * nb; e += nt) {
    const int i = e % nb, j = e / nb;
    double v = 0.0;
    for (int q = 0; q < na; ++q) v = fma(C[q + i * m], C[q + j * m], v);
    M[i + j * nb] = v;
  }
  __syncthreads();
  jacobi_eig(M, VC, nb, cs, sn, pp, qq);
  if (tid == 0) {
    // eigenvalues in descending order, clamped at zero
    for (int i = 0; i < nb; ++i) order[i] = i;
    for (int i = 1; i < nb; ++i) {
      const int k = order[i];
      const double v = M[k + k * nb];
      int j = i - 1;
      while (j >= 0 && M[order[j] + order[j] * nb] < v) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = k;
    }
    double total = 0.0;
    for (int i = 0; i < nb; ++i) total += fmax(M[order[i] + order[i] * nb], 0.0);
    int r = nb;
    if (total == 0.0) {
      r = 0;
    } else {
      const double thr = 0.25 * eps * eps * total;
      double tail = 0.0;
      while (r > 0 && tail + fmax(M[order[r - 1] + order[r - 1] * nb], 0.0) <= thr) {
        tail += fmax(M[order[r - 1] + order[r - 1] * nb], 0.0);
        --r;
      }
    }
    *rank = r;
  }
  __syncthreads();
  const int r = *rank;
  // TB (m x r) = VB b^-1/2 VC_r ; TA (m x r) = VA a^-1/2 C VC_r
  for (int e = tid; e < m * r; e += nt) {
    const int i = e % m, j = e / m;
    const int cj = order[j];
    double vb = 0.0;
    for (int q = 0; q < nb; ++q) vb = fma(VB[i + kb[q] * m] / sqrt(EB[kb[q] + kb[q] * m]), VC[q + cj * nb], vb);
    TB[i + j * m] = vb;
  }
  __syncthreads();
  // CV = C VC_r (na x r) in the VC-free part of the scratch (EB is free now)
  double* CV = EB;
  for (int e = tid; e < na * r; e += nt) {
    const int i = e % na, j = e / na;
    const int cj = order[j];
    double v = 0.0;
    for (int q = 0; q < nb; ++q) v = fma(C[i + q * m], VC[q + cj * nb], v);
    CV[i + j * m] = v;
  }
  __syncthreads();
  double* waw = VC;   // VC is no longer needed: keep a^-1/2 there
  for (int i = tid; i < na; i += nt) waw[i] = 1.0 / sqrt(wa[i]);
  __syncthreads();
  for (int e = tid; e < m * r; e += nt) {
    const int i = e % m, j = e / m;
    double v = 0.0;
    for (int q = 0; q < na; ++q) v = fma(VA[i + ka[q] * m] * waw[q], CV[q + j * m], v);
    EA[i + j * m] = v;   // M (in EA) is no longer needed
  }
  __syncthreads();
  for (int e = tid; e < m * r; e += nt) TA[e % m + (e / m) * m] = EA[e % m + (e / m) * m];
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
  if (m > 0) k_leaf_lu<<<1, 256, 0, st>>>(A, m, lda, err);
}

void launch_trsm(int kind, const double* F, int m, int64_t ldf, double* X, int n, int64_t ldx, cudaStream_t st) {
  if (m <= 0 || n <= 0) return;
  const int threads = 64;
  k_trsm<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(kind, F, m, ldf, X, n, ldx);
}

void launch_compress(const double* GA, const double* GB, int m, double eps, double* scratch, double* TA,
                     double* TB, int* rank, cudaStream_t st) {
  k_compress<<<1, 256, 256 * sizeof(double) + 256 * sizeof(int), st>>>(GA, GB, m, eps, scratch, TA, TB, rank);
}

void launch_dot(const double* x, const double* y, int64_t n, double* partial, double* out, cudaStream_t st) {
  k_dot_partial<<<kDotBlocks, 256, 0, st>>>(x, y, n, partial);
  k_dot_final<<<1, 256, 0, st>>>(partial, kDotBlocks, out);
}

void launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st) {
  if (n > 0) k_axpby<<<kDotBlocks, 256, 0, st>>>(n, a, x, b, y);
}

}  // namespace h2
