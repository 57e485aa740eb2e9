// Certified Gram path of the local low-rank update (Sections 4 and 5).
//
// When the truncation of every cluster of an update keeps the full extended
// rank K_t = k_t + u -- every singular value of V^_t B~_t^* above the
// threshold of the rank rule -- the new basis of t spans range(V~_t), and
// every quantity of steps 2-4 follows from K_t x K_t Gram matrices:
//   G_t = V~_t^* V~_t = R_t^* R_t = [[V_t^* V_t, C_t], [C_t^*, N_t]],
//         C_t = V_t^* A|_t, N_t = A|_t^* A|_t  (inner clusters: C_t = sum over
//         the sons of E_s^* C_s, N_t = sum of N_s)
//   ||Z~|_b||_F^2 = tr(S~_b^* G_t S~_b G_s)
//   W_t = B~_t^* B~_t  (sum of omega_b^2 S~_b G_s S~_b^* over row(t), plus
//                       E~_t W_{t+} E~_t^*)
//   sigma_i(V^_t B~_t^*)^2 = lambda_i(G_t W_t) = lambda_i(L^* W_t L), G_t = L L^*.
// The certificate is an LDL^* factorisation of L^* W_t L - (tau + delta) I
// with positive pivots, tau = (eps/2)^2 the threshold of the rank rule and
// delta a bound on the rounding of G_t, W_t and the factorisations.  When it
// holds the rank rule keeps all K_t columns and any orthonormal basis of
// range(V~_t) gives the same projection as the singular vectors; the path
// takes Q_t = V~_t L^{-*} (orthonormal: Q_t^* Q_t = L^{-1} G_t L^{-*} = I),
// R_t = Q_t^* V~_t = L^*, new transfer matrices L_s^* E~_s L_t^{-*} and the
// commit E_t0 <- L_t0^* [E_t0; 0].  An update for which any cluster fails
// the certificate is recomputed by the exact path (Householder R-factors
// and a one-sided Jacobi SVD).
//
// Orthonormal bases (V_t^* V_t = I, the normal case) make L block
// triangular: L = [[I, 0], [C_t^*, L_S]] with L_S L_S^* = N_t - C_t^* C_t, so
// the new basis is (V_t, (A|_t - V_t C_t) L_S^{-*}): the old basis is kept
// and extended by the orthonormalised new directions, the factorisation of
// G_t shrinks to u x u, and R_t [S_b; 0] = [S_b; 0] turns the one-sided
// reprojections into copies.
//
// Execution model: one warp per cluster (or block) task, small tiles in
// shared memory, and every matrix product spread over all 32 lanes (lane
// takes entries lane, lane + 32, ... of the result), so that float64
// instructions run with full lanes; symmetric results are computed on their
// lower triangle only.
#include <cfloat>

#include "h2_internal.h"
#include "update_kernels.h"

namespace h2 {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kLd = 33;     // leading dimension of the shared tiles (up to 32 rows)
constexpr int kNS = 17;     // lower-triangle entries of a 32 x 32 matrix per lane: ceil(528 / 32)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ int tri(int n) { return n * (n + 1) / 2; }

// a[side] without dynamic indexing of a kernel-parameter array (which would
// copy the parameter struct to local memory)
template <class T>
__device__ __forceinline__ T pick(T const (&a)[2], int side) {
  return side ? a[1] : a[0];
}

// Entry e of the lower triangle enumerated row by row: (0,0), (1,0), (1,1),
// (2,0), ...; the first tri(n) entries are the lower triangle of every n x n
// leading block.
__device__ __forceinline__ void tri_index(int e, int& i, int& j) {
  int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  if (tri(r + 1) <= e) ++r;
  if (tri(r) > e) --r;
  i = r;
  j = e - tri(r);
}

// 1/d for a normal d > 0: the hardware estimate rcp.approx.ftz.f64 refined
// by one cubic Newton-Raphson step y <- y (1 + e + e^2), e = 1 - d y (exact
// in one fused multiply-add).  The estimate's relative error is below 2^-19
// (measured over the exponent range through the quadratic step, whose error
// e^2 reached 9.4e-13), so the cubic step's truncation error e^3 is below
// 2^-57 and the result lies within one ulp of the correctly rounded 1/d
// (checked against CUDA's IEEE quotient by a GPU test).
__device__ __forceinline__ double recip(double d) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  const double e = fma(-d, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// rows x cols block (rows <= 32, lane = row) of a column-major global matrix
// (ld gld) into a tile (ld ld); eight columns' loads are issued before their
// stores, so that a column does not wait for the previous one.
__device__ __forceinline__ void load_tile(double* T, int ld, const double* g, int gld, int rows, int cols,
                                          int lane) {
  const bool act = lane < rows;
  for (int c0 = 0; c0 < cols; c0 += 8) {
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = (act && c0 + j < cols) ? g[lane + (size_t)(c0 + j) * gld] : 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (act && c0 + j < cols) T[lane + (c0 + j) * ld] = v[j];
  }
}

// In-place LDL^* of A - shift I (lower triangle of the n x n tile A, ld ld):
// on return the unit lower factor is below the diagonal and D on it.  lv
// holds 32 doubles of shared scratch.  Returns whether every pivot was
// positive (the same on every lane); the pivots are tested at the end, a
// failed factorisation only produces values nobody reads.
__device__ __forceinline__ bool ldl(double* A, int ld, int n, double shift, double* lv, int lane) {
  if (lane < n) A[lane * (ld + 1)] -= shift;
  __syncwarp();
  for (int j = 0; j < n; ++j) {
    const double d = A[j + j * ld];
    const double r = recip(d);
    const int m = n - j - 1;
    if (lane < m) lv[lane] = A[j + 1 + lane + j * ld] * r;
    __syncwarp();
    // trailing update A[p][q] -= a_pj l_qj for p >= q > j
    const int nt = tri(m);
    for (int e = lane; e < nt; e += 32) {
      int a, b;
      tri_index(e, a, b);
      const int p = j + 1 + a, q = j + 1 + b;
      A[p + q * ld] = fma(-A[p + j * ld], lv[b], A[p + q * ld]);
    }
    __syncwarp();
    if (lane < m) A[j + 1 + lane + j * ld] = lv[lane];
    __syncwarp();
  }
  const bool ok = lane >= n || A[lane * (ld + 1)] > 1e-300;
  return __all_sync(kFull, ok);
}

// Float32 LDL^* of the n x n lower triangle of F (ld ld), pivots tested at
// the end (positive and finite): the fast first try of the certificate.
__device__ __forceinline__ bool ldl_f32(float* F, int ld, int n, float* lv, int lane) {
  for (int j = 0; j < n; ++j) {
    const float d = F[j + j * ld];
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    const int m = n - j - 1;
    if (lane < m) lv[lane] = F[j + 1 + lane + j * ld] * r;
    __syncwarp();
    const int nt = tri(m);
    for (int e = lane; e < nt; e += 32) {
      int a, b;
      tri_index(e, a, b);
      const int p = j + 1 + a, q = j + 1 + b;
      F[p + q * ld] = fmaf(-F[p + j * ld], lv[b], F[p + q * ld]);
    }
    __syncwarp();
    if (lane < m) F[j + 1 + lane + j * ld] = lv[lane];
    __syncwarp();
  }
  const float d = lane < n ? F[lane * (ld + 1)] : 1.0f;
  const bool ok = d > 1e-30f && d < 1e30f;
  return __all_sync(kFull, ok);
}

// x 2^-ex as a float32, truncated toward zero (relative error below 2^-23)
// and flushed to zero below the normal range, by integer operations on the
// bits of x; |x| < 2^ex.  Leaves the float64 pipe free.
__device__ __forceinline__ float scaled_f32(double x, int ex) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int be = (int)((hi >> 20) & 0x7ffu);
  const int fe = be - 1023 - ex + 127;
  const unsigned f = (hi & 0x80000000u) | ((unsigned)fe << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  return (be != 0 && fe > 0) ? __uint_as_float(f) : 0.0f;
}

// Positive definiteness of A - shift I for the n x n lower triangle of the
// float64 tile A (ld ld), A = L^* W L symmetric positive semidefinite (so
// |a_ij| <= tr A, ||A||_F <= tr A).  First a float32 LDL^* of
// A 2^-e - (shift + c) 2^-e I (2^e ~ tr A, the shift rounded up) in the
// scratch tile Fs, with c = 4 (n + 2) 2^-24 tr A: by the verification of
// positive definiteness through a floating-point Cholesky factorisation of a
// shifted matrix (Rump, BIT 2006), success proves A - shift I positive
// definite, c covering the truncation to float32 (2^-23 ||A||_F), the
// rounding of the diagonal shift (2^-24 tr A) and the factorisation's
// backward error (gamma_{n+1} tr A, the approximate reciprocals included)
// with a margin of n 2^-24 tr A.  When
// the float32 factorisation fails, the float64 LDL^* of A - shift I decides
// (its rounding is inside delta).  A is not modified by the first try.
// Returns 1 (float32 proof), 2 (float64 proof) or 0 (not positive definite).
__device__ __forceinline__ int certify_pd(double* A, int ld, int n, double shift, float* Fs, double* lv,
                                          int lane) {
  const double trA = warp_sum(lane < n ? A[lane * (ld + 1)] : 0.0);
  if (trA > 0.0 && trA < DBL_MAX) {
    int ex = 0;
    frexp(trA, &ex);
    // shift of the float32 matrix, rounded up
    const float cf = __double2float_ru(ldexp(shift + 4.0 * (n + 2) * 0x1p-24 * trA, -ex));
    for (int e = lane; e < tri(n); e += 32) {
      int i, j;
      tri_index(e, i, j);
      const float v = scaled_f32(A[i + j * ld], ex);
      Fs[i + j * ld] = i == j ? v - cf : v;
    }
    __syncwarp();
    if (ldl_f32(Fs, ld, n, reinterpret_cast<float*>(lv), lane)) return 1;
  }
  return ldl(A, ld, n, shift, lv, lane) ? 2 : 0;
}

// The factor L D^{1/2} of a successful ldl in place (lower triangle).
__device__ __forceinline__ void ldl_to_cholesky(double* A, int ld, int n, double* dsq, int lane) {
  if (lane < n) dsq[lane] = sqrt(A[lane * (ld + 1)]);
  __syncwarp();
  for (int e = lane; e < tri(n); e += 32) {
    int i, j;
    tri_index(e, i, j);
    A[i + j * ld] = i == j ? dsq[j] : A[i + j * ld] * dsq[j];
  }
  __syncwarp();
}

// Rows of the outside-block stack of one block: X[r][q] = S_b[q][r] on the
// row side (rows of S_b^*), S_b[r][q] on the column side; l x k.
__device__ __forceinline__ void load_block_rows(double* X, const double* S, int kcap, int side, int l, int k,
                                                int lane, int ld = kLd) {
  if (side == 0) {
    // X = S_b^*: lane q reads row q of S_b, column by column (8 at a time)
    for (int r0 = 0; r0 < l; r0 += 8) {
      double v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = (lane < k && r0 + j < l) ? S[lane + (size_t)(r0 + j) * kcap] : 0.0;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (lane < k && r0 + j < l) X[(r0 + j) + lane * ld] = v[j];
    }
  } else {
    load_tile(X, ld, S, kcap, l, k, lane);
  }
}

// acc (lower triangle of the k x k block in the per-lane layout) += w X^* X
// for the l x k tile X.
template <int NS>
__device__ __forceinline__ void acc_gram(double (&acc)[NS], const double* X, int l, int k, double w, int lane,
                                         int ld = kLd) {
  const int nt = tri(k);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (32 * s >= nt) break;
    const int e = lane + 32 * s;
    if (e < nt) {
      int i, j;
      tri_index(e, i, j);
      double g = 0.0;
      for (int r = 0; r < l; ++r) g = fma(X[r + i * ld], X[r + j * ld], g);
      acc[s] = fma(w, g, acc[s]);
    }
  }
}

__device__ __forceinline__ double sum_squares(const double* X, int l, int k, int lane, int ld = kLd) {
  double part = 0.0;
  for (int e = lane; e < l * k; e += 32) {
    const double v = X[e % l + (e / l) * ld];
    part = fma(v, v, part);
  }
  return warp_sum(part);
}

// Store the lower-triangle accumulator as a full symmetric n x n matrix
// (global slot, ld 32).
template <int NS>
__device__ __forceinline__ void store_sym(double* G, const double (&acc)[NS], int n, int lane) {
  const int nt = tri(n);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (32 * s >= nt) break;
    const int e = lane + 32 * s;
    if (e < nt) {
      int i, j;
      tri_index(e, i, j);
      G[i + j * 32] = acc[s];
      G[j + i * 32] = acc[s];
    }
  }
}

// Visit the entries of [begin, end) whose block lies inside the update
// (other >= 0) or outside it: fetched 32 at a time, one per lane, so that
// walking a long block row costs one load latency per 32 entries, then
// broadcast one by one; fn(en) runs on the whole warp.
template <class Fn>
__device__ __forceinline__ void for_entries(const Entry* __restrict__ ents, int begin, int end, bool inside,
                                            int lane, Fn&& fn) {
  for (int e0 = begin; e0 < end; e0 += 32) {
    const bool have = e0 + lane < end;
    Entry mine{0, -1, 0, -1};
    if (have) mine = ents[e0 + lane];
    unsigned m = __ballot_sync(kFull, have && ((mine.other >= 0) == inside));
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      Entry en;
      en.slot = __shfl_sync(kFull, mine.slot, src);
      en.other = __shfl_sync(kFull, mine.other, src);
      en.other_cluster = __shfl_sync(kFull, mine.other_cluster, src);
      en.norm = __shfl_sync(kFull, mine.norm, src);
      fn(en);
    }
  }
}

// G_t (K x K) of a cluster task into a tile: the V_t^* V_t block from the
// unchanged basis (the identity when V_t is orthonormal), C_t and N_t from
// the task's slot.
__device__ __forceinline__ void load_gram(double* T, int ld, const double* Gv, const double* Vg, bool orth, int k,
                                          int K, int lane) {
  const int r = lane;
  for (int c0 = 0; c0 < K; c0 += 8) {
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = c0 + j;
      double x = 0.0;
      if (r < K && c < K) {
        if (r < k && c < k)
          x = orth ? (r == c ? 1.0 : 0.0) : Vg[r + c * 32];
        else
          x = Gv[r + c * 32];
      }
      v[j] = x;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (r < K && c0 + j < K) T[r + (c0 + j) * ld] = v[j];
  }
}

// ------------------------------------------------- the unchanged matrix
// Orthonormal cluster bases.  A nested basis V_t is orthonormal when every
// cluster below it is locally orthonormal: V_t^* V_t = I for a leaf,
// sum over the sons of E_s^* E_s = I for an inner cluster (given orthonormal
// sons).  k_orth_local tests every cluster of both sides in one launch and
// writes the local verdict into orth; k_orth_mark then clears orth on every
// ancestor of a cluster that failed, so that orth_c = 1 exactly when the
// whole subtree of c passed (a sufficient condition; local deviations of
// kOrthLocalTol add up over at most the tree depth).  k_vgram computes
// V_t^* V_t level by level for the clusters left with orth_c = 0 only (the
// others have V_t^* V_t = I and nobody reads their slot).
constexpr double kOrthLocalTol = 2e-14;

__global__ void k_orth_local(MatView M, const int32_t* __restrict__ list, int n, BaseWeights BW) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int idx = blockIdx.x * (blockDim.x >> 5) + w;
  if (idx >= n) return;
  const int kcap = M.kcap;
  double* T0 = smem + (size_t)w * kLd * kcap;
  const int side = list[idx] >> 30;
  const int c = list[idx] & 0x3fffffff;
  const int32_t* rank = pick(M.rank, side);
  const int32_t* subtree = pick(M.subtree, side);
  const int k = rank[c];
  bool ok = k <= 32;
  if (ok) {
    const int nt = tri(k);
    double acc[kNS];
#pragma unroll
    for (int s = 0; s < kNS; ++s) acc[s] = 0.0;
    if (subtree[c] == 1) {
      const double* V = pick(M.leaf, side) + pick(M.leaf_off, side)[c];
      const int m = pick(M.size, side)[c];
      for (int r0 = 0; r0 < m; r0 += 32) {
        const int ch = min(32, m - r0);
        load_tile(T0, kLd, V + r0, m, ch, k, lane);
        __syncwarp();
        acc_gram(acc, T0, ch, k, 1.0, lane);
        __syncwarp();
      }
    } else {
      for (int si = 0; si < 2; ++si) {
        const int s = si == 0 ? c + 1 : c + 1 + subtree[c + 1];
        load_tile(T0, kLd, pick(M.transfer, side) + (size_t)s * kcap * kcap, kcap, rank[s], k, lane);
        __syncwarp();
        acc_gram(acc, T0, rank[s], k, 1.0, lane);
        __syncwarp();
      }
    }
#pragma unroll
    for (int s = 0; s < kNS; ++s) {
      const int e = lane + 32 * s;
      if (e < nt) {
        int i, j;
        tri_index(e, i, j);
        if (!(fabs(acc[s] - (i == j ? 1.0 : 0.0)) <= kOrthLocalTol)) ok = false;
      }
    }
  }
  ok = __all_sync(kFull, ok);
  if (lane == 0) pick(BW.orth, side)[c] = ok ? 1 : 0;
}

// One thread per cluster of both sides: a cluster that failed clears orth on
// its ancestors (stores of 0 only, so concurrent walks agree).
__global__ void k_orth_mark(MatView M, const int32_t* __restrict__ list, int n, BaseWeights BW) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int side = list[idx] >> 30;
  const int c = list[idx] & 0x3fffffff;
  int32_t* orth = pick(BW.orth, side);
  if (orth[c]) return;
  const int32_t* father = pick(M.father, side);
  for (int f = father[c]; f >= 0; f = father[f]) orth[f] = 0;
}

// Vg_c = V_c^* V_c, bottom-up (one launch per level), for clusters with
// orth_c = 0: leaf Gram of V_c, inner sum over the sons of E_s^* Vg_s E_s
// (Vg_s = I for an orthonormal son).
__global__ void k_vgram(MatView M, const int32_t* __restrict__ list, int n, BaseWeights BW) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int idx = blockIdx.x * (blockDim.x >> 5) + w;
  if (idx >= n) return;
  const int side = list[idx] >> 30;
  const int c = list[idx] & 0x3fffffff;
  const int32_t* orth = pick(BW.orth, side);
  if (orth[c]) return;
  const int kcap = M.kcap;
  double* T0 = smem + (size_t)w * 3 * kLd * kcap;
  double* T1 = T0 + kLd * kcap;
  double* T2 = T1 + kLd * kcap;
  const int32_t* rank = pick(M.rank, side);
  const int32_t* subtree = pick(M.subtree, side);
  const int k = rank[c];
  if (k > 32) return;
  const int nt = tri(k);
  double acc[kNS];
#pragma unroll
  for (int s = 0; s < kNS; ++s) acc[s] = 0.0;
  if (subtree[c] == 1) {
    const double* V = pick(M.leaf, side) + pick(M.leaf_off, side)[c];
    const int m = pick(M.size, side)[c];
    for (int r0 = 0; r0 < m; r0 += 32) {
      const int ch = min(32, m - r0);
      load_tile(T0, kLd, V + r0, m, ch, k, lane);
      __syncwarp();
      acc_gram(acc, T0, ch, k, 1.0, lane);
      __syncwarp();
    }
  } else {
    for (int si = 0; si < 2; ++si) {
      const int s = si == 0 ? c + 1 : c + 1 + subtree[c + 1];
      const int ks = rank[s];
      load_tile(T1, kLd, pick(M.transfer, side) + (size_t)s * kcap * kcap, kcap, ks, k, lane);
      __syncwarp();
      if (orth[s]) {
        acc_gram(acc, T1, ks, k, 1.0, lane);
        __syncwarp();
        continue;
      }
      load_tile(T0, kLd, pick(BW.Vg, side) + (size_t)s * kSlot, 32, ks, ks, lane);
      __syncwarp();
      // T2 = Vg_s E_s (ks x k)
      for (int e = lane; e < ks * k; e += 32) {
        const int i = e % ks, j = e / ks;
        double v = 0.0;
        for (int q = 0; q < ks; ++q) v = fma(T0[i + q * kLd], T1[q + j * kLd], v);
        T2[i + j * kLd] = v;
      }
      __syncwarp();
#pragma unroll
      for (int s2 = 0; s2 < kNS; ++s2) {
        if (32 * s2 >= nt) break;
        const int e = lane + 32 * s2;
        if (e < nt) {
          int i, j;
          tri_index(e, i, j);
          double v = acc[s2];
          for (int q = 0; q < ks; ++q) v = fma(T1[q + i * kLd], T2[q + j * kLd], v);
          acc[s2] = v;
        }
      }
      __syncwarp();
    }
  }
  store_sym(pick(BW.Vg, side) + (size_t)c * kSlot, acc, k, lane);
}

// Wo_c = sum over b in row(c) of omega_b^2 S_b S_b^* (column side S_b^* S_b),
// omega_b = sqrt(#T_c) / ||S_b||_F, for every cluster of both sides; the
// Gram of the stack whose R-factor the exact path folds.
template <int NS>
__global__ void k_bgram(MatView M, const int32_t* __restrict__ list, int n, BlockLists BL, BaseWeights BW,
                        int* err) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int idx = blockIdx.x * (blockDim.x >> 5) + w;
  if (idx >= n) return;
  const int kcap = M.kcap;
  double* X = smem + (size_t)w * kLd * kcap;
  const int side = list[idx] >> 30;
  const int c = list[idx] & 0x3fffffff;
  const int k = pick(M.rank, side)[c];
  if (k > 32) {
    if (lane == 0) atomicOr(err, kErrCols);
    return;
  }
  const double st = (double)pick(M.subtree, side)[c];
  const int32_t* orank = pick(M.rank, 1 - side);
  const int32_t* other = pick(BL.other, side);
  const int32_t* adm = pick(BL.adm, side);
  double acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.0;
  for (int e = pick(BL.ptr, side)[c]; e < pick(BL.ptr, side)[c + 1]; ++e) {
    const int slot = adm[e];
    const int l = orank[other[slot]];
    load_block_rows(X, M.S + (size_t)slot * kcap * kcap, kcap, side, l, k, lane);
    __syncwarp();
    const double nrm2 = sum_squares(X, l, k, lane);
    const double w2 = nrm2 > 1e-300 ? st * recip(nrm2) : 0.0;
    acc_gram(acc, X, l, k, w2, lane);
    __syncwarp();
  }
  store_sym(pick(BW.Wo, side) + (size_t)c * kSlot, acc, k, lane);
}

// W0_c = Wo_c + E_c W0_{c+} E_c^* top-down (one launch per level), one
// block of kDownWarps warps per cluster: the few clusters of the upper levels
// would otherwise wait on one warp's chain of float64 instructions.
constexpr int kDownWarps = 4;

__global__ void k_bgram_down(MatView M, const int32_t* __restrict__ list, int n, BaseWeights BW) {
  __shared__ double T0[kLd * 32];   // W0_{c+} (kf x kf)
  __shared__ double T1[kLd * 32];   // E_c (k x kf)
  __shared__ double T2[kLd * 32];   // E_c W0_{c+} (k x kf)
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int w = tid >> 5;
  constexpr int nthr = 32 * kDownWarps;
  if ((int)blockIdx.x >= n) return;
  const int kcap = M.kcap;
  const int side = list[blockIdx.x] >> 30;
  const int c = list[blockIdx.x] & 0x3fffffff;
  const int k = pick(M.rank, side)[c];
  if (k > 32 || kcap > 32) return;
  const double* Wo = pick(BW.Wo, side) + (size_t)c * kSlot;
  double* W0 = pick(BW.W0, side) + (size_t)c * kSlot;
  const int f = pick(M.father, side)[c];
  const int nt = tri(k);
  if (f < 0) {
    for (int e = tid; e < nt; e += nthr) {
      int i, j;
      tri_index(e, i, j);
      W0[i + j * 32] = W0[j + i * 32] = Wo[i + j * 32];
    }
    return;
  }
  const int kf = pick(M.rank, side)[f];
  if (w == 0) load_tile(T0, kLd, pick(BW.W0, side) + (size_t)f * kSlot, 32, kf, kf, lane);
  if (w == 1) load_tile(T1, kLd, pick(M.transfer, side) + (size_t)c * kcap * kcap, kcap, k, kf, lane);
  __syncthreads();
  for (int e = tid; e < k * kf; e += nthr) {
    const int i = e % k, j = e / k;
    double v = 0.0;
    for (int q = 0; q < kf; ++q) v = fma(T1[i + q * kLd], T0[q + j * kLd], v);
    T2[i + j * kLd] = v;
  }
  __syncthreads();
  for (int e = tid; e < nt; e += nthr) {
    int i, j;
    tri_index(e, i, j);
    double v = Wo[i + j * 32];
    for (int q = 0; q < kf; ++q) v = fma(T2[i + q * kLd], T1[j + q * kLd], v);
    W0[i + j * 32] = W0[j + i * 32] = v;
  }
}

// ------------------------------------------------------------- step 2
// C_t = V_t^* A|_t and N_t = A|_t^* A|_t bottom-up: leaves over chunks of 32
// rows of (V_t, A|_t) (k_fgram, one warp per leaf), inner clusters
// C_t = sum E_s^* C_s, N_t = sum N_s (k_fgram_inner, one block of
// kInnerWarps warps per cluster: the upper levels have few clusters).
// Entry e of the per-lane list is C_t[e % k][e / k] for e < k u, then the
// lower triangle of N_t.  The V_t^* V_t block of G_t comes from k_vgram.
template <int NS>
__global__ void __launch_bounds__(128, 6) k_fgram(MatView M, const Item* __restrict__ items, const int32_t* __restrict__ list, int n, int u,
                        int tc, const double* __restrict__ A, const double* __restrict__ B, ItemBuffers IB,
                        int* err) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int idx = blockIdx.x * (blockDim.x >> 5) + w;
  if (idx >= n) return;
  double* T0 = smem + (size_t)w * kLd * tc;
  const int id = list[idx];
  const Item it = items[id];
  const int side = it.side;
  const int k = it.k;
  const int K = k + u;
  if (K > tc) {
    if (lane == 0) atomicOr(err, kErrCols);
    return;
  }
  const int ncu = k * u;
  const int nt = ncu + tri(u);
  double acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.0;
  {
    const double* V = pick(M.leaf, side) + pick(M.leaf_off, side)[it.cluster];
    const double* F = (side == 0 ? A : B) + it.foff;
    const int m = it.size;
    for (int r0 = 0; r0 < m; r0 += 32) {
      const int ch = min(32, m - r0);
      load_tile(T0, kLd, V + r0, m, ch, k, lane);
      load_tile(T0 + k * kLd, kLd, F + it.rowoff + r0, it.ld, ch, u, lane);
      __syncwarp();
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (32 * s >= nt) break;
        const int e = lane + 32 * s;
        if (e < nt) {
          int c1, c2;
          if (e < ncu) {
            c1 = e % k;
            c2 = k + e / k;
          } else {
            tri_index(e - ncu, c1, c2);
            c1 += k;
            c2 += k;
          }
          double g = acc[s];
          for (int r = 0; r < ch; ++r) g = fma(T0[r + c1 * kLd], T0[r + c2 * kLd], g);
          acc[s] = g;
        }
      }
      __syncwarp();
    }
  }
  double* G = IB.Gv + (size_t)id * kSlot;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (32 * s >= nt) break;
    const int e = lane + 32 * s;
    if (e < nt) {
      int i, j;
      if (e < ncu) {
        i = e % k;
        j = k + e / k;
      } else {
        tri_index(e - ncu, i, j);
        i += k;
        j += k;
      }
      G[i + j * 32] = acc[s];
      G[j + i * 32] = acc[s];
    }
  }
}

constexpr int kInnerWarps = 4;

__global__ void k_fgram_inner(MatView M, const Item* __restrict__ items, const int32_t* __restrict__ list, int n,
                              int u, ItemBuffers IB, int* err) {
  __shared__ double Cs[2][kLd * 32];   // C_s (k_s x u) of the two sons
  __shared__ double Es[2][kLd * 32];   // E_s (k_s x k)
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int w = tid >> 5;
  if ((int)blockIdx.x >= n) return;
  const int id = list[blockIdx.x];
  const Item it = items[id];
  const int side = it.side;
  const int k = it.k;
  const int kcap = M.kcap;
  if (k + u > 32 || kcap > 32) {
    if (tid == 0) atomicOr(err, kErrCols);
    return;
  }
  const int sid[2] = {it.son0, it.son1};
  const int ks0 = items[it.son0].k, ks1 = items[it.son1].k;
  {
    const int si = w & 1;
    const Item sn = items[si ? sid[1] : sid[0]];
    if (w < 2)
      load_tile(Cs[si], kLd, IB.Gv + (size_t)(si ? sid[1] : sid[0]) * kSlot + sn.k * 32, 32, sn.k, u, lane);
    else
      load_tile(Es[si], kLd, pick(M.transfer, side) + (size_t)sn.cluster * kcap * kcap, kcap, sn.k, k, lane);
  }
  __syncthreads();
  const int ncu = k * u;
  const int nt = ncu + tri(u);
  const double* G0 = IB.Gv + (size_t)it.son0 * kSlot;
  const double* G1 = IB.Gv + (size_t)it.son1 * kSlot;
  double* G = IB.Gv + (size_t)id * kSlot;
  for (int e = tid; e < nt; e += 32 * kInnerWarps) {
    int i, j;
    double v = 0.0;
    if (e < ncu) {
      i = e % k;
      j = e / k;
      for (int q = 0; q < ks0; ++q) v = fma(Es[0][q + i * kLd], Cs[0][q + j * kLd], v);
      for (int q = 0; q < ks1; ++q) v = fma(Es[1][q + i * kLd], Cs[1][q + j * kLd], v);
      j += k;
    } else {
      int a, b;
      tri_index(e - ncu, a, b);
      v += G0[(ks0 + a) + (ks0 + b) * 32];
      v += G1[(ks1 + a) + (ks1 + b) * 32];
      i = k + a;
      j = k + b;
    }
    G[i + j * 32] = v;
    G[j + i * 32] = v;
  }
}

// ||Z~|_b||_F^2 = tr(S~_b^* G_t S~_b G_s) for the blocks inside the update,
// S~_b = diag(S_b, I_u): entry (i, j) of G_t S~_b times entry (i, j) of
// S~_b G_s, summed.
__global__ void k_fnorms(MatView M, const Item* __restrict__ items, const NormTask* __restrict__ tasks, int n,
                         int u, int tc, BaseWeights BW, ItemBuffers IB) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int idx = blockIdx.x * (blockDim.x >> 5) + w;
  if (idx >= n) return;
  double* T0 = smem + (size_t)w * 3 * kLd * tc;
  double* T1 = T0 + kLd * tc;
  double* T2 = T1 + kLd * tc;
  const NormTask tk = tasks[idx];
  const Item it = items[tk.it], is = items[tk.is];
  const int kt = it.k, ls = is.k;
  const int Kt = kt + u, Ks = ls + u;
  const int kcap = M.kcap;
  const double* Gt = IB.Gv + (size_t)tk.it * kSlot;
  const double* Gs = IB.Gv + (size_t)tk.is * kSlot;
  if (BW.orth[0][it.cluster] && BW.orth[1][is.cluster]) {
    // ||S||^2 + 2 <C_t, S C_s> + <N_t, N_s> (orthonormal V_t, W_s)
    load_tile(T2, kLd, M.S + (size_t)tk.slot * kcap * kcap, kcap, kt, ls, lane);
    load_tile(T1, kLd, Gs + ls * 32, 32, ls, u, lane);   // C_s (ls x u)
    __syncwarp();
    double part = 0.0;
    for (int e = lane; e < kt * ls; e += 32) {
      const double v = T2[e % kt + (e / kt) * kLd];
      part = fma(v, v, part);
    }
    for (int e = lane; e < kt * u; e += 32) {
      const int i = e % kt, j = e / kt;
      double v = 0.0;
      for (int q = 0; q < ls; ++q) v = fma(T2[i + q * kLd], T1[q + j * kLd], v);
      part = fma(2.0 * Gt[i + (kt + j) * 32], v, part);
    }
    for (int e = lane; e < u * u; e += 32) {
      const int a = e % u, b = e / u;
      part = fma(Gt[(kt + a) + (kt + b) * 32], Gs[(ls + a) + (ls + b) * 32], part);
    }
    const double s2 = warp_sum(part);
    if (lane == 0) IB.norms[idx] = sqrt(fmax(s2, 0.0));
    return;
  }
  load_gram(T0, kLd, IB.Gv + (size_t)tk.it * kSlot, BW.Vg[0] + (size_t)it.cluster * kSlot,
            BW.orth[0][it.cluster] != 0, kt, Kt, lane);
  load_gram(T1, kLd, IB.Gv + (size_t)tk.is * kSlot, BW.Vg[1] + (size_t)is.cluster * kSlot,
            BW.orth[1][is.cluster] != 0, ls, Ks, lane);
  load_tile(T2, kLd, M.S + (size_t)tk.slot * kcap * kcap, kcap, kt, ls, lane);
  __syncwarp();
  double part = 0.0;
  for (int e = lane; e < Kt * Ks; e += 32) {
    const int i = e % Kt, j = e / Kt;
    double x, y;
    if (j < ls) {
      x = 0.0;
      for (int q = 0; q < kt; ++q) x = fma(T0[i + q * kLd], T2[q + j * kLd], x);
    } else {
      x = T0[i + (kt + j - ls) * kLd];
    }
    if (i < kt) {
      y = 0.0;
      for (int q = 0; q < ls; ++q) y = fma(T2[i + q * kLd], T1[q + j * kLd], y);
    } else {
      y = T1[ls + i - kt + j * kLd];
    }
    part = fma(x, y, part);
  }
  const double s = warp_sum(part);
  if (lane == 0) IB.norms[idx] = sqrt(fmax(s, 0.0));
}

// ------------------------------------------------------------- step 3
// W_t top-down: the outside blocks of row(t) (Wo_t of the unchanged matrix
// when V_t is orthonormal, minus the base terms of the blocks inside the
// update; otherwise summed with ||Z~|_b||_F = ||R_kk S_b||_F), plus
// omega_b^2 P G_o P^* for every block inside the update (P = diag(S_b, I_u)
// on the row side, diag(S_b^*, I_u) on the column side), plus the father's
// part E~_t W_{t+} E~_t^* (subtree root: E_t W0_{t+} E_t^* of the unchanged
// matrix).
// Shared doubles of the three k_fweights tiles of one warp.
__host__ __device__ constexpr int fweights_doubles(int tc, int kcap) { return (kcap + 1) * kcap + 2 * (tc + 1) * tc; }

// One warp: cluster task id with its three tiles: T0 (blocks of couplings
// and E_t, at most kcap x kcap, leading dimension ld0) and T1, T2 (leading
// dimension ld).
template <int NS>
__device__ __forceinline__ void fweights_warp(const MatView& M, const Item* __restrict__ items,
                                              const Entry* __restrict__ ents, int id, int u, int ld, int ld0,
                                              const BaseWeights& BW, const ItemBuffers& IB, double* T0, double* T1,
                                              double* T2, int lane) {
  const Item it = items[id];
  const int side = it.side;
  const int k = it.k;
  const int K = k + u;
  const int kcap = M.kcap;
  const int nt = tri(K);
  const int ntk = tri(k);
  const double st = (double)pick(M.subtree, side)[it.cluster];
  const int32_t* orank = pick(M.rank, 1 - side);
  const double* Sbase = M.S;
  const bool orth = pick(BW.orth, side)[it.cluster] != 0;
  double acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.0;
  if (orth) {
    const double* Wo = pick(BW.Wo, side) + (size_t)it.cluster * kSlot;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int e = lane + 32 * s;
      if (e < ntk) {
        int i, j;
        tri_index(e, i, j);
        acc[s] = Wo[i + j * 32];
      }
    }
  } else {
    load_tile(T1, ld, pick(BW.Vg, side) + (size_t)it.cluster * kSlot, 32, k, k, lane);
    for_entries(ents, it.ent_begin, it.ent_end, false, lane, [&](const Entry& en) {
      const int l = orank[en.other_cluster];
      load_block_rows(T0, Sbase + (size_t)en.slot * kcap * kcap, kcap, side, l, k, lane, ld0);
      __syncwarp();
      // ||R_kk S_b||_F^2 = sum over rows x of X of x G_kk x^*
      double part = 0.0;
      for (int e2 = lane; e2 < l * k; e2 += 32) {
        const int r = e2 % l, q = e2 / l;
        double y = 0.0;
        for (int p = 0; p < k; ++p) y = fma(T0[r + p * ld0], T1[p + q * ld], y);
        part = fma(y, T0[r + q * ld0], part);
      }
      const double nrm2 = warp_sum(part);
      const double w2 = nrm2 > 1e-300 ? st * recip(nrm2) : 0.0;
      acc_gram(acc, T0, l, k, w2, lane, ld0);
      __syncwarp();
    });
  }
  if (lane == 0) IB.jac[4 * (size_t)id + 3] = orth ? 0ull : 1ull;
  // blocks inside the update: omega_b^2 P G_o P^*, and, when the outside
  // part came from Wo_t, minus the block's term in Wo_t (omega0_b^2 S' S'^*,
  // omega0_b = sqrt(#T_t) / ||S_b||_F).  X = S'^* (l x k) in T0.  For an
  // orthonormal W_o, G_o = [[I, C_o], [C_o^*, N_o]] and
  // P G_o P^* = [[S' S'^*, S' C_o], [C_o^* S'^*, N_o]].
  if (it.flags & kItemInside) {
    const double* Vgo = pick(BW.Vg, 1 - side);
    const int32_t* orth_o = pick(BW.orth, 1 - side);
    for_entries(ents, it.ent_begin, it.ent_end, true, lane, [&](const Entry& en) {
      const Item ot = items[en.other];
      const int l = ot.k;
      const int Ko = l + u;
      const double nrm = IB.norms[en.norm];
      const double w2 = nrm > 1e-150 ? st * recip(nrm * nrm) : 0.0;
      const double* Go = IB.Gv + (size_t)en.other * kSlot;
      load_block_rows(T0, Sbase + (size_t)en.slot * kcap * kcap, kcap, side, l, k, lane, ld0);
      __syncwarp();
      double w02 = 0.0;
      if (orth) {
        const double nrm2 = sum_squares(T0, l, k, lane, ld0);
        w02 = nrm2 > 1e-300 ? st * recip(nrm2) : 0.0;
      }
      if (orth_o[ot.cluster]) {
        load_tile(T1, ld, Go + l * 32, 32, l, u, lane);   // C_o (l x u)
        __syncwarp();
        acc_gram(acc, T0, l, k, w2 - w02, lane, ld0);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          if (32 * s >= nt) break;
          const int e2 = lane + 32 * s;
          if (e2 >= ntk && e2 < nt) {
            int i, j;
            tri_index(e2, i, j);
            double v;
            if (j < k) {
              v = 0.0;
              for (int q = 0; q < l; ++q) v = fma(T1[q + (i - k) * ld], T0[q + j * ld0], v);
            } else {
              v = Go[(l + i - k) + (l + j - k) * 32];
            }
            acc[s] = fma(w2, v, acc[s]);
          }
        }
        __syncwarp();
        return;
      }
      if (orth) acc_gram(acc, T0, l, k, -w02, lane, ld0);
      load_gram(T1, ld, Go, Vgo + (size_t)ot.cluster * kSlot, false, l, Ko, lane);
      __syncwarp();
      // T2 = P G_o (K x Ko), S'[i][q] = X[q][i]
      for (int e2 = lane; e2 < K * Ko; e2 += 32) {
        const int i = e2 % K, j = e2 / K;
        double v;
        if (i < k) {
          v = 0.0;
          for (int q = 0; q < l; ++q) v = fma(T0[q + i * ld0], T1[q + j * ld], v);
        } else {
          v = T1[l + i - k + j * ld];
        }
        T2[i + j * ld] = v;
      }
      __syncwarp();
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (32 * s >= nt) break;
        const int e2 = lane + 32 * s;
        if (e2 < nt) {
          int i, j;
          tri_index(e2, i, j);
          double v;
          if (j < k) {
            v = 0.0;
            for (int q = 0; q < l; ++q) v = fma(T2[i + q * ld], T0[q + j * ld0], v);
          } else {
            v = T2[i + (l + j - k) * ld];
          }
          acc[s] = fma(w2, v, acc[s]);
        }
      }
      __syncwarp();
    });
  }
  // father's part
  const double* E = pick(M.transfer, side) + (size_t)it.cluster * kcap * kcap;   // k x kf
  if (it.flags & kItemRoot) {
    if (!(it.flags & kItemTreeRoot)) {
      const int f = pick(M.father, side)[it.cluster];
      const int kf = it.kf;
      load_tile(T1, ld, pick(BW.W0, side) + (size_t)f * kSlot, 32, kf, kf, lane);
      load_tile(T0, ld0, E, kcap, k, kf, lane);
      __syncwarp();
      for (int e2 = lane; e2 < k * kf; e2 += 32) {
        const int i = e2 % k, j = e2 / k;
        double v = 0.0;
        for (int q = 0; q < kf; ++q) v = fma(T0[i + q * ld0], T1[q + j * ld], v);
        T2[i + j * ld] = v;
      }
      __syncwarp();
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (32 * s >= ntk) break;
        const int e2 = lane + 32 * s;
        if (e2 < ntk) {
          int i, j;
          tri_index(e2, i, j);
          double v = acc[s];
          for (int q = 0; q < kf; ++q) v = fma(T2[i + q * ld], T0[j + q * ld0], v);
          acc[s] = v;
        }
      }
    }
  } else {
    const int kf = items[it.parent].k;
    const int Kf = kf + u;
    load_tile(T1, ld, IB.Wg + (size_t)it.parent * kSlot, 32, Kf, Kf, lane);
    load_tile(T0, ld0, E, kcap, k, kf, lane);
    __syncwarp();
    // T2 = E W11 (k x kf); rows k.. of E~_t W_p are rows kf.. of W_p
    for (int e2 = lane; e2 < k * kf; e2 += 32) {
      const int i = e2 % k, j = e2 / k;
      double v = 0.0;
      for (int q = 0; q < kf; ++q) v = fma(T0[i + q * ld0], T1[q + j * ld], v);
      T2[i + j * ld] = v;
    }
    __syncwarp();
    // lower triangle of E~_t W_p E~_t^*, block by block so that one warp
    // instruction never mixes products with copies: (i, j < k) rows of T2
    // times E^* (the first tri(k) entries); (i >= k, j < k) rows kf + i - k
    // of W_p times E^*; (i, j >= k) W22
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (32 * s >= ntk) break;
      const int e2 = lane + 32 * s;
      if (e2 < ntk) {
        int i, j;
        tri_index(e2, i, j);
        double v = acc[s];
        for (int q = 0; q < kf; ++q) v = fma(T2[i + q * ld], T0[j + q * ld0], v);
        acc[s] = v;
      }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (32 * s >= nt) break;
      const int e2 = lane + 32 * s;
      if (e2 >= ntk && e2 < nt) {
        int i, j;
        tri_index(e2, i, j);
        double v = acc[s];
        if (j < k) {
          for (int q = 0; q < kf; ++q) v = fma(T1[(kf + i - k) + q * ld], T0[j + q * ld0], v);
        } else {
          v += T1[(kf + i - k) + (kf + j - k) * ld];
        }
        acc[s] = v;
      }
    }
  }
  store_sym(IB.Wg + (size_t)id * kSlot, acc, K, lane);
}

template <int NS>
__global__ void k_fweights(MatView M, const Item* __restrict__ items, const Entry* __restrict__ ents,
                           const int32_t* __restrict__ list, int n, int u, int tc, BaseWeights BW, ItemBuffers IB) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int idx = blockIdx.x * (blockDim.x >> 5) + w;
  if (idx >= n) return;
  // T1, T2 hold at most max(K, kcap) = tc rows (leading dimension tc + 1),
  // T0 at most kcap (leading dimension kcap + 1)
  const int ld = tc + 1;
  const int ld0 = M.kcap + 1;
  double* T0 = smem + (size_t)w * fweights_doubles(tc, M.kcap);
  double* T1 = T0 + ld0 * M.kcap;
  fweights_warp<NS>(M, items, ents, list[idx], u, ld, ld0, BW, IB, T0, T1, T1 + ld * tc, lane);
}

// The same with one block of kWideWarps warps per cluster task, for the
// levels with few tasks (where one warp's chain of instructions would set
// the launch's duration): the entries of W_t and of the products are spread
// over the block, each entry of W_t summed by one thread in the order of
// k_fweights, so that both kernels give the same bits.  Tasks whose V_t is
// not orthonormal run the one-warp code on warp 0.
constexpr int kWideWarps = 4;
constexpr int kWideMaxTasks = 1024;   // levels with at most this many tasks take k_fweights_wide
constexpr int kWideThreads = 32 * kWideWarps;
constexpr int kWS = (kNS * 32 + kWideThreads - 1) / kWideThreads;   // entries of W_t per thread

__global__ void k_fweights_wide(MatView M, const Item* __restrict__ items, const Entry* __restrict__ ents,
                                const int32_t* __restrict__ list, int n, int u, int tc, BaseWeights BW,
                                ItemBuffers IB) {
  extern __shared__ double smem[];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int w = tid >> 5;
  if ((int)blockIdx.x >= n) return;
  const int ld = tc + 1;
  const int ld0 = M.kcap + 1;
  double* T0 = smem;
  double* T1 = T0 + ld0 * M.kcap;
  double* T2 = T1 + ld * tc;
  const int id = list[blockIdx.x];
  const Item it = items[id];
  const int side = it.side;
  if (!pick(BW.orth, side)[it.cluster]) {
    if (w == 0) fweights_warp<kNS>(M, items, ents, id, u, ld, ld0, BW, IB, T0, T1, T2, lane);
    return;
  }
  const int k = it.k;
  const int K = k + u;
  const int kcap = M.kcap;
  const int nt = tri(K);
  const int ntk = tri(k);
  const double st = (double)pick(M.subtree, side)[it.cluster];
  double acc[kWS];
  int ei[kWS], ej[kWS];
#pragma unroll
  for (int s = 0; s < kWS; ++s) {
    const int e = tid + kWideThreads * s;
    int i = 0, j = 0;
    if (e < nt) tri_index(e, i, j);
    ei[s] = i;
    ej[s] = j;
    acc[s] = e < ntk ? pick(BW.Wo, side)[(size_t)it.cluster * kSlot + i + j * 32] : 0.0;
  }
  if (tid == 0) IB.jac[4 * (size_t)id + 3] = 0ull;
  if (it.flags & kItemInside) {
    const double* Vgo = pick(BW.Vg, 1 - side);
    const int32_t* orth_o = pick(BW.orth, 1 - side);
    // every warp walks the same entries, so that all reach the same barriers
    for_entries(ents, it.ent_begin, it.ent_end, true, lane, [&](const Entry& en) {
      const Item ot = items[en.other];
      const int l = ot.k;
      const int Ko = l + u;
      const double nrm = IB.norms[en.norm];
      const double w2 = nrm > 1e-150 ? st * recip(nrm * nrm) : 0.0;
      const double* Go = IB.Gv + (size_t)en.other * kSlot;
      const bool oo = orth_o[ot.cluster] != 0;
      if (w == 0) load_block_rows(T0, M.S + (size_t)en.slot * kcap * kcap, kcap, side, l, k, lane, ld0);
      if (w == 1) {
        if (oo)
          load_tile(T1, ld, Go + l * 32, 32, l, u, lane);   // C_o (l x u)
        else
          load_gram(T1, ld, Go, Vgo + (size_t)ot.cluster * kSlot, false, l, Ko, lane);
      }
      __syncthreads();
      const double nrm2 = sum_squares(T0, l, k, lane, ld0);   // the same in every warp
      const double w02 = nrm2 > 1e-300 ? st * recip(nrm2) : 0.0;
      const double wb = oo ? w2 - w02 : -w02;
#pragma unroll
      for (int s = 0; s < kWS; ++s) {
        const int e = tid + kWideThreads * s;
        if (e < ntk) {
          double g = 0.0;
          for (int r = 0; r < l; ++r) g = fma(T0[r + ei[s] * ld0], T0[r + ej[s] * ld0], g);
          acc[s] = fma(wb, g, acc[s]);
        }
      }
      if (oo) {
#pragma unroll
        for (int s = 0; s < kWS; ++s) {
          const int e = tid + kWideThreads * s;
          if (e >= ntk && e < nt) {
            const int i = ei[s], j = ej[s];
            double v;
            if (j < k) {
              v = 0.0;
              for (int q = 0; q < l; ++q) v = fma(T1[q + (i - k) * ld], T0[q + j * ld0], v);
            } else {
              v = Go[(l + i - k) + (l + j - k) * 32];
            }
            acc[s] = fma(w2, v, acc[s]);
          }
        }
        __syncthreads();
        return;
      }
      // T2 = P G_o (K x Ko), S'[i][q] = X[q][i]
      for (int e2 = tid; e2 < K * Ko; e2 += kWideThreads) {
        const int i = e2 % K, j = e2 / K;
        double v;
        if (i < k) {
          v = 0.0;
          for (int q = 0; q < l; ++q) v = fma(T0[q + i * ld0], T1[q + j * ld], v);
        } else {
          v = T1[l + i - k + j * ld];
        }
        T2[i + j * ld] = v;
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < kWS; ++s) {
        const int e = tid + kWideThreads * s;
        if (e < nt) {
          const int i = ei[s], j = ej[s];
          double v;
          if (j < k) {
            v = 0.0;
            for (int q = 0; q < l; ++q) v = fma(T2[i + q * ld], T0[q + j * ld0], v);
          } else {
            v = T2[i + (l + j - k) * ld];
          }
          acc[s] = fma(w2, v, acc[s]);
        }
      }
      __syncthreads();
    });
  }
  // father's part
  const double* E = pick(M.transfer, side) + (size_t)it.cluster * kcap * kcap;   // k x kf
  const bool root = it.flags & kItemRoot;
  if (!root || !(it.flags & kItemTreeRoot)) {
    const int kf = root ? it.kf : items[it.parent].k;
    const int Kf = root ? kf : kf + u;
    if (w == 0) {
      if (root)
        load_tile(T1, ld, pick(BW.W0, side) + (size_t)pick(M.father, side)[it.cluster] * kSlot, 32, kf, kf, lane);
      else
        load_tile(T1, ld, IB.Wg + (size_t)it.parent * kSlot, 32, Kf, Kf, lane);
    }
    if (w == 1) load_tile(T0, ld0, E, kcap, k, kf, lane);
    __syncthreads();
    // T2 = E W11 (k x kf)
    for (int e2 = tid; e2 < k * kf; e2 += kWideThreads) {
      const int i = e2 % k, j = e2 / k;
      double v = 0.0;
      for (int q = 0; q < kf; ++q) v = fma(T0[i + q * ld0], T1[q + j * ld], v);
      T2[i + j * ld] = v;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kWS; ++s) {
      const int e = tid + kWideThreads * s;
      if (e < ntk) {
        double v = acc[s];
        for (int q = 0; q < kf; ++q) v = fma(T2[ei[s] + q * ld], T0[ej[s] + q * ld0], v);
        acc[s] = v;
      }
    }
    if (!root) {
      // (i >= k, j < k): rows kf + i - k of W_p times E^*; (i, j >= k): W22
#pragma unroll
      for (int s = 0; s < kWS; ++s) {
        const int e = tid + kWideThreads * s;
        if (e >= ntk && e < nt) {
          const int i = ei[s], j = ej[s];
          double v = acc[s];
          if (j < k) {
            for (int q = 0; q < kf; ++q) v = fma(T1[(kf + i - k) + q * ld], T0[j + q * ld0], v);
          } else {
            v += T1[(kf + i - k) + (kf + j - k) * ld];
          }
          acc[s] = v;
        }
      }
    }
  }
  double* G = IB.Wg + (size_t)id * kSlot;
#pragma unroll
  for (int s = 0; s < kWS; ++s) {
    const int e = tid + kWideThreads * s;
    if (e < nt) {
      G[ei[s] + ej[s] * 32] = acc[s];
      G[ej[s] + ei[s] * 32] = acc[s];
    }
  }
}

// ------------------------------------------------------------- step 4
// Certificate and R_t = L^* for every cluster task of the batch: L^* W_t L -
// (tau + delta) I = L2 D2 L2^* with positive pivots, G_t = L L^*.  delta =
// 8 (levels + 4) (K + 32) eps_mach tr(G_t) tr(W_t) bounds the rounding of
// the Gram sums over the levels of the tree, the K-term products and
// factorisations and the orthonormality tolerance of the unchanged basis,
// with slack (normwise bounds, tr(G_t) tr(W_t) >= ||G_t|| ||W_t||).  Tiles
// have leading dimension ld = largest K + 1.  Two launches over all tasks:
// kGeneral = false takes the tasks whose V_t is orthonormal (block formulas,
// a K x u tile for C_t and L_S), kGeneral = true the others (factorisation
// of the whole G_t).
// Doubles of the third tile of k_certify: the general form keeps W L (K x K);
// the block form keeps Y and Z (u x K, ld u + 1) and then the float32 copy
// of the certificate matrix (K x K floats, ld ld).
__host__ __device__ inline int certify_t2(bool general, int ld, int u) {
  const int tile = ld * (ld - 1);
  const int yz = (u + 1) * (ld - 1);
  const int fs = (tile + 1) / 2;
  return general ? tile : (yz > fs ? yz : fs);
}

template <bool kGeneral>
__global__ void k_certify(const Item* __restrict__ items, int n, int u, int ld, int levels, double eps,
                          BaseWeights BW, ItemBuffers IB) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int id = blockIdx.x * (blockDim.x >> 5) + w;
  if (id >= n) return;
  const Item it = items[id];
  const bool orth = pick(BW.orth, it.side)[it.cluster] != 0;
  if (orth == kGeneral) return;
  const int k = it.k;
  const int K = k + u;
  const int tile = ld * (ld - 1);
  // general: T0 = G_t / L (K x K); orthonormal: T0 = [C_t; S or L_S] (K x u)
  const int t0 = kGeneral ? tile : ld * u;
  const int t2 = certify_t2(kGeneral, ld, u);
  double* T0 = smem + (size_t)w * (tile + t0 + t2 + 64);
  double* T1 = T0 + t0;
  double* T2 = T1 + tile;
  double* lv = T2 + t2;
  double* dsq = lv + 32;
  const double* Gv = IB.Gv + (size_t)id * kSlot;
  load_tile(T1, ld, IB.Wg + (size_t)id * kSlot, 32, K, K, lane);
  const double trW = warp_sum(lane < K ? IB.Wg[(size_t)id * kSlot + lane * 33] : 0.0);
  double trG;
  bool ok;
  if constexpr (!kGeneral) {
    // C(p, q) = T0[p + q ld] (p < k), S(a, b) = Sb[a + b ld] = T0[k + a + b ld]
    load_tile(T0, ld, Gv + k * 32, 32, K, u, lane);
    trG = k + warp_sum(lane < u ? Gv[(k + lane) * 33] : 0.0);
    __syncwarp();
    double* Sb = T0 + k;
    for (int e = lane; e < tri(u); e += 32) {
      int a, b;
      tri_index(e, a, b);
      double v = Sb[a + b * ld];
      for (int p = 0; p < k; ++p) v = fma(-T0[p + a * ld], T0[p + b * ld], v);
      Sb[a + b * ld] = v;
    }
    __syncwarp();
    ok = trG > 0.0 && trW > 0.0 && trG * trW < DBL_MAX && ldl(Sb, ld, u, 0.0, lv, lane);
    if (ok) {
      ldl_to_cholesky(Sb, ld, u, dsq, lane);
      // C2 = L^* W L with L = [[I, 0], [C^*, L_S]], blockwise:
      //   Y = W21 + W22 C^* (u x k), Z = W22 L_S (u x u) into T2, then over W
      //   C2_11 = W11 + W12 C^* + C Y, C2_21 = L_S^* Y, C2_22 = L_S^* Z
      const int ldy = u + 1;
      for (int e = lane; e < u * K; e += 32) {
        const int a = e % u, j = e / u;
        double v;
        if (j < k) {
          v = T1[(k + a) + j * ld];
          for (int q = 0; q < u; ++q) v = fma(T1[(k + a) + (k + q) * ld], T0[j + q * ld], v);
        } else {
          const int b = j - k;
          v = 0.0;
          for (int p = b; p < u; ++p) v = fma(T1[(k + a) + (k + p) * ld], Sb[p + b * ld], v);
        }
        T2[a + j * ldy] = v;
      }
      __syncwarp();
      for (int e = lane; e < tri(K); e += 32) {
        int i, j;
        tri_index(e, i, j);
        double v;
        if (i < k) {
          v = T1[i + j * ld];
          for (int q = 0; q < u; ++q) v = fma(T1[i + (k + q) * ld], T0[j + q * ld], v);
          for (int q = 0; q < u; ++q) v = fma(T0[i + q * ld], T2[q + j * ldy], v);
        } else {
          const int a = i - k;
          v = 0.0;
          for (int q = a; q < u; ++q) v = fma(Sb[q + a * ld], T2[q + j * ldy], v);
        }
        T1[i + j * ld] = v;
      }
      __syncwarp();
    }
  } else {
    load_gram(T0, ld, Gv, pick(BW.Vg, it.side) + (size_t)it.cluster * kSlot, false, k, K, lane);
    __syncwarp();
    trG = warp_sum(lane < K ? T0[lane * (ld + 1)] : 0.0);
    ok = K >= 1 && trG > 0.0 && trW > 0.0 && trG * trW < DBL_MAX && ldl(T0, ld, K, 0.0, lv, lane);
    if (ok) {
      ldl_to_cholesky(T0, ld, K, dsq, lane);
      // T2 = W L
      for (int e = lane; e < K * K; e += 32) {
        const int i = e % K, j = e / K;
        double v = 0.0;
        for (int q = j; q < K; ++q) v = fma(T1[i + q * ld], T0[q + j * ld], v);
        T2[i + j * ld] = v;
      }
      __syncwarp();
      // C2 = L^* T2 (lower triangle) over W
      for (int e = lane; e < tri(K); e += 32) {
        int i, j;
        tri_index(e, i, j);
        double v = 0.0;
        for (int q = i; q < K; ++q) v = fma(T0[q + i * ld], T2[q + j * ld], v);
        T1[i + j * ld] = v;
      }
      __syncwarp();
    }
  }
  if (ok) {
    const double delta = 8.0 * (levels + 4) * (K + 32) * DBL_EPSILON * trG * trW;
    const int how = certify_pd(T1, ld, K, 0.25 * eps * eps + delta, reinterpret_cast<float*>(T2), lv, lane);
    ok = how != 0;
    if (lane == 0) IB.jac[4 * (size_t)id] = how == 2 ? 1ull : 0ull;   // float64 factorisation ran
  }
  if (!ok) {
    if (lane == 0) IB.fail[it.update] = 1;
    return;
  }
  // R_t = L^* (K x K upper, rows K..31 zero)
  double* Rt = IB.Rt + (size_t)id * kSlot;
  for (int e = lane; e < 32 * K; e += 32) {
    const int p = e & 31, c = e >> 5;
    double v = 0.0;
    if constexpr (!kGeneral) {
      if (c < k)
        v = p == c ? 1.0 : 0.0;
      else if (p < k)
        v = T0[p + (c - k) * ld];                         // C_t
      else if (p <= c)
        v = T0[c + (p - k) * ld];                         // L_S^*
    } else {
      if (p <= c) v = T0[c + p * ld];
    }
    Rt[p + c * 32] = v;
  }
  if (lane == 0) IB.rank[id] = K;
}

// Shared doubles of one k_fbasis warp (tiles of tc columns).
__host__ __device__ constexpr int fbasis_doubles(int tc, bool general) {
  return (general ? 2 : 1) * (tc + 1) * tc + kLd * tc + 32;
}

// New leaf bases V~_t L_t^{-*}, transfer matrices L_t^* E~_t L_{t+}^{-*} and
// the commit E_t0 <- L_t0^* [E_t0; 0] for the certified updates (one launch,
// one warp per cluster task, lane = row, forward substitution with the
// factor in shared memory).  With orthonormal bases they reduce to
// (V_t, (A|_t - V_t C_t) L_S^{-*}), [[E_t, (C_t - E_t C_p) L_Sp^{-*}],
// [0, L_St^* L_Sp^{-*}]] and [E_t0; 0].  Two launches over all tasks:
// kGeneral = false does the parts that have the block form and marks, for
// the tasks of updates whose certificate failed, their cluster and its
// ancestors for the exact path; kGeneral = true does the other parts.
// Block-form launches use two warps per block and ten blocks per SM (their
// shared tiles allow ten; the register budget is held to match).
constexpr int kFbWarps = 2;

template <bool kGeneral, int UMAX>
__global__ void __launch_bounds__(kGeneral ? 128 : 32 * kFbWarps, kGeneral ? 1 : 10)
k_fbasis(MatView M, const Item* __restrict__ items, int n, int u, int tc,
                         const double* __restrict__ A, const double* __restrict__ B, ItemBuffers IB,
                         BaseWeights BW) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int id = blockIdx.x * (blockDim.x >> 5) + w;
  if (id >= n) return;
  // R_t and E_t tiles with leading dimension tc + 1, the tile of 32 rows of
  // V_t (or R_{t+}) with kLd
  // (the block-form variant reads E_t from global memory and has no third tile)
  const int ldt = tc + 1;
  double* T0 = smem + (size_t)w * fbasis_doubles(tc, kGeneral);
  double* T1 = T0 + ldt * tc;
  double* T2 = T1 + kLd * tc;
  double* ri = kGeneral ? T2 + ldt * tc : T2;
  const Item it = items[id];
  const int side = it.side;
  if (IB.fail[it.update]) {
    if (!kGeneral && lane == 0) {
      const int32_t* father = pick(M.father, side);
      int32_t* need = pick(BW.need, side);
      for (int c = it.cluster; c >= 0; c = father[c]) need[c] = 1;
    }
    return;
  }
  const int k = it.k;
  const int K = k + u;
  const int kcap = M.kcap;
  const int32_t* orthv = pick(BW.orth, side);
  const bool orth = orthv[it.cluster] != 0;
  const bool has_transfer = !(it.flags & kItemTreeRoot);
  const bool root = it.flags & kItemRoot;
  const bool orth_p = has_transfer && !root && orthv[pick(M.father, side)[it.cluster]] != 0;
  // which kernel does which part: the block form needs V_t (and, for a
  // transfer matrix below the subtree root, V_{t+}) orthonormal
  const bool do_leaf = (it.flags & kItemLeaf) && (orth == !kGeneral);
  const bool do_transfer = has_transfer && ((root ? orth : orth && orth_p) == !kGeneral);
  if (!do_leaf && !do_transfer) return;
  // R_t = L_t^* (upper) into T0, as stored
  load_tile(T0, ldt, IB.Rt + (size_t)id * kSlot, 32, K, K, lane);   // zero below the diagonal
  __syncwarp();
  if (do_leaf) {
    if (lane < K) ri[lane] = recip(T0[lane * (ldt + 1)]);
    __syncwarp();
    const double* V = pick(M.leaf, side) + pick(M.leaf_off, side)[it.cluster];
    const double* F = (side == 0 ? A : B) + it.foff;
    const int m = it.size;
    double* Q = IB.Q + it.qoff;
    for (int r0 = 0; r0 < m; r0 += 32) {
      const int r = r0 + lane;
      const bool act = r < m;
      if constexpr (!kGeneral) {
        // y = (row of A|_t - row of V_t C_t) L_S^{-*}; V_t is copied (its
        // rows staged in T1, lane = row)
        load_tile(T1, kLd, V + r0, m, min(32, m - r0), k, lane);
        __syncwarp();
        if (act)
          for (int c = 0; c < k; ++c) Q[r + (size_t)c * m] = T1[lane + c * kLd];
        double y[UMAX];
#pragma unroll
        for (int q = 0; q < UMAX; ++q)
          if (q < u) {
            double a = act ? F[(it.rowoff + r) + (size_t)q * it.ld] : 0.0;
            for (int p = 0; p < k; ++p) a = fma(-T1[lane + p * kLd], T0[p + (k + q) * ldt], a);
#pragma unroll
            for (int p = 0; p < q; ++p) a = fma(-T0[(k + p) + (k + q) * ldt], y[p], a);
            y[q] = a * ri[k + q];
          }
        if (act)
#pragma unroll
          for (int q = 0; q < UMAX; ++q)
            if (q < u) Q[r + (size_t)(k + q) * m] = y[q];
      } else {
        double y[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          if (c < K) {
            double v = 0.0;
            if (act) v = c < k ? V[r + (size_t)c * m] : F[(it.rowoff + r) + (size_t)(c - k) * it.ld];
#pragma unroll
            for (int p = 0; p < c; ++p) v = fma(-T0[p + c * ldt], y[p], v);
            y[c] = v * ri[c];
          }
        }
        if (act)
#pragma unroll
          for (int c = 0; c < 32; ++c)
            if (c < K) Q[r + (size_t)c * m] = y[c];
      }
    }
    __syncwarp();
  }
  if (!do_transfer) return;
  const int kf = it.kf;
  const double* Eg = pick(M.transfer, side) + (size_t)it.cluster * kcap * kcap;   // E_t (k x kf, ld kcap)
  if constexpr (kGeneral) load_tile(T2, ldt, Eg, kcap, k, kf, lane);
  double* Fo = IB.F + (size_t)id * kSlot;
  const int i = lane;
  __syncwarp();
  if (root) {
    // commit: E_t0 <- L^* [E_t0; 0] (K x kf), lane = row; [E_t0; 0] when
    // V_t0 is orthonormal
    if constexpr (!kGeneral) {
      if (i < K)
        for (int j = 0; j < kf; ++j) Fo[i + j * 32] = i < k ? Eg[i + (size_t)j * kcap] : 0.0;
    } else {
      double z[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) z[j] = 0.0;
      for (int q = 0; q < k; ++q) {
        const double lq = (i < K && q >= i) ? T0[i + q * ldt] : 0.0;
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < kf) z[j] = fma(lq, T2[q + j * ldt], z[j]);
      }
      if (i < K)
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < kf) Fo[i + j * 32] = z[j];
    }
    return;
  }
  // new transfer matrix (K x Kf), lane = row
  const int Kf = kf + u;
  load_tile(T1, kLd, IB.Rt + (size_t)it.parent * kSlot, 32, Kf, Kf, lane);   // R_p = L_p^* (upper)
  __syncwarp();
  if (lane < Kf) ri[lane] = recip(T1[lane * (kLd + 1)]);
  __syncwarp();
  if constexpr (!kGeneral) {
    // rows i < k: [E_t, (C_t - E_t C_p) L_Sp^{-*}]; rows k + a: [0, (row a
    // of L_St^*) L_Sp^{-*}].  C_t - E_t C_p over all lanes (entry (ii, q)
    // per lane, in place of C_t in the tile of R_t), then lane = row.
    for (int e = lane; e < k * u; e += 32) {
      const int ii = e % k, q = e / k;
      double v = T0[ii + (k + q) * ldt];
      for (int p = 0; p < kf; ++p) v = fma(-Eg[ii + (size_t)p * kcap], T1[p + (kf + q) * kLd], v);
      T0[ii + (k + q) * ldt] = v;
    }
    __syncwarp();
    double x[UMAX];
#pragma unroll
    for (int q = 0; q < UMAX; ++q)
      if (q < u) x[q] = (i < K && k + q >= i) ? T0[i + (k + q) * ldt] : 0.0;
#pragma unroll
    for (int q = 0; q < UMAX; ++q)
      if (q < u) {
        double v = x[q];
#pragma unroll
        for (int p = 0; p < q; ++p) v = fma(-T1[(kf + p) + (kf + q) * kLd], x[p], v);
        x[q] = v * ri[kf + q];
      }
    if (i < K) {
      for (int j = 0; j < kf; ++j) Fo[i + j * 32] = i < k ? Eg[i + (size_t)j * kcap] : 0.0;
#pragma unroll
      for (int q = 0; q < UMAX; ++q)
        if (q < u) Fo[i + (kf + q) * 32] = x[q];
    }
    return;
  } else {
  // general: L_t^* E~_t L_p^{-*}
  double z[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) z[j] = 0.0;
  for (int q = 0; q < k; ++q) {
    const double lq = (i < K && q >= i) ? T0[i + q * ldt] : 0.0;
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < kf) z[j] = fma(lq, T2[q + j * ldt], z[j]);
  }
  // identity part of E~_t: column kf + jj picks row k + jj of L_t^*
#pragma unroll
  for (int j = 0; j < 32; ++j)
    if (j >= kf && j < Kf) {
      const int q = k + j - kf;
      z[j] = (i < K && q >= i) ? T0[i + q * ldt] : 0.0;
    }
  // z <- z L_p^{-*}: forward substitution over the columns
#pragma unroll
  for (int j = 0; j < 32; ++j)
    if (j < Kf) {
      double v = z[j];
#pragma unroll
      for (int q = 0; q < j; ++q) v = fma(-T1[q + j * kLd], z[q], v);
      z[j] = v * ri[j];
    }
  if (i < K)
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < Kf) Fo[i + j * 32] = z[j];
  }
}

constexpr int kWarps = 4;

// Per-lane accumulator slots for `entries` lower-triangle entries: 5, 10 or
// kNS (the fewer, the fewer registers a lane holds).
int slots_for(int entries) {
  const int need = (entries + 31) / 32;
  return need <= 5 ? 5 : need <= 10 ? 10 : kNS;
}



int blocks_for(int n) { return (n + kWarps - 1) / kWarps; }

// Columns of the shared tiles: the largest extended rank of the batch or the
// largest rank of the matrix (fathers of the subtree roots).
int tile_cols(const Pipeline& P) { return P.kl > P.M.kcap ? P.kl : P.M.kcap; }

size_t tiles_bytes(int ntiles, int cols, int extra) {
  return (size_t)kWarps * (ntiles * kLd * cols + extra) * sizeof(double);
}

}  // namespace

void launch_gram_orth(const Pipeline& P, cudaStream_t st) {
  static std::atomic<unsigned long long> done{0};
  const int n = P.cl_ptr[P.levels];
  if (n <= 0) return;
  smem_limit(k_orth_local, tiles_bytes(1, 32, 0), done);
  k_orth_local<<<blocks_for(n), 32 * kWarps, tiles_bytes(1, P.M.kcap, 0), st>>>(P.M, P.cl_list, n, P.BW);
  k_orth_mark<<<(n + 127) / 128, 128, 0, st>>>(P.M, P.cl_list, n, P.BW);
}

void launch_gram_vbasis_level(const Pipeline& P, int level, cudaStream_t st) {
  static std::atomic<unsigned long long> done{0};
  const int n = P.cl_ptr[level + 1] - P.cl_ptr[level];
  if (n <= 0) return;
  smem_limit(k_vgram, tiles_bytes(3, 32, 0), done);
  k_vgram<<<blocks_for(n), 32 * kWarps, tiles_bytes(3, P.M.kcap, 0), st>>>(P.M, P.cl_list + P.cl_ptr[level], n,
                                                                          P.BW);
}

void launch_gram_base(const Pipeline& P, cudaStream_t st) {
  static std::atomic<unsigned long long> done{0};
  const int n = P.cl_ptr[P.levels];
  if (n <= 0) return;
  const auto go = [&](auto kern) {
    smem_limit(kern, tiles_bytes(1, 32, 0), done);
    kern<<<blocks_for(n), 32 * kWarps, tiles_bytes(1, P.M.kcap, 0), st>>>(P.M, P.cl_list, n, P.BL, P.BW, P.err);
  };
  const int ns = slots_for(P.M.kcap * (P.M.kcap + 1) / 2);
  if (ns == 5)
    go(k_bgram<5>);
  else if (ns == 10)
    go(k_bgram<10>);
  else
    go(k_bgram<kNS>);
}

void launch_gram_base_level(const Pipeline& P, int level, cudaStream_t st) {
  const int n = P.cl_ptr[level + 1] - P.cl_ptr[level];
  if (n <= 0) return;
  k_bgram_down<<<n, 32 * kDownWarps, 0, st>>>(P.M, P.cl_list + P.cl_ptr[level], n, P.BW);
}

int launch_gram_basis(const Pipeline& P, int level) {
  static std::atomic<unsigned long long> done{0};
  const int n = P.lvl_ptr[level + 1] - P.lvl_ptr[level];
  if (n <= 0) return 0;
  const int nl = P.lvl_leaves[level];
  const int32_t* list = P.lvl_list + P.lvl_ptr[level];
  int launches = 0;
  if (nl > 0) {
    const int tc = tile_cols(P);
    const auto go = [&](auto kern) {
      smem_limit(kern, tiles_bytes(1, 32, 0), done);
      kern<<<blocks_for(nl), 32 * kWarps, tiles_bytes(1, tc, 0), P.stream>>>(P.M, P.items, list, nl, P.u, tc, P.A,
                                                                            P.B, P.IB, P.err);
    };
    const int kk = P.M.kcap;
    const int ns = slots_for(kk * P.u + P.u * (P.u + 1) / 2);
    if (ns == 5)
      go(k_fgram<5>);
    else if (ns == 10)
      go(k_fgram<10>);
    else
      go(k_fgram<kNS>);
    ++launches;
  }
  if (n > nl) {
    k_fgram_inner<<<n - nl, 32 * kInnerWarps, 0, P.stream>>>(P.M, P.items, list + nl, n - nl, P.u, P.IB, P.err);
    ++launches;
  }
  return launches;
}

void launch_gram_norms(const Pipeline& P) {
  static std::atomic<unsigned long long> done{0};
  if (P.n_norms <= 0) return;
  const int tc = tile_cols(P);
  smem_limit(k_fnorms, tiles_bytes(3, 32, 0), done);
  k_fnorms<<<blocks_for(P.n_norms), 32 * kWarps, tiles_bytes(3, tc, 0), P.stream>>>(P.M, P.items, P.norms,
                                                                                    P.n_norms, P.u, tc, P.BW, P.IB);
}

void launch_gram_weights(const Pipeline& P, int level) {
  static std::atomic<unsigned long long> done{0};
  const int n = P.lvl_ptr[level + 1] - P.lvl_ptr[level];
  if (n <= 0) return;
  const int tc = tile_cols(P);
  const auto bytes = [](int warps, int c, int kc) { return (size_t)warps * fweights_doubles(c, kc) * sizeof(double); };
  if (n <= kWideMaxTasks) {
    // few tasks: one block of kWideWarps warps per task, one set of tiles
    static std::atomic<unsigned long long> done_wide{0};
    smem_limit(k_fweights_wide, bytes(1, 32, 32), done_wide);
    k_fweights_wide<<<n, kWideThreads, bytes(1, tc, P.M.kcap), P.stream>>>(P.M, P.items, P.ents,
                                                                 P.lvl_list + P.lvl_ptr[level], n, P.u, tc, P.BW,
                                                                 P.IB);
    return;
  }
  // two warps per block, tiles of (tc + 1) x tc
  constexpr int warps = 2;
  const auto go = [&](auto kern) {
    smem_limit(kern, bytes(warps, 32, 32), done);
    kern<<<(n + warps - 1) / warps, 32 * warps, bytes(warps, tc, P.M.kcap), P.stream>>>(
        P.M, P.items, P.ents, P.lvl_list + P.lvl_ptr[level], n, P.u, tc, P.BW, P.IB);
  };
  if (slots_for(P.kl * (P.kl + 1) / 2) <= 10)
    go(k_fweights<10>);
  else
    go(k_fweights<kNS>);
}

void launch_gram_certify(const Pipeline& P) {
  static std::atomic<unsigned long long> done[2] = {{0}, {0}};
  const int n = P.lvl_ptr[P.levels];
  if (n <= 0) return;
  const int ld = P.kl + 1;
  const auto bytes = [](bool general, int l, int u) {
    const int tile = l * (l - 1);
    return (size_t)kWarps * (tile + (general ? tile : l * u) + certify_t2(general, l, u) + 64) * sizeof(double);
  };
  smem_limit(k_certify<false>, bytes(true, 33, 32), done[0]);
  smem_limit(k_certify<true>, bytes(true, 33, 32), done[1]);
  k_certify<false><<<blocks_for(n), 32 * kWarps, bytes(false, ld, P.u), P.stream>>>(P.items, n, P.u, ld, P.levels,
                                                                                     P.eps, P.BW, P.IB);
  k_certify<true><<<blocks_for(n), 32 * kWarps, bytes(true, ld, P.u), P.stream>>>(P.items, n, P.u, ld, P.levels,
                                                                                  P.eps, P.BW, P.IB);
}

// two warps per block: the per-warp tiles, not the block size, limit the
// warps per SM, and smaller blocks pack the shared memory more tightly

template <int UMAX>
void launch_fbasis_block_form(const Pipeline& P, int n, int tc) {
  static std::atomic<unsigned long long> done{0};
  const size_t bytes = (size_t)kFbWarps * fbasis_doubles(tc, false) * sizeof(double);
  smem_limit(k_fbasis<false, UMAX>, (size_t)kFbWarps * fbasis_doubles(32, false) * sizeof(double), done);
  k_fbasis<false, UMAX><<<(n + kFbWarps - 1) / kFbWarps, 32 * kFbWarps, bytes, P.stream>>>(P.M, P.items, n, P.u,
                                                                                          tc, P.A, P.B, P.IB, P.BW);
}

void launch_gram_outputs(const Pipeline& P) {
  static std::atomic<unsigned long long> done{0};
  const int n = P.lvl_ptr[P.levels];
  if (n <= 0) return;
  const int tc = tile_cols(P);
  if (P.u <= 8)
    launch_fbasis_block_form<8>(P, n, tc);
  else if (P.u <= 16)
    launch_fbasis_block_form<16>(P, n, tc);
  else
    launch_fbasis_block_form<32>(P, n, tc);
  smem_limit(k_fbasis<true, 32>, (size_t)kWarps * fbasis_doubles(32, true) * sizeof(double), done);
  k_fbasis<true, 32><<<blocks_for(n), 32 * kWarps, (size_t)kWarps * fbasis_doubles(tc, true) * sizeof(double),
                       P.stream>>>(P.M, P.items, n, P.u, tc, P.A, P.B, P.IB, P.BW);
}

// The reciprocal above, element by element, for a check of its error bound
// against the correctly rounded quotient (diagnostic entry point).
__global__ void k_recip_check(const double* d, int64_t n, double* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = recip(d[i]);
}

void launch_recip_check(const double* d, int64_t n, double* out, cudaStream_t st) {
  if (n <= 0) return;
  const int threads = 256;
  k_recip_check<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(d, n, out);
}

}  // namespace h2
