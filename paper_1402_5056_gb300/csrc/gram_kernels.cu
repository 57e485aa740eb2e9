// Certified Gram path of the local low-rank update (Sections 4 and 5).
//
// When the truncation of every cluster of an update keeps the full extended
// rank K_t = k_t + u -- every singular value of V^_t B~_t^* above the
// threshold of the rank rule -- the new basis of t spans range(V~_t), and
// every quantity of steps 2-4 follows from K_t x K_t Gram matrices:
//   G_t = V~_t^* V~_t = R_t^* R_t  (leaf: Gram of (V_t, A|_t); inner: sum over
//                                   the sons of E~_s^* G_s E~_s)
//   ||Z~|_b||_F^2 = tr(S~_b^* G_t S~_b G_s)
//   W_t = B~_t^* B~_t             (sum of omega_b^2 S~_b G_s S~_b^* over
//                                   row(t), plus E~_t W_{t+} E~_t^*)
//   sigma_i(V^_t B~_t^*)^2 = lambda_i(G_t W_t) = lambda_i(L^* W_t L), G_t = L L^*.
// The certificate is an LDL^* factorisation of L^* W_t L - (tau + delta) I
// with positive pivots, tau = (eps/2)^2 the threshold of the rank rule and
// delta a bound on the rounding of G_t, W_t and the factorisations.  When it
// holds the rank rule keeps all K_t columns and any orthonormal basis of
// range(V~_t) gives the same projection as the singular vectors; the path
// takes Q_t = V~_t L^{-*} (orthonormal: Q_t^* Q_t = L^{-1} G_t L^{-*} = I),
// R_t = Q_t^* V~_t = L^*, new transfer matrices L_s^* E~_s L_t^{-*} and the
// commit E_t0 <- L_t0^* [E_t0; 0].  An update for which any cluster fails the
// certificate is recomputed by the exact path (Householder R-factors and a
// one-sided Jacobi SVD).
//
// Execution model: one warp per cluster (or block) task, K x K tiles in
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

// 1/d for a normal d > 0: the hardware estimate (relative error below
// 2^-22) refined by one cubic Newton-Raphson step y <- y (1 + e + e^2),
// e = 1 - d y, and one quadratic step, which leaves a few ulp.
__device__ __forceinline__ double recip(double d) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  double e = fma(-d, y, 1.0);
  y = fma(y, fma(e, e, e), y);
  e = fma(-d, y, 1.0);
  return fma(y, e, y);
}

// rows x cols block of a column-major global matrix (ld gld) into a tile.
__device__ __forceinline__ void load_tile(double* T, const double* g, int gld, int rows, int cols, int lane) {
  for (int c = 0; c < cols; ++c)
    for (int r = lane; r < rows; r += 32) T[r + c * kLd] = g[r + (size_t)c * gld];
}

// In-place LDL^* of A - shift I (lower triangle of the n x n tile A): on
// return the unit lower factor is below the diagonal and D on it.  lv holds
// 32 doubles of shared scratch.  Returns false (on every lane) as soon as a
// pivot is not positive.
__device__ __forceinline__ bool ldl(double* A, int n, double shift, double* lv, int lane) {
  if (lane < n) A[lane * (kLd + 1)] -= shift;
  __syncwarp();
  for (int j = 0; j < n; ++j) {
    const double d = A[j + j * kLd];
    if (!(d > 1e-300)) return false;
    const double r = recip(d);
    const int m = n - j - 1;
    if (lane < m) lv[lane] = A[j + 1 + lane + j * kLd] * r;
    __syncwarp();
    // trailing update A[p][q] -= a_pj l_qj for p >= q > j
    const int nt = tri(m);
    for (int e = lane; e < nt; e += 32) {
      int a, b;
      tri_index(e, a, b);
      const int p = j + 1 + a, q = j + 1 + b;
      A[p + q * kLd] = fma(-A[p + j * kLd], lv[b], A[p + q * kLd]);
    }
    __syncwarp();
    if (lane < m) A[j + 1 + lane + j * kLd] = lv[lane];
    __syncwarp();
  }
  return true;
}

// Rows of the outside-block stack of one block: X[r][q] = S_b[q][r] on the
// row side (rows of S_b^*), S_b[r][q] on the column side; l x k.
__device__ __forceinline__ void load_block_rows(double* X, const double* S, int kcap, int side, int l, int k,
                                                int lane) {
  if (side == 0) {
    for (int r = 0; r < l; ++r)
      if (lane < k) X[r + lane * kLd] = S[lane + (size_t)r * kcap];
  } else {
    for (int q = 0; q < k; ++q)
      if (lane < l) X[lane + q * kLd] = S[lane + (size_t)q * kcap];
  }
}

// acc (lower triangle of the k x k block in the per-lane layout) += w X^* X
// for the l x k tile X.
__device__ __forceinline__ void acc_gram(double (&acc)[kNS], const double* X, int l, int k, double w, int lane) {
  const int nt = tri(k);
#pragma unroll
  for (int s = 0; s < kNS; ++s) {
    if (32 * s >= nt) break;
    const int e = lane + 32 * s;
    if (e < nt) {
      int i, j;
      tri_index(e, i, j);
      double g = 0.0;
      for (int r = 0; r < l; ++r) g = fma(X[r + i * kLd], X[r + j * kLd], g);
      acc[s] = fma(w, g, acc[s]);
    }
  }
}

__device__ __forceinline__ double sum_squares(const double* X, int l, int k, int lane) {
  double part = 0.0;
  for (int e = lane; e < l * k; e += 32) {
    const double v = X[e % l + (e / l) * kLd];
    part = fma(v, v, part);
  }
  return warp_sum(part);
}

// Store the lower-triangle accumulator as a full symmetric n x n matrix
// (global slot, ld 32).
__device__ __forceinline__ void store_sym(double* G, const double (&acc)[kNS], int n, int lane) {
  const int nt = tri(n);
#pragma unroll
  for (int s = 0; s < kNS; ++s) {
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

// ------------------------------------------------- weights of the unchanged matrix
// Wo_c = sum over b in row(c) of omega_b^2 S_b S_b^* (column side S_b^* S_b),
// omega_b = sqrt(#T_c) / ||S_b||_F, for every cluster of both sides; the
// Gram of the stack whose R-factor the exact path folds.
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
  double acc[kNS];
#pragma unroll
  for (int s = 0; s < kNS; ++s) acc[s] = 0.0;
  for (int e = pick(BL.ptr, side)[c]; e < pick(BL.ptr, side)[c + 1]; ++e) {
    const int slot = pick(BL.adm, side)[e];
    const int l = pick(M.rank, 1 - side)[pick(BL.other, side)[slot]];
    load_block_rows(X, M.S + (size_t)slot * kcap * kcap, kcap, side, l, k, lane);
    __syncwarp();
    const double nrm2 = sum_squares(X, l, k, lane);
    const double w2 = nrm2 > 1e-300 ? st * recip(nrm2) : 0.0;
    acc_gram(acc, X, l, k, w2, lane);
    __syncwarp();
  }
  store_sym(pick(BW.Wo, side) + (size_t)c * kSlot, acc, k, lane);
}

// W0_c = Wo_c + E_c W0_{c+} E_c^* top-down (one launch per level).
__global__ void k_bgram_down(MatView M, const int32_t* __restrict__ list, int n, BaseWeights BW) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int idx = blockIdx.x * (blockDim.x >> 5) + w;
  if (idx >= n) return;
  const int kcap = M.kcap;
  double* T0 = smem + (size_t)w * 3 * kLd * kcap;
  double* T1 = T0 + kLd * kcap;
  double* T2 = T1 + kLd * kcap;
  const int side = list[idx] >> 30;
  const int c = list[idx] & 0x3fffffff;
  const int k = pick(M.rank, side)[c];
  if (k > 32) return;
  const double* Wo = pick(BW.Wo, side) + (size_t)c * kSlot;
  const int f = pick(M.father, side)[c];
  const int nt = tri(k);
  double acc[kNS];
#pragma unroll
  for (int s = 0; s < kNS; ++s) {
    const int e = lane + 32 * s;
    double v = 0.0;
    if (e < nt) {
      int i, j;
      tri_index(e, i, j);
      v = Wo[i + j * 32];
    }
    acc[s] = v;
  }
  if (f >= 0) {
    const int kf = pick(M.rank, side)[f];
    load_tile(T0, pick(BW.W0, side) + (size_t)f * kSlot, 32, kf, kf, lane);
    load_tile(T1, pick(M.transfer, side) + (size_t)c * kcap * kcap, kcap, k, kf, lane);
    __syncwarp();
    // T2 = E W0_f (k x kf)
    for (int e = lane; e < k * kf; e += 32) {
      const int i = e % k, j = e / k;
      double v = 0.0;
      for (int q = 0; q < kf; ++q) v = fma(T1[i + q * kLd], T0[q + j * kLd], v);
      T2[i + j * kLd] = v;
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < kNS; ++s) {
      if (32 * s >= nt) break;
      const int e = lane + 32 * s;
      if (e < nt) {
        int i, j;
        tri_index(e, i, j);
        double v = acc[s];
        for (int q = 0; q < kf; ++q) v = fma(T2[i + q * kLd], T1[j + q * kLd], v);
        acc[s] = v;
      }
    }
  }
  store_sym(pick(BW.W0, side) + (size_t)c * kSlot, acc, k, lane);
}

// ------------------------------------------------------------- step 2
// G_t = V~_t^* V~_t bottom-up: leaf Gram of (V_t, A|_t) over chunks of 32
// rows; inner sum over the sons of E~_s^* G_s E~_s, E~_s = diag(E_s, I_u).
__global__ void k_fgram(MatView M, const Item* __restrict__ items, const int32_t* __restrict__ list, int n, int u,
                        int tc, const double* __restrict__ A, const double* __restrict__ B, ItemBuffers IB,
                        int* err) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int idx = blockIdx.x * (blockDim.x >> 5) + w;
  if (idx >= n) return;
  double* T0 = smem + (size_t)w * 3 * kLd * tc;
  double* T1 = T0 + kLd * tc;
  double* T2 = T1 + kLd * tc;
  const int id = list[idx];
  const Item it = items[id];
  const int side = it.side;
  const int k = it.k;
  const int K = k + u;
  if (K > tc) {
    if (lane == 0) atomicOr(err, kErrCols);
    return;
  }
  const int nt = tri(K);
  double acc[kNS];
#pragma unroll
  for (int s = 0; s < kNS; ++s) acc[s] = 0.0;
  if (it.flags & kItemLeaf) {
    const double* V = pick(M.leaf, side) + pick(M.leaf_off, side)[it.cluster];
    const double* F = (side == 0 ? A : B) + it.foff;
    const int m = it.size;
    for (int r0 = 0; r0 < m; r0 += 32) {
      const int ch = min(32, m - r0);
      if (lane < ch) {
        for (int c = 0; c < k; ++c) T0[lane + c * kLd] = V[(r0 + lane) + (size_t)c * m];
        for (int c = 0; c < u; ++c) T0[lane + (k + c) * kLd] = F[(it.rowoff + r0 + lane) + (size_t)c * it.ld];
      }
      __syncwarp();
      acc_gram(acc, T0, ch, K, 1.0, lane);
      __syncwarp();
    }
  } else {
    const int kcap = M.kcap;
    for (int si = 0; si < 2; ++si) {
      const int sid = si == 0 ? it.son0 : it.son1;
      const Item sn = items[sid];
      const int ks = sn.k;
      const int Ks = ks + u;
      load_tile(T0, IB.Gv + (size_t)sid * kSlot, 32, Ks, Ks, lane);
      load_tile(T1, pick(M.transfer, side) + (size_t)sn.cluster * kcap * kcap, kcap, ks, k, lane);
      __syncwarp();
      // T2 = G_s E~_s (Ks x K)
      for (int e = lane; e < Ks * K; e += 32) {
        const int i = e % Ks, j = e / Ks;
        double v;
        if (j < k) {
          v = 0.0;
          for (int q = 0; q < ks; ++q) v = fma(T0[i + q * kLd], T1[q + j * kLd], v);
        } else {
          v = T0[i + (ks + j - k) * kLd];
        }
        T2[i + j * kLd] = v;
      }
      __syncwarp();
      // acc += E~_s^* T2
#pragma unroll
      for (int s = 0; s < kNS; ++s) {
        if (32 * s >= nt) break;
        const int e = lane + 32 * s;
        if (e < nt) {
          int i, j;
          tri_index(e, i, j);
          double v = acc[s];
          if (i < k) {
            for (int q = 0; q < ks; ++q) v = fma(T1[q + i * kLd], T2[q + j * kLd], v);
          } else {
            v += T2[ks + i - k + j * kLd];
          }
          acc[s] = v;
        }
      }
      __syncwarp();
    }
  }
  store_sym(IB.Gv + (size_t)id * kSlot, acc, K, lane);
}

// ||Z~|_b||_F^2 = tr(S~_b^* G_t S~_b G_s) for the blocks inside the update,
// S~_b = diag(S_b, I_u): entry (i, j) of G_t S~_b times entry (i, j) of
// S~_b G_s, summed.
__global__ void k_fnorms(MatView M, const Item* __restrict__ items, const NormTask* __restrict__ tasks, int n,
                         int u, int tc, ItemBuffers IB) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int idx = blockIdx.x * (blockDim.x >> 5) + w;
  if (idx >= n) return;
  double* T0 = smem + (size_t)w * 3 * kLd * tc;
  double* T1 = T0 + kLd * tc;
  double* T2 = T1 + kLd * tc;
  const NormTask tk = tasks[idx];
  const int kt = items[tk.it].k, ls = items[tk.is].k;
  const int Kt = kt + u, Ks = ls + u;
  const int kcap = M.kcap;
  load_tile(T0, IB.Gv + (size_t)tk.it * kSlot, 32, Kt, Kt, lane);
  load_tile(T1, IB.Gv + (size_t)tk.is * kSlot, 32, Ks, Ks, lane);
  load_tile(T2, M.S + (size_t)tk.slot * kcap * kcap, kcap, kt, ls, lane);
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
__global__ void k_fweights(MatView M, const Item* __restrict__ items, const Entry* __restrict__ ents,
                           const int32_t* __restrict__ list, int n, int u, int tc, BaseWeights BW, ItemBuffers IB) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int idx = blockIdx.x * (blockDim.x >> 5) + w;
  if (idx >= n) return;
  double* T0 = smem + (size_t)w * 3 * kLd * tc;
  double* T1 = T0 + kLd * tc;
  double* T2 = T1 + kLd * tc;
  const int id = list[idx];
  const Item it = items[id];
  const int side = it.side;
  const int k = it.k;
  const int K = k + u;
  const int kcap = M.kcap;
  const int nt = tri(K);
  const int ntk = tri(k);
  const double st = (double)pick(M.subtree, side)[it.cluster];
  const double* Gt = IB.Gv + (size_t)id * kSlot;
  // V_t orthonormal: |V_t^* V_t - I| within rounding
  bool orth = true;
  for (int e = lane; e < ntk; e += 32) {
    int i, j;
    tri_index(e, i, j);
    const double g = Gt[i + j * 32] - (i == j ? 1.0 : 0.0);
    if (fabs(g) > 256.0 * DBL_EPSILON) orth = false;
  }
  orth = __all_sync(kFull, orth);
  if (lane == 0) IB.jac[4 * (size_t)id + 3] = orth ? 0ull : 1ull;
  double acc[kNS];
#pragma unroll
  for (int s = 0; s < kNS; ++s) acc[s] = 0.0;
  if (orth) {
    const double* Wo = pick(BW.Wo, side) + (size_t)it.cluster * kSlot;
#pragma unroll
    for (int s = 0; s < kNS; ++s) {
      const int e = lane + 32 * s;
      if (e < ntk) {
        int i, j;
        tri_index(e, i, j);
        acc[s] = Wo[i + j * 32];
      }
    }
    if (it.flags & kItemInside)
      for (int e = it.ent_begin; e < it.ent_end; ++e) {
        const Entry en = ents[e];
        if (en.other < 0) continue;
        const int l = pick(M.rank, 1 - side)[en.other_cluster];
        load_block_rows(T0, M.S + (size_t)en.slot * kcap * kcap, kcap, side, l, k, lane);
        __syncwarp();
        const double nrm2 = sum_squares(T0, l, k, lane);
        const double w2 = nrm2 > 1e-300 ? st * recip(nrm2) : 0.0;
        acc_gram(acc, T0, l, k, -w2, lane);
        __syncwarp();
      }
  } else {
    load_tile(T1, Gt, 32, k, k, lane);
    for (int e = it.ent_begin; e < it.ent_end; ++e) {
      const Entry en = ents[e];
      if (en.other >= 0) continue;
      const int l = pick(M.rank, 1 - side)[en.other_cluster];
      load_block_rows(T0, M.S + (size_t)en.slot * kcap * kcap, kcap, side, l, k, lane);
      __syncwarp();
      // ||R_kk S_b||_F^2 = sum over rows x of X of x G_kk x^*
      double part = 0.0;
      for (int e2 = lane; e2 < l * k; e2 += 32) {
        const int r = e2 % l, q = e2 / l;
        double y = 0.0;
        for (int p = 0; p < k; ++p) y = fma(T0[r + p * kLd], T1[p + q * kLd], y);
        part = fma(y, T0[r + q * kLd], part);
      }
      const double nrm2 = warp_sum(part);
      const double w2 = nrm2 > 1e-300 ? st * recip(nrm2) : 0.0;
      acc_gram(acc, T0, l, k, w2, lane);
      __syncwarp();
    }
  }
  // blocks inside the update
  if (it.flags & kItemInside)
    for (int e = it.ent_begin; e < it.ent_end; ++e) {
      const Entry en = ents[e];
      if (en.other < 0) continue;
      const int l = items[en.other].k;
      const int Ko = l + u;
      const double nrm = IB.norms[en.norm];
      const double w2 = nrm > 1e-150 ? st * recip(nrm * nrm) : 0.0;
      load_tile(T1, IB.Gv + (size_t)en.other * kSlot, 32, Ko, Ko, lane);
      // T0 = S' (k x l): S_b on the row side, S_b^* on the column side
      const double* S = M.S + (size_t)en.slot * kcap * kcap;
      if (side == 0) {
        load_tile(T0, S, kcap, k, l, lane);
      } else {
        for (int q = 0; q < l; ++q)
          if (lane < k) T0[lane + q * kLd] = S[q + (size_t)lane * kcap];
      }
      __syncwarp();
      // T2 = P G_o (K x Ko)
      for (int e2 = lane; e2 < K * Ko; e2 += 32) {
        const int i = e2 % K, j = e2 / K;
        double v;
        if (i < k) {
          v = 0.0;
          for (int q = 0; q < l; ++q) v = fma(T0[i + q * kLd], T1[q + j * kLd], v);
        } else {
          v = T1[l + i - k + j * kLd];
        }
        T2[i + j * kLd] = v;
      }
      __syncwarp();
#pragma unroll
      for (int s = 0; s < kNS; ++s) {
        if (32 * s >= nt) break;
        const int e2 = lane + 32 * s;
        if (e2 < nt) {
          int i, j;
          tri_index(e2, i, j);
          double v;
          if (j < k) {
            v = 0.0;
            for (int q = 0; q < l; ++q) v = fma(T2[i + q * kLd], T0[j + q * kLd], v);
          } else {
            v = T2[i + (l + j - k) * kLd];
          }
          acc[s] = fma(w2, v, acc[s]);
        }
      }
      __syncwarp();
    }
  // father's part
  if (it.flags & kItemRoot) {
    if (!(it.flags & kItemTreeRoot)) {
      const int f = pick(M.father, side)[it.cluster];
      const int kf = it.kf;
      load_tile(T1, pick(BW.W0, side) + (size_t)f * kSlot, 32, kf, kf, lane);
      load_tile(T0, pick(M.transfer, side) + (size_t)it.cluster * kcap * kcap, kcap, k, kf, lane);
      __syncwarp();
      for (int e2 = lane; e2 < k * kf; e2 += 32) {
        const int i = e2 % k, j = e2 / k;
        double v = 0.0;
        for (int q = 0; q < kf; ++q) v = fma(T0[i + q * kLd], T1[q + j * kLd], v);
        T2[i + j * kLd] = v;
      }
      __syncwarp();
#pragma unroll
      for (int s = 0; s < kNS; ++s) {
        if (32 * s >= ntk) break;
        const int e2 = lane + 32 * s;
        if (e2 < ntk) {
          int i, j;
          tri_index(e2, i, j);
          double v = acc[s];
          for (int q = 0; q < kf; ++q) v = fma(T2[i + q * kLd], T0[j + q * kLd], v);
          acc[s] = v;
        }
      }
    }
  } else {
    const int kf = items[it.parent].k;
    const int Kf = kf + u;
    load_tile(T1, IB.Wg + (size_t)it.parent * kSlot, 32, Kf, Kf, lane);
    load_tile(T0, pick(M.transfer, side) + (size_t)it.cluster * kcap * kcap, kcap, k, kf, lane);
    __syncwarp();
    // T2 = E~_t W_p (K x Kf)
    for (int e2 = lane; e2 < K * Kf; e2 += 32) {
      const int i = e2 % K, j = e2 / K;
      double v;
      if (i < k) {
        v = 0.0;
        for (int q = 0; q < kf; ++q) v = fma(T0[i + q * kLd], T1[q + j * kLd], v);
      } else {
        v = T1[kf + i - k + j * kLd];
      }
      T2[i + j * kLd] = v;
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < kNS; ++s) {
      if (32 * s >= nt) break;
      const int e2 = lane + 32 * s;
      if (e2 < nt) {
        int i, j;
        tri_index(e2, i, j);
        double v = acc[s];
        if (j < k) {
          for (int q = 0; q < kf; ++q) v = fma(T2[i + q * kLd], T0[j + q * kLd], v);
        } else {
          v += T2[i + (kf + j - k) * kLd];
        }
        acc[s] = v;
      }
    }
  }
  store_sym(IB.Wg + (size_t)id * kSlot, acc, K, lane);
}

// ------------------------------------------------------------- step 4
// Certificate and R_t = L^* for every cluster task of the batch (one
// launch): G_t = L D L^*, L_G = L D^{1/2}, C = L_G^* W_t L_G, LDL^* of
// C - (tau + delta) I.  delta = 8 (levels + 4) (K + 32) eps_mach tr(G_t)
// tr(W_t) bounds the rounding of the Gram sums over the levels of the tree
// and the K-term products and factorisations, with slack (normwise bounds,
// tr(G_t) tr(W_t) >= ||G_t|| ||W_t||).
__global__ void k_certify(const Item* __restrict__ items, int n, int u, int tc, int levels, double eps,
                          ItemBuffers IB) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int id = blockIdx.x * (blockDim.x >> 5) + w;
  if (id >= n) return;
  double* T0 = smem + (size_t)w * (3 * kLd * tc + 64);
  double* T1 = T0 + kLd * tc;
  double* T2 = T1 + kLd * tc;
  double* lv = T2 + kLd * tc;
  double* dsq = lv + 32;
  const Item it = items[id];
  const int K = it.k + u;
  load_tile(T0, IB.Gv + (size_t)id * kSlot, 32, K, K, lane);
  load_tile(T1, IB.Wg + (size_t)id * kSlot, 32, K, K, lane);
  __syncwarp();
  const double trG = warp_sum(lane < K ? T0[lane * (kLd + 1)] : 0.0);
  const double trW = warp_sum(lane < K ? T1[lane * (kLd + 1)] : 0.0);
  const double scale = trG * trW;
  bool ok = K >= 1 && trG > 0.0 && trW > 0.0 && scale < DBL_MAX;
  if (ok) ok = ldl(T0, K, 0.0, lv, lane);
  if (ok) {
    // L_G = L D^{1/2}
    if (lane < K) dsq[lane] = sqrt(T0[lane * (kLd + 1)]);
    __syncwarp();
    for (int e = lane; e < tri(K); e += 32) {
      int i, j;
      tri_index(e, i, j);
      T0[i + j * kLd] = i == j ? dsq[j] : T0[i + j * kLd] * dsq[j];
    }
    __syncwarp();
    // T2 = W L_G
    for (int e = lane; e < K * K; e += 32) {
      const int i = e % K, j = e / K;
      double v = 0.0;
      for (int q = j; q < K; ++q) v = fma(T1[i + q * kLd], T0[q + j * kLd], v);
      T2[i + j * kLd] = v;
    }
    __syncwarp();
    // C = L_G^* T2 (lower triangle) over W
    for (int e = lane; e < tri(K); e += 32) {
      int i, j;
      tri_index(e, i, j);
      double v = 0.0;
      for (int q = i; q < K; ++q) v = fma(T0[q + i * kLd], T2[q + j * kLd], v);
      T1[i + j * kLd] = v;
    }
    __syncwarp();
    const double delta = 8.0 * (levels + 4) * (K + 32) * DBL_EPSILON * scale;
    ok = ldl(T1, K, 0.25 * eps * eps + delta, lv, lane);
  }
  if (!ok) {
    if (lane == 0) IB.fail[it.update] = 1;
    return;
  }
  // R_t = L_G^* (K x K upper, rows K..31 zero)
  double* Rt = IB.Rt + (size_t)id * kSlot;
  for (int e = lane; e < 32 * K; e += 32) {
    const int p = e & 31, c = e >> 5;
    Rt[p + c * 32] = (p <= c) ? T0[c + p * kLd] : 0.0;
  }
  if (lane == 0) IB.rank[id] = K;
}

// New leaf bases V~_t L_t^{-*}, transfer matrices L_t^* E~_t L_{t+}^{-*} and
// the commit E_t0 <- L_t0^* [E_t0; 0] for the certified updates (one launch,
// one warp per cluster task, lane = row, forward substitution with the
// factor in shared memory).  Tasks of updates whose certificate failed mark
// their cluster and its ancestors for the exact path instead.
__global__ void k_fbasis(MatView M, const Item* __restrict__ items, int n, int u, int tc,
                         const double* __restrict__ A, const double* __restrict__ B, ItemBuffers IB,
                         BaseWeights BW) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int id = blockIdx.x * (blockDim.x >> 5) + w;
  if (id >= n) return;
  double* T0 = smem + (size_t)w * (3 * kLd * tc + 32);
  double* T1 = T0 + kLd * tc;
  double* T2 = T1 + kLd * tc;
  double* ri = T2 + kLd * tc;
  const Item it = items[id];
  const int side = it.side;
  if (IB.fail[it.update]) {
    if (lane == 0)
      for (int c = it.cluster; c >= 0; c = pick(M.father, side)[c]) pick(BW.need, side)[c] = 1;
    return;
  }
  const int k = it.k;
  const int K = k + u;
  const int kcap = M.kcap;
  // L_t (lower) from R_t = L_t^*
  const double* Rt = IB.Rt + (size_t)id * kSlot;
  for (int c = 0; c < K; ++c)
    if (lane <= c) T0[c + lane * kLd] = Rt[lane + c * 32];
  __syncwarp();
  if (it.flags & kItemLeaf) {
    if (lane < K) ri[lane] = recip(T0[lane * (kLd + 1)]);
    __syncwarp();
    const double* V = pick(M.leaf, side) + pick(M.leaf_off, side)[it.cluster];
    const double* F = (side == 0 ? A : B) + it.foff;
    const int m = it.size;
    double* Q = IB.Q + it.qoff;
    for (int r0 = 0; r0 < m; r0 += 32) {
      const int r = r0 + lane;
      const bool act = r < m;
      double y[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c < K) {
          double v = 0.0;
          if (act) v = c < k ? V[r + (size_t)c * m] : F[(it.rowoff + r) + (size_t)(c - k) * it.ld];
#pragma unroll
          for (int p = 0; p < c; ++p) v = fma(-T0[c + p * kLd], y[p], v);
          y[c] = v * ri[c];
        }
      }
      if (act)
#pragma unroll
        for (int c = 0; c < 32; ++c)
          if (c < K) Q[r + (size_t)c * m] = y[c];
    }
    __syncwarp();
  }
  if (it.flags & kItemTreeRoot) return;
  const int kf = it.kf;
  load_tile(T2, pick(M.transfer, side) + (size_t)it.cluster * kcap * kcap, kcap, k, kf, lane);
  double* Fo = IB.F + (size_t)id * kSlot;
  if (it.flags & kItemRoot) {
    // commit: E_t0 <- L^* [E_t0; 0] (K x kf), lane = row
    __syncwarp();
    const int i = lane;
    double z[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) z[j] = 0.0;
    for (int q = 0; q < k; ++q) {
      const double lq = (i < K && q >= i) ? T0[q + i * kLd] : 0.0;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < kf) z[j] = fma(lq, T2[q + j * kLd], z[j]);
    }
    if (i < K)
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < kf) Fo[i + j * 32] = z[j];
    return;
  }
  // new transfer matrix: L_t^* E~_t L_p^{-*} (K x Kf), lane = row
  const int Kf = kf + u;
  const double* Rp = IB.Rt + (size_t)it.parent * kSlot;
  for (int c = 0; c < Kf; ++c)
    if (lane <= c) T1[c + lane * kLd] = Rp[lane + c * 32];
  __syncwarp();
  if (lane < Kf) ri[lane] = recip(T1[lane * (kLd + 1)]);
  __syncwarp();
  const int i = lane;
  double z[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) z[j] = 0.0;
  for (int q = 0; q < k; ++q) {
    const double lq = (i < K && q >= i) ? T0[q + i * kLd] : 0.0;
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < kf) z[j] = fma(lq, T2[q + j * kLd], z[j]);
  }
  // identity part of E~_t: column kf + jj picks row k + jj of L_t^*
#pragma unroll
  for (int j = 0; j < 32; ++j)
    if (j >= kf && j < Kf) {
      const int q = k + j - kf;
      z[j] = (i < K && q >= i) ? T0[q + i * kLd] : 0.0;
    }
  // z <- z L_p^{-*}: forward substitution over the columns
#pragma unroll
  for (int j = 0; j < 32; ++j)
    if (j < Kf) {
      double v = z[j];
#pragma unroll
      for (int q = 0; q < j; ++q) v = fma(-T1[j + q * kLd], z[q], v);
      z[j] = v * ri[j];
    }
  if (i < K)
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < Kf) Fo[i + j * 32] = z[j];
}

constexpr int kWarps = 4;

int blocks_for(int n) { return (n + kWarps - 1) / kWarps; }

// Raise the dynamic shared memory limit of a kernel once per device.
template <class Kern>
void smem_limit(Kern kern, size_t bytes, unsigned long long& done) {
  int dev = 0;
  H2_CUDA(cudaGetDevice(&dev));
  if (dev < 64 && (done >> dev) & 1ull) return;
  H2_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  if (dev < 64) done |= 1ull << dev;
}

// Columns of the shared tiles: the largest extended rank of the batch or the
// largest rank of the matrix (fathers of the subtree roots).
int tile_cols(const Pipeline& P) { return P.kl > P.M.kcap ? P.kl : P.M.kcap; }

size_t tiles_bytes(int cols, int extra) { return (size_t)kWarps * (3 * kLd * cols + extra) * sizeof(double); }

}  // namespace

void launch_gram_base(const Pipeline& P, cudaStream_t st) {
  static unsigned long long done = 0;
  const int n = P.cl_ptr[P.levels];
  if (n <= 0) return;
  const size_t sm = (size_t)kWarps * kLd * P.M.kcap * sizeof(double);
  smem_limit(k_bgram, (size_t)kWarps * kLd * 32 * sizeof(double), done);
  k_bgram<<<blocks_for(n), 32 * kWarps, sm, st>>>(P.M, P.cl_list, n, P.BL, P.BW, P.err);
}

void launch_gram_base_level(const Pipeline& P, int level, cudaStream_t st) {
  static unsigned long long done = 0;
  const int n = P.cl_ptr[level + 1] - P.cl_ptr[level];
  if (n <= 0) return;
  smem_limit(k_bgram_down, tiles_bytes(32, 0), done);
  k_bgram_down<<<blocks_for(n), 32 * kWarps, tiles_bytes(P.M.kcap, 0), st>>>(P.M, P.cl_list + P.cl_ptr[level], n,
                                                                            P.BW);
}

void launch_gram_basis(const Pipeline& P, int level) {
  const int tc = tile_cols(P);
  static unsigned long long done = 0;
  const int n = P.lvl_ptr[level + 1] - P.lvl_ptr[level];
  if (n <= 0) return;
  smem_limit(k_fgram, tiles_bytes(32, 0), done);
  k_fgram<<<blocks_for(n), 32 * kWarps, tiles_bytes(tc, 0), P.stream>>>(
      P.M, P.items, P.lvl_list + P.lvl_ptr[level], n, P.u, tc, P.A, P.B, P.IB, P.err);
}

void launch_gram_norms(const Pipeline& P) {
  const int tc = tile_cols(P);
  static unsigned long long done = 0;
  if (P.n_norms <= 0) return;
  smem_limit(k_fnorms, tiles_bytes(32, 0), done);
  k_fnorms<<<blocks_for(P.n_norms), 32 * kWarps, tiles_bytes(tc, 0), P.stream>>>(P.M, P.items, P.norms,
                                                                                   P.n_norms, P.u, tc, P.IB);
}

void launch_gram_weights(const Pipeline& P, int level) {
  const int tc = tile_cols(P);
  static unsigned long long done = 0;
  const int n = P.lvl_ptr[level + 1] - P.lvl_ptr[level];
  if (n <= 0) return;
  smem_limit(k_fweights, tiles_bytes(32, 0), done);
  k_fweights<<<blocks_for(n), 32 * kWarps, tiles_bytes(tc, 0), P.stream>>>(
      P.M, P.items, P.ents, P.lvl_list + P.lvl_ptr[level], n, P.u, tc, P.BW, P.IB);
}

void launch_gram_certify(const Pipeline& P) {
  const int tc = tile_cols(P);
  static unsigned long long done = 0;
  const int n = P.lvl_ptr[P.levels];
  if (n <= 0) return;
  smem_limit(k_certify, tiles_bytes(32, 64), done);
  k_certify<<<blocks_for(n), 32 * kWarps, tiles_bytes(tc, 64), P.stream>>>(P.items, n, P.u, tc, P.levels,
                                                                             P.eps, P.IB);
}

void launch_gram_outputs(const Pipeline& P) {
  const int tc = tile_cols(P);
  static unsigned long long done = 0;
  const int n = P.lvl_ptr[P.levels];
  if (n <= 0) return;
  smem_limit(k_fbasis, tiles_bytes(32, 32), done);
  k_fbasis<<<blocks_for(n), 32 * kWarps, tiles_bytes(tc, 32), P.stream>>>(P.M, P.items, n, P.u, tc, P.A, P.B,
                                                                            P.IB, P.BW);
}

}  // namespace h2
