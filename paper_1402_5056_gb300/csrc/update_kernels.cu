// Batched FP64 kernels of the H^2 local low-rank update (Sections 4 and 5).
//
// Execution model: one warp per cluster task ("item") or per coupling
// task; lane c owns column c of every small matrix (at most 32 columns),
// so Householder reflections and Jacobi rotations are column operations
// without cross-lane reductions.  All clusters of one tree level of every
// update of the batch go into one launch; the host walks the levels
// bottom-up (R-factors, truncation) or top-down (weights).
#include <cfloat>
#include <cstdio>

#include "h2_internal.h"
#include "update_kernels.h"

namespace h2 {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kLdr = 33;          // leading dimension of R tiles in shared memory
constexpr int kCh = 32;           // rows per folded chunk
constexpr int kMaxSweeps = 40;

__device__ __forceinline__ void flag(int* err, int code) { atomicOr(err, code); }

// a[side] without dynamic indexing of a kernel-parameter array (which would
// copy the parameter struct to local memory)
template <class T>
__device__ __forceinline__ T pick(T const (&a)[2], int side) {
  return side ? a[1] : a[0];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// ---------------------------------------------------------------- teams
// A cluster task runs on a team of NW warps.  A warp issues its float64
// instructions to one sub-partition of the SM, which runs them at a
// quarter of the SM's float64 rate; a launch with few tasks (the
// factorisation applies its updates one at a time) therefore gives every
// task a block of kTW = 4 warps, one per sub-partition, and a launch with
// many tasks (a batch) runs one warp per task without block barriers.
// (Eight warps per task, two per sub-partition, measured slower: 31.8 s
// against 22.9 s for the local updates of the 128^2-cell factorisation.)  The arithmetic is the
// same in both forms: the rows of a task are dealt to kTW virtual warps,
// each forms its partial sums in row order, and the kTW partial sums are
// added by one pairwise tree -- one warp plays all kTW virtual warps when
// NW = 1.  An update gives the same bits whichever form its launches take.
constexpr int kTW = 4;               // virtual warps of a task
constexpr int kRW = kCh / kTW;       // rows of a 32-row chunk per virtual warp

// pairwise sum of the kTW partials p[0..kTW), the same tree everywhere
template <class T>
__device__ __forceinline__ T tree_sum(const T* p) {
  T q[kTW];
#pragma unroll
  for (int i = 0; i < kTW; ++i) q[i] = p[i];
#pragma unroll
  for (int h = 1; h < kTW; h <<= 1)
#pragma unroll
    for (int i = 0; i < kTW; i += 2 * h) q[i] = q[i] + q[i + h];
  return q[0];
}

template <int NW>
struct Team {
  static_assert(NW == 1 || NW == kTW, "a task runs on one warp or on kTW warps");
  static constexpr int VW = kTW / NW;   // virtual warps per warp
  static constexpr int kBuf = 3 * 32 * kTW;
  int wp;        // warp of the task (0 when NW = 1)
  int lane;
  double* buf;   // NW > 1: two buffers of kBuf doubles for the sums
  int ph;
  __device__ __forceinline__ int vw(int v) const { return wp * VW + v; }
  __device__ __forceinline__ bool lead() const { return wp == 0; }
  __device__ __forceinline__ void sync() const {
    if constexpr (NW > 1) __syncthreads();
    else __syncwarp();
  }
  // the kTW partials of this lane, gathered from the warps' slots of b
  template <class T>
  __device__ __forceinline__ T gather_sum(const double* b) const {
    T p[kTW];
#pragma unroll
    for (int w = 0; w < kTW; ++w) p[w] = (T)b[32 * w + lane];
    return tree_sum(p);
  }
  // Per-lane sums over the kTW virtual warps of x[v], added by the same
  // pairwise tree in both forms.  NW > 1: one barrier per call; the two
  // buffers alternate, so a buffer is written again only after every
  // thread passed the barrier of the call in between.  Every thread of the
  // team makes the same calls.
  template <class T>
  __device__ __forceinline__ void sum3(const T (&x)[VW], const T (&y)[VW], const T (&z)[VW], T& sx, T& sy, T& sz) {
    if constexpr (NW == 1) {
      sx = tree_sum(x);
      sy = tree_sum(y);
      sz = tree_sum(z);
    } else {
      double* b = buf + ph * kBuf;
      ph ^= 1;
      b[wp * 32 + lane] = x[0];
      b[32 * kTW + wp * 32 + lane] = y[0];
      b[64 * kTW + wp * 32 + lane] = z[0];
      __syncthreads();
      sx = gather_sum<T>(b);
      sy = gather_sum<T>(b + 32 * kTW);
      sz = gather_sum<T>(b + 64 * kTW);
    }
  }
  __device__ __forceinline__ double sum1(const double (&x)[VW]) {
    if constexpr (NW == 1) {
      return tree_sum(x);
    } else {
      double* b = buf + ph * kBuf;
      ph ^= 1;
      b[wp * 32 + lane] = x[0];
      __syncthreads();
      return gather_sum<double>(b);
    }
  }
  // maximum over the warps of a value (exact in any order)
  __device__ __forceinline__ double max1(double x) {
    if constexpr (NW == 1) {
      return x;
    } else {
      double* b = buf + ph * kBuf;
      ph ^= 1;
      b[wp * 32 + lane] = x;
      __syncthreads();
      double m = b[lane];
#pragma unroll
      for (int w = 1; w < kTW; ++w) m = fmax(m, b[32 * w + lane]);
      return m;
    }
  }
};

// R (ncol x ncol, upper triangular, shared, ld kLdr) <- R-factor of [R; X].
// X has `ch` rows; slot (v, ii) of the team's registers holds row
// kTW ii + vw(v), x[v][ii] = X[kTW ii + vw(v)][lane] (lane = column).  One
// Householder reflection H = I - tau u u^* per column j, u = [R_jj - beta;
// X[:, j]], beta = -sign(R_jj) ||[R_jj; X[:, j]]||, tau = -1 / (beta u_0):
// column j goes to vb (shared, by row), the two sums over the rows a column
// needs (its norm and its products with the trailing columns) come from one
// warp-order reduction, and the lead warp writes R.  R keeps ncol rows
// (rows beyond the rank stay zero).  R is complete on return.
template <int NW>
__device__ __forceinline__ void fold_t(double* R, double* vb, double (&x)[Team<NW>::VW][kRW], int ch, int ncol,
                                       Team<NW>& tm) {
  constexpr int VW = Team<NW>::VW;
  const int lane = tm.lane;
  for (int j = 0; j < ncol; ++j) {
    __syncwarp();   // the warp's reads of vb for the previous column are done
    double xi = 0.0;
#pragma unroll
    for (int v = 0; v < VW; ++v)
#pragma unroll
      for (int ii = 0; ii < kRW; ++ii)
        if (kTW * ii + tm.vw(v) < ch) {
          const double t = __shfl_sync(kFull, x[v][ii], j);
          if (lane == ii * VW + v) xi = t;
        }
    if (lane < kRW * VW) {
      const int i = kTW * (lane / VW) + tm.vw(lane % VW);
      if (i < ch) vb[i] = xi;
    }
    __syncwarp();
    // squared norm of the virtual warps' parts of column j: a butterfly over
    // the lanes that hold them (lane ii VW + v), the same tree in both forms
    double q = __dmul_rn(xi, xi);   // rounded here: never fused into the first sum
#pragma unroll
    for (int o = VW; o < kRW * VW; o <<= 1) q += __shfl_xor_sync(kFull, q, o);
    const bool trail = lane > j && lane < ncol;
    double s2[VW], dot[VW], none[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      s2[v] = __shfl_sync(kFull, q, v);
      dot[v] = 0.0;
      none[v] = 0.0;
      if (trail)
#pragma unroll
        for (int ii = 0; ii < kRW; ++ii) {
          const int i = kTW * ii + tm.vw(v);
          if (i < ch) dot[v] = fma(vb[i], x[v][ii], dot[v]);
        }
    }
    const double alpha = R[j + j * kLdr];   // read before the lead warp writes R below
    const double rjc = trail ? R[j + lane * kLdr] : 0.0;
    double S2, DOT, NONE;
    tm.sum3(s2, dot, none, S2, DOT, NONE);
    if (S2 == 0.0) continue;   // nothing below the diagonal: H = I
    const double nrm = sqrt(fma(alpha, alpha, S2));
    const double beta = alpha >= 0.0 ? -nrm : nrm;
    const double u0 = alpha - beta;
    const double tau = -1.0 / (beta * u0);
    if (lane == j) {
      if (tm.lead()) R[j + j * kLdr] = beta;
#pragma unroll
      for (int v = 0; v < VW; ++v)
#pragma unroll
        for (int ii = 0; ii < kRW; ++ii) x[v][ii] = 0.0;
    } else if (trail) {
      const double wc = tau * fma(u0, rjc, DOT);
      if (tm.lead()) R[j + lane * kLdr] = fma(-wc, u0, rjc);
#pragma unroll
      for (int v = 0; v < VW; ++v)
#pragma unroll
        for (int ii = 0; ii < kRW; ++ii) {
          const int i = kTW * ii + tm.vw(v);
          if (i < ch) x[v][ii] = fma(-wc, vb[i], x[v][ii]);
        }
    }
  }
  tm.sync();
}

template <int NW>
__device__ __forceinline__ void zero_tile_t(double* R, const Team<NW>& tm) {
  for (int c = tm.wp; c < 32; c += NW) R[tm.lane + c * kLdr] = 0.0;
  tm.sync();
}

// Copy the ncol x ncol upper part of a shared R tile to a global 32x32
// slot (columns beyond ncol are not written).
template <int NW>
__device__ __forceinline__ void store_tile_t(double* dst, const double* R, int ncol, const Team<NW>& tm) {
  tm.sync();
  for (int c = tm.wp; c < ncol; c += NW) dst[tm.lane + c * 32] = tm.lane < ncol ? R[tm.lane + c * kLdr] : 0.0;
}

// Shared memory of one task of the fold kernels (doubles): the R tile, the
// pivot column and, for kTW-warp teams, the sum buffers.
__host__ __device__ constexpr int fold_doubles(int nw) { return 32 * kLdr + 32 + (nw > 1 ? 2 * 96 * kTW : 0); }

// Task index, team and shared memory of a task of a kernel launched with
// one block of kTW warps per task (NW = kTW) or one warp per task (NW = 1);
// `per` doubles of dynamic shared memory per task.
template <int NW>
__device__ __forceinline__ int team_task(Team<NW>& tm, double*& base, double* smem, int per, int sums_off) {
  const int w = threadIdx.x >> 5;
  tm.lane = threadIdx.x & 31;
  tm.ph = 0;
  if constexpr (NW > 1) {
    tm.wp = w;
    base = smem;
    tm.buf = smem + sums_off;
    return blockIdx.x;
  } else {
    tm.wp = 0;
    base = smem + (size_t)w * per;
    tm.buf = nullptr;
    return blockIdx.x * (blockDim.x >> 5) + w;
  }
}

__device__ __forceinline__ int jacobi_partner(int lane, int r, int n2) {
  // round-robin tournament over n2 (even) players: player n2-1 meets r,
  // the others meet (2r - lane) mod (n2-1); lanes >= n2 sit out
  const int nr = n2 - 1;
  if (lane >= n2) return lane;
  if (lane == nr) return r;
  if (lane == r) return nr;
  int p = (2 * r - lane) % nr;
  return p < 0 ? p + nr : p;
}

// --------------------------------------------------------------- prepass
// Weights of the unchanged matrix (Section 4, the recursive construction of
// the weight matrices), for both sides:
//   G_t  = qr_R([omega_b S_b^* for b in row(t)])      (k_blockweights, all
//          clusters in one launch: G_t does not depend on the father)
//   B~_t = qr_R([G_t; B~_{t+} E_t^*])                  (k_baseweights, one
//          launch per level, top-down)
// omega_b = sqrt(#T_t) / ||S_b||_F (block-relative reading).  Column side:
// S_b instead of S_b^* and col(s).  Cluster lists encode side << 30 | id.
template <int NW>
__global__ void __launch_bounds__(32 * kTW) k_blockweights(MatView M, const int32_t* __restrict__ list, int n,
                                                     BlockLists BL, BaseWeights BW, int* err) {
  extern __shared__ double smem[];
  Team<NW> tm;
  double* R;
  const int idx = team_task<NW>(tm, R, smem, fold_doubles(1), fold_doubles(1));
  if (idx >= n) return;
  double* vb = R + 32 * kLdr;
  const int lane = tm.lane;
  constexpr int VW = Team<NW>::VW;
  const int side = list[idx] >> 30;
  const int c = list[idx] & 0x3fffffff;
  if (!pick(BW.need, side)[c]) return;
  const int k = pick(M.rank, side)[c];
  const int kcap = M.kcap;
  if (k > 32) {
    if (tm.lead() && lane == 0) flag(err, kErrCols);
    return;
  }
  zero_tile_t(R, tm);
  const double st = sqrt((double)pick(M.subtree, side)[c]);
  double x[VW][kRW];
  for (int e = pick(BL.ptr, side)[c]; e < pick(BL.ptr, side)[c + 1]; ++e) {
    const int slot = pick(BL.adm, side)[e];
    const int o = pick(BL.other, side)[slot];
    const int l = pick(M.rank, 1 - side)[o];
    const double* S = M.S + (size_t)slot * kcap * kcap;
    // ||S_b||_F (every warp of the team alike)
    double part = 0.0;
    const int scols = side == 0 ? l : k;
    const int srows = side == 0 ? k : l;
    if (lane < scols)
      for (int i = 0; i < srows; ++i) {
        const double v = S[i + lane * kcap];
        part = fma(v, v, part);
      }
    const double nrm = sqrt(warp_sum(part));
    const double om = nrm > 0.0 ? st / nrm : 0.0;
    // rows of the stack: side 0 -> S^* (l x k), side 1 -> S (l x k); l = other side's rank
#pragma unroll
    for (int v = 0; v < VW; ++v)
#pragma unroll
      for (int ii = 0; ii < kRW; ++ii) {
        const int i = kTW * ii + tm.vw(v);
        double y = 0.0;
        if (i < l && lane < k) y = side == 0 ? S[lane + i * kcap] : S[i + lane * kcap];
        x[v][ii] = om * y;
      }
    fold_t(R, vb, x, l, k, tm);
  }
  store_tile_t(pick(BW.G, side) + (size_t)c * kSlot, R, k, tm);
}

template <int NW>
__global__ void __launch_bounds__(32 * kTW) k_baseweights(MatView M, const int32_t* __restrict__ list, int n,
                                                    BaseWeights BW, int* err) {
  extern __shared__ double smem[];
  Team<NW> tm;
  double* R;
  const int idx = team_task<NW>(tm, R, smem, fold_doubles(1), fold_doubles(1));
  if (idx >= n) return;
  double* vb = R + 32 * kLdr;
  const int lane = tm.lane;
  constexpr int VW = Team<NW>::VW;
  const int side = list[idx] >> 30;
  const int c = list[idx] & 0x3fffffff;
  if (!pick(BW.need, side)[c]) return;
  const int k = pick(M.rank, side)[c];
  const int kcap = M.kcap;
  if (k > 32) {
    if (tm.lead() && lane == 0) flag(err, kErrCols);
    return;
  }
  zero_tile_t(R, tm);
  const double* G = pick(BW.G, side) + (size_t)c * kSlot;
  if (tm.lead() && lane < k)
    for (int i = 0; i <= lane; ++i) R[i + lane * kLdr] = G[i + lane * 32];
  tm.sync();
  const int f = pick(M.father, side)[c];
  if (f >= 0) {
    const int kf = pick(M.rank, side)[f];
    const double* P = pick(BW.B, side) + (size_t)f * kSlot;
    const double* E = pick(M.transfer, side) + (size_t)c * kcap * kcap;   // k x kf
    double x[VW][kRW];
#pragma unroll
    for (int v = 0; v < VW; ++v)
#pragma unroll
      for (int ii = 0; ii < kRW; ++ii) {
        const int i = kTW * ii + tm.vw(v);
        double y = 0.0;
        if (i < kf && lane < k)
          for (int q = i; q < kf; ++q) y = fma(P[i + q * 32], E[lane + q * kcap], y);
        x[v][ii] = y;
      }
    fold_t(R, vb, x, kf, k, tm);
  }
  store_tile_t(pick(BW.B, side) + (size_t)c * kSlot, R, k, tm);
}

// ------------------------------------------------------------- step 2
// Basis R-factors bottom-up: leaf qr_R((V_t, F|_t)); inner
// qr_R([R_{t1} E~_{t1}; R_{t2} E~_{t2}]) with E~ = diag(E, I_u).
template <int NW>
__global__ void __launch_bounds__(32 * kTW) k_rfactor(MatView M, const Item* __restrict__ items,
                                                const int32_t* __restrict__ list, int n, int u,
                                                const double* __restrict__ A, const double* __restrict__ B,
                                                ItemBuffers IB, int* err) {
  extern __shared__ double smem[];
  Team<NW> tm;
  double* R;
  const int idx = team_task<NW>(tm, R, smem, fold_doubles(1), fold_doubles(1));
  if (idx >= n) return;
  double* vb = R + 32 * kLdr;
  const int lane = tm.lane;
  constexpr int VW = Team<NW>::VW;
  const int id = list[idx];
  const Item it = items[id];
  if (!IB.fail[it.update]) return;
  const int side = it.side;
  const int k = it.k;
  const int K = k + u;
  if (K > 32) {
    if (tm.lead() && lane == 0) flag(err, kErrCols);
    return;
  }
  zero_tile_t(R, tm);
  double x[VW][kRW];
  if (it.flags & kItemLeaf) {
    const double* V = pick(M.leaf, side) + pick(M.leaf_off, side)[it.cluster];
    const double* F = (side == 0 ? A : B) + it.foff;
    const int m = it.size;
    for (int r0 = 0; r0 < m; r0 += kCh) {
      const int ch = min(kCh, m - r0);
#pragma unroll
      for (int v = 0; v < VW; ++v)
#pragma unroll
        for (int ii = 0; ii < kRW; ++ii) {
          const int i = kTW * ii + tm.vw(v);
          double y = 0.0;
          if (i < ch) {
            if (lane < k)
              y = V[(r0 + i) + lane * m];
            else if (lane < K)
              y = F[(it.rowoff + r0 + i) + (size_t)(lane - k) * it.ld];
          }
          x[v][ii] = y;
        }
      fold_t(R, vb, x, ch, K, tm);
    }
  } else {
    const int sons[2] = {it.son0, it.son1};
    for (int si = 0; si < 2; ++si) {
      const Item sn = items[sons[si]];
      const int ks = sn.k;
      const int Ks = ks + u;
      const double* Rs = IB.Rq + (size_t)sons[si] * kSlot;
      const double* E = pick(M.transfer, side) + (size_t)sn.cluster * M.kcap * M.kcap;   // ks x k
#pragma unroll
      for (int v = 0; v < VW; ++v)
#pragma unroll
        for (int ii = 0; ii < kRW; ++ii) {
          const int i = kTW * ii + tm.vw(v);
          double y = 0.0;
          if (i < Ks) {
            if (lane < k) {
              for (int q = 0; q < ks; ++q) y = fma(Rs[i + q * 32], E[q + lane * M.kcap], y);
            } else if (lane < K) {
              y = Rs[i + (ks + lane - k) * 32];
            }
          }
          x[v][ii] = y;
        }
      fold_t(R, vb, x, Ks, K, tm);
    }
  }
  store_tile_t(IB.Rq + (size_t)id * kSlot, R, K, tm);
}

// Norms ||R_t S~_b R_s^*||_F of the blocks inside the update (both sides
// extended), needed for omega_b.
__global__ void k_norms(MatView M, const Item* __restrict__ items, const NormTask* __restrict__ tasks,
                        int n, int u, ItemBuffers IB) {
  const int lane = threadIdx.x & 31;
  const int idx = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (idx >= n) return;
  const NormTask tk = tasks[idx];
  const Item it = items[tk.it];
  if (!IB.fail[it.update]) return;
  const Item is = items[tk.is];
  const int kt = it.k, ls = is.k;
  const int Kt = kt + u, Ks = ls + u;
  const double* S = M.S + (size_t)tk.slot * M.kcap * M.kcap;
  const double* Rt = IB.Rq + (size_t)tk.it * kSlot;
  const double* Rs = IB.Rq + (size_t)tk.is * kSlot;
  double part = 0.0;
  if (lane < Ks) {
    // T[:, lane] = S~ R_s^*[:, lane] = S~ * row `lane` of R_s
    double T[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      double v = 0.0;
      if (i < kt) {
        for (int q = 0; q < ls; ++q) v = fma(S[i + q * M.kcap], Rs[lane + q * 32], v);
      } else if (i < Kt) {
        v = Rs[lane + (ls + i - kt) * 32];
      }
      T[i] = v;
    }
    for (int p = 0; p < Kt; ++p) {
      double y = 0.0;
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (i >= p && i < Kt) y = fma(Rt[p + i * 32], T[i], y);
      part = fma(y, y, part);
    }
  }
  const double s = warp_sum(part);
  if (lane == 0) IB.norms[idx] = sqrt(s);
}

// ------------------------------------------------------------- step 3
// Weights top-down: B~_t = qr_R([omega_b R_{W,s} S~_b^* for s in row(t);
// B~_{t+} E~_t^*]) (Sections 4 and 5).  The blocks of row(t) whose other
// cluster lies outside the update contribute omega_b [S_b^*, 0]; when
// V_t is orthonormal and no block of row(t) lies inside the update their
// R-factor is the precomputed G_t.  Otherwise k_outside folds them first,
// for every such cluster task at once (it does not depend on the father).

// V_t orthonormal <=> the leading k x k block of its R-factor is diag(+-1);
// then ||Z~|_b||_F = ||R_kk S_b||_F equals ||S_b||_F for outside blocks.
__device__ __forceinline__ bool basis_orthonormal(const double* Rown, int k, int lane) {
  bool orth = true;
  if (lane < k)
    for (int i = 0; i < k; ++i) {
      const double v = Rown[i + lane * 32];
      const double want = (i == lane) ? copysign(1.0, v) : 0.0;
      if (fabs(v - want) > 64.0 * DBL_EPSILON) orth = false;
    }
  return __all_sync(kFull, orth);
}

template <int NW>
__global__ void __launch_bounds__(32 * kTW) k_outside(MatView M, const Item* __restrict__ items,
                                                const Entry* __restrict__ ents, const int32_t* __restrict__ list,
                                                int n, int u, ItemBuffers IB) {
  extern __shared__ double smem[];
  Team<NW> tm;
  double* R;
  const int idx = team_task<NW>(tm, R, smem, fold_doubles(1), fold_doubles(1));
  if (idx >= n) return;
  double* vb = R + 32 * kLdr;
  const int lane = tm.lane;
  constexpr int VW = Team<NW>::VW;
  const int id = list[idx];
  const Item it = items[id];
  if (!IB.fail[it.update]) return;
  const int side = it.side;
  const int k = it.k;
  const int kcap = M.kcap;
  const double* Rown = IB.Rq + (size_t)id * kSlot;
  const bool orth = basis_orthonormal(Rown, k, lane);   // every warp of the team alike
  const bool own = (it.flags & kItemInside) || !orth;
  if (tm.lead() && lane == 0) IB.own[id] = own ? 1 : 0;
  if (!own) return;
  zero_tile_t(R, tm);
  const double st = sqrt((double)pick(M.subtree, side)[it.cluster]);
  double x[VW][kRW];
  for (int e = it.ent_begin; e < it.ent_end; ++e) {
    const Entry en = ents[e];
    if (en.other >= 0) continue;
    const double* S = M.S + (size_t)en.slot * kcap * kcap;
    const int l = pick(M.rank, 1 - side)[en.other_cluster];
    double part = 0.0;
    if (orth) {
      // ||S_b||_F
      const int scols = side == 0 ? l : k;
      const int srows = side == 0 ? k : l;
      if (lane < scols)
        for (int i = 0; i < srows; ++i) {
          const double y = S[i + lane * kcap];
          part = fma(y, y, part);
        }
    } else if (lane < l) {
      // ||R_kk S_b||_F (side 0, S is k x l) or ||S_b R_kk^*||_F (side 1, S is l x k)
      for (int p = 0; p < k; ++p) {
        double y = 0.0;
        for (int q = p; q < k; ++q)
          y = fma(Rown[p + q * 32], side == 0 ? S[q + lane * kcap] : S[lane + q * kcap], y);
        part = fma(y, y, part);
      }
    }
    const double nrm = sqrt(warp_sum(part));
    const double om = nrm > 0.0 ? st / nrm : 0.0;
#pragma unroll
    for (int v = 0; v < VW; ++v)
#pragma unroll
      for (int ii = 0; ii < kRW; ++ii) {
        const int i = kTW * ii + tm.vw(v);
        double y = 0.0;
        if (i < l && lane < k) y = side == 0 ? S[lane + i * kcap] : S[i + lane * kcap];
        x[v][ii] = om * y;
      }
    fold_t(R, vb, x, l, k, tm);
  }
  store_tile_t(IB.Bw + (size_t)id * kSlot, R, k, tm);
}

template <int NW>
__global__ void __launch_bounds__(32 * kTW) k_weights(MatView M, const Item* __restrict__ items,
                                                const Entry* __restrict__ ents, const int32_t* __restrict__ list,
                                                int n, int u, BaseWeights BW, ItemBuffers IB, int* err) {
  extern __shared__ double smem[];
  Team<NW> tm;
  double* R;
  const int idx = team_task<NW>(tm, R, smem, fold_doubles(1), fold_doubles(1));
  if (idx >= n) return;
  double* vb = R + 32 * kLdr;
  const int lane = tm.lane;
  constexpr int VW = Team<NW>::VW;
  const int id = list[idx];
  const Item it = items[id];
  if (!IB.fail[it.update]) return;
  const int side = it.side;
  const int k = it.k;
  const int K = k + u;
  const int kcap = M.kcap;
  zero_tile_t(R, tm);
  double x[VW][kRW];
  const double st = sqrt((double)pick(M.subtree, side)[it.cluster]);
  // outside blocks: their R-factor, padded with zero columns to K
  {
    const double* G = IB.own[id] ? IB.Bw + (size_t)id * kSlot : pick(BW.G, side) + (size_t)it.cluster * kSlot;
    if (tm.lead() && lane < k)
      for (int i = 0; i <= lane; ++i) R[i + lane * kLdr] = G[i + lane * 32];
    tm.sync();
  }
  // blocks inside the update: omega_b R_{W,s} S~_b^* (K_s x K_t)
  if (it.flags & kItemInside)
    for (int e = it.ent_begin; e < it.ent_end; ++e) {
      const Entry en = ents[e];
      if (en.other < 0) continue;
      const double* S = M.S + (size_t)en.slot * kcap * kcap;
      const Item ot = items[en.other];
      const int l = ot.k;
      const int Ko = l + u;
      const double nrm = IB.norms[en.norm];
      const double om = nrm > 0.0 ? st / nrm : 0.0;
      const double* Ro = IB.Rq + (size_t)en.other * kSlot;
#pragma unroll
      for (int v = 0; v < VW; ++v)
#pragma unroll
        for (int ii = 0; ii < kRW; ++ii) {
          const int i = kTW * ii + tm.vw(v);
          double y = 0.0;
          if (i < Ko) {
            if (lane < k) {
              // side 0: (R_W,s S~^*)[i, lane] = sum_q R[i,q] S[lane,q]
              // side 1: (R_V,t S~)[i, lane]   = sum_q R[i,q] S[q,lane]
              for (int q = i; q < l; ++q)
                y = fma(Ro[i + q * 32], side == 0 ? S[lane + q * kcap] : S[q + lane * kcap], y);
            } else if (lane < K) {
              y = Ro[i + (l + lane - k) * 32];
            }
          }
          x[v][ii] = om * y;
        }
      fold_t(R, vb, x, Ko, K, tm);
    }
  // father's part
  if (it.flags & kItemRoot) {
    if (!(it.flags & kItemTreeRoot)) {
      const int f = pick(M.father, side)[it.cluster];
      const int kf = it.kf;
      const double* P = pick(BW.B, side) + (size_t)f * kSlot;
      const double* E = pick(M.transfer, side) + (size_t)it.cluster * kcap * kcap;   // k x kf
#pragma unroll
      for (int v = 0; v < VW; ++v)
#pragma unroll
        for (int ii = 0; ii < kRW; ++ii) {
          const int i = kTW * ii + tm.vw(v);
          double y = 0.0;
          if (i < kf && lane < k)
            for (int q = i; q < kf; ++q) y = fma(P[i + q * 32], E[lane + q * kcap], y);
          x[v][ii] = y;
        }
      fold_t(R, vb, x, kf, K, tm);
    }
  } else {
    const Item pt = items[it.parent];
    const int kf = pt.k;
    const int Kf = kf + u;
    const double* P = IB.Bw + (size_t)it.parent * kSlot;
    const double* E = pick(M.transfer, side) + (size_t)it.cluster * kcap * kcap;   // k x kf
#pragma unroll
    for (int v = 0; v < VW; ++v)
#pragma unroll
      for (int ii = 0; ii < kRW; ++ii) {
        const int i = kTW * ii + tm.vw(v);
        double y = 0.0;
        if (i < Kf) {
          if (lane < k) {
            for (int q = i; q < kf; ++q) y = fma(P[i + q * 32], E[lane + q * kcap], y);
          } else if (lane < K) {
            y = P[i + (kf + lane - k) * 32];
          }
        }
        x[v][ii] = y;
      }
    fold_t(R, vb, x, Kf, K, tm);
  }
  store_tile_t(IB.Bw + (size_t)id * kSlot, R, K, tm);
  (void)err;
}

// ------------------------------------------------------------- step 4
// Truncation bottom-up: SVD of M = V^_t B~_t^* (leaf: V^_t = V~_t),
// rank by the block-relative rule sum_{i>r} sigma_i^2 <= (eps/2)^2, Q^_t
// from the leading left singular vectors, R_t = Q^_t^* V^_t; the rows of
// Q^_t become the sons' new transfer matrices (Eq. (Qt_nested)), and the
// subtree root commits E_t0 <- R_t0 [E_t0; 0] (Eqs. (Qt_condensed),
// (hatQt_condensed)).
//
// A task runs on a team (one warp, or a block of kTW).  Lane c owns column
// c.  Virtual warp w owns the rows i of the tall matrices with
// (i / 2) mod kTW = w (two of every 2 kTW, see trow), register slot (v, h) of
// a warp holding row trow(h, vw(v)); the K x K products are split by their
// output rows over the warps of the team.

// row of the tall matrices held in slot h of virtual warp w
__device__ __forceinline__ int trow(int h, int w) { return 2 * kTW * (h >> 1) + 2 * w + (h & 1); }

// One-sided (Hestenes) Jacobi on the K columns (a[v][h]: the team's rows,
// zero beyond `rows`): on return the columns are U Sigma, mutually
// orthogonal.  Round-robin pairs; within a virtual warp the two lanes of a
// pair split the rows (the lower lane the even slots, the upper the odd
// ones) and add their partial sums, and the virtual warps' sums are added
// in warp order, so every thread takes the same rotation.
template <int RW, int NW>
__device__ __forceinline__ void jacobi_t(double (&a)[Team<NW>::VW][RW], int rows, int ncol, Team<NW>& tm,
                                         unsigned long long* cnt, int* err) {
  constexpr int VW = Team<NW>::VW;
  const int lane = tm.lane;
  const int n2 = ncol + (ncol & 1);
  const int nr = n2 - 1;
  const double tol2 = (16.0 * DBL_EPSILON) * (16.0 * DBL_EPSILON);
  unsigned long long pairs = 0, rots = 0;
  bool converged = (ncol < 2);
  for (int sweep = 0; sweep < kMaxSweeps && !converged; ++sweep) {
    int any = 0;
    for (int r = 0; r < nr; ++r) {
      const int p = jacobi_partner(lane, r, n2);
      const bool lo = lane < p;
      double al[VW], be[VW], ga[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        const int w = tm.vw(v);
        double x1 = 0.0, y1 = 0.0, g1 = 0.0;
#pragma unroll
        for (int h = 0; h < RW / 2; ++h)
          if (trow(2 * h, w) < rows) {
            const double r0 = a[v][2 * h], r1 = a[v][2 * h + 1];
            const double got = __shfl_sync(kFull, lo ? r1 : r0, p);
            const double xx = lo ? r0 : got;
            const double yy = lo ? got : r1;
            x1 = fma(xx, xx, x1);
            y1 = fma(yy, yy, y1);
            g1 = fma(xx, yy, g1);
          }
        x1 += __shfl_sync(kFull, x1, p);
        y1 += __shfl_sync(kFull, y1, p);
        g1 += __shfl_sync(kFull, g1, p);
        al[v] = x1;
        be[v] = y1;
        ga[v] = g1;
      }
      double AL, BE, GA;
      tm.sum3(al, be, ga, AL, BE, GA);
      const bool active = lane < n2 && p != lane;
      // rotate when |gamma| > tol sqrt(alpha beta); the columns are scaled
      // to max |entry| < 1, so the squares neither overflow nor matter when
      // they underflow
      const bool rot = active && GA * GA > tol2 * (AL * BE);
      double c = 1.0, s = 0.0;
      if (rot) {
        // t = tan(theta) of the rotation that makes the pair orthogonal:
        // t = gamma / (d + sign(d) sqrt(d^2 + gamma^2)), d = (beta - alpha) / 2
        const double d = 0.5 * (BE - AL);
        const double t = GA / (d + copysign(sqrt(fma(d, d, GA * GA)), d));
        c = rsqrt(fma(t, t, 1.0));
        s = c * t;
      }
      if (__any_sync(kFull, rot)) {
#pragma unroll
        for (int v = 0; v < VW; ++v)
#pragma unroll
          for (int h = 0; h < RW; ++h)
            if (trow(h, tm.vw(v)) < rows) {
              const double o = __shfl_sync(kFull, a[v][h], p);
              if (rot) a[v][h] = lo ? fma(c, a[v][h], -s * o) : fma(s, o, c * a[v][h]);
            }
      }
      if (active && lo) {
        pairs += 1;
        rots += rot ? 1 : 0;
      }
      any |= rot ? 1 : 0;
    }
    converged = !__any_sync(kFull, any);
  }
  if (!converged && tm.lead() && lane == 0) flag(err, kErrJacobi);
  // per-item counters (pairs checked, rotations) for the flop statistics
  if (tm.lead()) {
    unsigned long long ps = pairs, rs = rots;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ps += __shfl_xor_sync(kFull, ps, o);
      rs += __shfl_xor_sync(kFull, rs, o);
    }
    if (lane == 0 && cnt) {
      cnt[0] = ps;
      cnt[1] = rs;
    }
  }
}

// Float32 one-sided Jacobi used as a preconditioner: rotates the float copy
// af of the columns until they are orthogonal to float accuracy and
// accumulates the rotations in V (vf[v][jj] = V[kTW jj + vw(v)][lane]), so
// that M V has nearly orthogonal columns.
template <int RW, int NW>
__device__ __forceinline__ void jacobi32_t(float (&af)[Team<NW>::VW][RW], float (&vf)[Team<NW>::VW][32 / kTW], int rows,
                                           int ncol, Team<NW>& tm) {
  constexpr int VW = Team<NW>::VW;
  const int lane = tm.lane;
  const int n2 = ncol + (ncol & 1);
  const int nr = n2 - 1;
  const float tol = 1.0e-6f;
  if (ncol < 2) return;
  for (int sweep = 0; sweep < 12; ++sweep) {
    int any = 0;
    for (int r = 0; r < nr; ++r) {
      const int p = jacobi_partner(lane, r, n2);
      const bool lo = lane < p;
      float al[VW], be[VW], ga[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        float x1 = 0.f, y1 = 0.f, g1 = 0.f;
#pragma unroll
        for (int h = 0; h < RW; ++h)
          if (trow(h, tm.vw(v)) < rows) {
            const float o = __shfl_sync(kFull, af[v][h], p);
            const float xx = lo ? af[v][h] : o;
            const float yy = lo ? o : af[v][h];
            x1 = fmaf(xx, xx, x1);
            y1 = fmaf(yy, yy, y1);
            g1 = fmaf(xx, yy, g1);
          }
        al[v] = x1;
        be[v] = y1;
        ga[v] = g1;
      }
      float AL, BE, GA;
      tm.sum3(al, be, ga, AL, BE, GA);
      const bool active = lane < n2 && p != lane;
      const bool rot = active && AL > 0.f && BE > 0.f && fabsf(GA) > tol * sqrtf(AL) * sqrtf(BE);
      float c = 1.f, s = 0.f;
      if (rot) {
        const float zeta = (BE - AL) / (2.f * GA);
        const float t = copysignf(1.f, zeta) / (fabsf(zeta) + hypotf(1.f, zeta));
        c = rsqrtf(fmaf(t, t, 1.f));
        s = c * t;
      }
      if (__any_sync(kFull, rot)) {
#pragma unroll
        for (int v = 0; v < VW; ++v) {
#pragma unroll
          for (int h = 0; h < RW; ++h)
            if (trow(h, tm.vw(v)) < rows) {
              const float o = __shfl_sync(kFull, af[v][h], p);
              if (rot) af[v][h] = lo ? fmaf(c, af[v][h], -s * o) : fmaf(s, o, c * af[v][h]);
            }
#pragma unroll
          for (int jj = 0; jj < 32 / kTW; ++jj)
            if (kTW * jj + tm.vw(v) < ncol) {
              const float o = __shfl_sync(kFull, vf[v][jj], p);
              if (rot) vf[v][jj] = lo ? fmaf(c, vf[v][jj], -s * o) : fmaf(s, o, c * vf[v][jj]);
            }
        }
      }
      any |= rot ? 1 : 0;
    }
    if (!__any_sync(kFull, any)) break;
  }
}

// Two Newton-Schulz steps V <- V (3I - V^* V) / 2 in float64 on V (ncol x
// ncol in Vs, ld ldg), with G = V^* V in Gs: turns the float32-accurate
// rotation product into an orthogonal matrix to float64 accuracy.  The
// warps of the team split the rows of G and of the new V.
template <int NW>
__device__ __forceinline__ void orthonormalize_t(double* Vs, double* Gs, int ncol, int ldg, const Team<NW>& tm) {
  const int lane = tm.lane;
  for (int step = 0; step < 2; ++step) {
    if (lane < ncol)
      for (int i = tm.wp; i < ncol; i += NW) {
        double x = 0.0;
        for (int j = 0; j < ncol; ++j) x = fma(Vs[j + i * ldg], Vs[j + lane * ldg], x);
        Gs[i + lane * ldg] = x;
      }
    tm.sync();
    double nv[32 / NW];
#pragma unroll
    for (int jj = 0; jj < 32 / NW; ++jj) {
      const int j = jj * NW + tm.wp;
      double x = 0.0;
      if (j < ncol && lane < ncol)
        for (int i = 0; i < ncol; ++i) x = fma(Vs[j + i * ldg], Gs[i + lane * ldg], x);
      nv[jj] = (j < ncol && lane < ncol) ? fma(1.5, Vs[j + lane * ldg], -0.5 * x) : 0.0;
    }
    tm.sync();   // every read of V is done
#pragma unroll
    for (int jj = 0; jj < 32 / NW; ++jj) {
      const int j = jj * NW + tm.wp;
      if (j < ncol && lane < ncol) Vs[j + lane * ldg] = nv[jj];
    }
    tm.sync();
  }
}

// ---------------------------------------------- certified full-rank path
// When every singular value of the weighted matrix M exceeds the
// truncation threshold, the rank rule keeps all of range(M) and any
// orthonormal basis of range(M) gives the same projection Q Q^* V^ as the
// singular vectors (Eq. (Qt_condensed)).  The certificate is the Cholesky
// factorisation of M^* M - (tau + delta) I succeeding, tau = (eps/2)^2 and
// delta a bound on the rounding of the Gram matrix and of the
// factorisation; the basis then comes from Cholesky-QR passes.  X is the
// tall matrix in shared memory (ld ldx), xr[v][h] the team's rows of column
// lane.

// G = X^* X (K x K, ld ldg): the warps split the rows j of G, each entry one
// sum over the rows in order.
template <int NW>
__device__ __forceinline__ void gram_t(const double* X, int ldx, int rows, int K, double* Gs, int ldg,
                                       const Team<NW>& tm) {
  const int lane = tm.lane;
  if (lane < K)
    for (int j = tm.wp; j < K; j += NW) {
      double g = 0.0;
      for (int i = 0; i < rows; ++i) g = fma(X[i + j * ldx], X[i + lane * ldx], g);
      Gs[j + lane * ldg] = g;
    }
  tm.sync();
}

// In-place Cholesky factorisation G - shift I = L L^* of the lower triangle
// of Gs (ld ldg): lane i owns row i, the warps split the columns of the
// trailing update.  Returns false (on every thread alike) when a pivot is
// not positive.
template <int NW>
__device__ __forceinline__ bool chol_t(double* Gs, int K, double shift, int ldg, const Team<NW>& tm) {
  const int lane = tm.lane;
  if (tm.lead() && lane < K) Gs[lane + lane * ldg] -= shift;
  tm.sync();
  for (int j = 0; j < K; ++j) {
    const double d = Gs[j + j * ldg];
    if (!(d > 0.0)) return false;
    const double ljj = sqrt(d);
    const double inv = 1.0 / ljj;
    tm.sync();   // every thread has read the pivot
    if (tm.lead()) {
      if (lane == j) Gs[j + j * ldg] = ljj;
      if (lane > j && lane < K) Gs[lane + j * ldg] *= inv;
    }
    tm.sync();
    if (lane > j && lane < K) {
      const double lij = Gs[lane + j * ldg];
      for (int k = j + 1 + ((tm.wp - j - 1) & (NW - 1)); k <= lane; k += NW)
        Gs[lane + k * ldg] = fma(-lij, Gs[k + j * ldg], Gs[lane + k * ldg]);
    }
    tm.sync();
  }
  return true;
}

// Xs = L^{-1} (lower triangular, ld ldg) for the Cholesky factor in Ls, one
// row after the other: X[i][c] = -(sum_{c<=p<i} L[i][p] X[p][c]) / L[i][i],
// lane c, the sum split over the virtual warps by p mod 4.  dinv receives
// the reciprocal diagonal.
template <int NW>
__device__ __forceinline__ void trinv_t(const double* Ls, double* Xs, double* dinv, int K, int ldg, Team<NW>& tm) {
  constexpr int VW = Team<NW>::VW;
  const int lane = tm.lane;
  if (tm.lead() && lane < K) {
    const double di = 1.0 / Ls[lane + lane * ldg];
    dinv[lane] = di;
    Xs[lane + lane * ldg] = di;
  }
  tm.sync();
  for (int i = 1; i < K; ++i) {
    double t[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const int w = tm.vw(v);
      double x = 0.0;
      if (lane < i)
        for (int p = lane + ((w - lane) & (kTW - 1)); p < i; p += kTW) x = fma(Ls[i + p * ldg], Xs[p + lane * ldg], x);
      t[v] = x;
    }
    const double ts = tm.sum1(t);
    if (tm.lead() && lane < i) Xs[i + lane * ldg] = -ts * dinv[i];
    tm.sync();
  }
}

// X <- X L^{-*} for the Cholesky factor L in Gs; xr receives the new rows
// of the team.
template <int RW, int NW>
__device__ __forceinline__ void apply_inverse_t(double* X, int ldx, double (&xr)[Team<NW>::VW][RW], int rows, int K,
                                                const double* Gs, double* Xs, double* dinv, int ldg, Team<NW>& tm) {
  constexpr int VW = Team<NW>::VW;
  const int lane = tm.lane;
  trinv_t(Gs, Xs, dinv, K, ldg, tm);
#pragma unroll
  for (int v = 0; v < VW; ++v)
#pragma unroll
    for (int h = 0; h < RW; ++h) xr[v][h] = 0.0;
  if (lane < K)
    for (int j = 0; j <= lane; ++j) {
      const double x = Xs[lane + j * ldg];
#pragma unroll
      for (int v = 0; v < VW; ++v)
#pragma unroll
        for (int h = 0; h < RW; ++h) {
          const int i = trow(h, tm.vw(v));
          if (i < rows) xr[v][h] = fma(X[i + j * ldx], x, xr[v][h]);
        }
    }
  __syncwarp();   // the warp's rows are read before they are written
  if (lane < K)
#pragma unroll
    for (int v = 0; v < VW; ++v)
#pragma unroll
      for (int h = 0; h < RW; ++h) {
        const int i = trow(h, tm.vw(v));
        if (i < rows) X[i + lane * ldx] = xr[v][h];
      }
  tm.sync();
}

// One Cholesky-QR pass: G = X^* X = L L^*, X <- X L^{-*}.  False if the
// factorisation breaks down.
template <int RW, int NW>
__device__ __forceinline__ bool cholqr_t(double* X, int ldx, double (&xr)[Team<NW>::VW][RW], int rows, int K,
                                         double* Gs, double* Xs, double* dinv, int ldg, Team<NW>& tm) {
  gram_t(X, ldx, rows, K, Gs, ldg, tm);
  if (!chol_t(Gs, K, 0.0, ldg, tm)) return false;
  apply_inverse_t<RW, NW>(X, ldx, xr, rows, K, Gs, Xs, dinv, ldg, tm);
  return true;
}

// Second orthogonalisation of X when it is already orthonormal to within
// 1e-7: with G = X^* X, X <- X (3I - G) / 2 leaves an orthogonality error of
// order |G - I|^2.  Returns false, leaving X unchanged, when |G - I| is
// larger.
template <int RW, int NW>
__device__ __forceinline__ bool polish_t(double* X, int ldx, double (&xr)[Team<NW>::VW][RW], int rows, int K,
                                         double* Gs, int ldg, const Team<NW>& tm) {
  constexpr int VW = Team<NW>::VW;
  const int lane = tm.lane;
  gram_t(X, ldx, rows, K, Gs, ldg, tm);
  double dev = 0.0;   // every warp reads all of G: the same maximum everywhere
  if (lane < K)
    for (int j = 0; j < K; ++j) dev = fmax(dev, fabs(Gs[j + lane * ldg] - (j == lane ? 1.0 : 0.0)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dev = fmax(dev, __shfl_xor_sync(kFull, dev, o));
  if (!(dev < 1e-7)) return false;
  // column c: 1.5 x_c - 0.5 sum_j x_j G[j][c]
  if (lane < K) {
#pragma unroll
    for (int v = 0; v < VW; ++v)
#pragma unroll
      for (int h = 0; h < RW; ++h) xr[v][h] *= 1.5;
    for (int j = 0; j < K; ++j) {
      const double g = -0.5 * Gs[j + lane * ldg];
#pragma unroll
      for (int v = 0; v < VW; ++v)
#pragma unroll
        for (int h = 0; h < RW; ++h) {
          const int i = trow(h, tm.vw(v));
          if (i < rows) xr[v][h] = fma(X[i + j * ldx], g, xr[v][h]);
        }
    }
  }
  __syncwarp();
  if (lane < K)
#pragma unroll
    for (int v = 0; v < VW; ++v)
#pragma unroll
      for (int h = 0; h < RW; ++h) {
        const int i = trow(h, tm.vw(v));
        if (i < rows) X[i + lane * ldx] = xr[v][h];
      }
  tm.sync();
  return true;
}

// Shared memory of one truncation task (doubles): V^ and Q (ld MR + 1, kl
// columns each), two K x K tiles (ld ldg), 32 reciprocal pivots and, for a
// kTW-warp team, the sum buffers.
__host__ __device__ constexpr int trunc_ldg(int kl) { return (kl + 1) | 1; }
__host__ __device__ constexpr size_t trunc_doubles(int mr, int kl, int nw) {
  return 2 * (size_t)(mr + 1) * kl + 2 * (size_t)kl * trunc_ldg(kl) + 32 + (nw > 1 ? 2 * 96 * kTW : 0);
}

template <int MR, int NW>
__global__ void __launch_bounds__(32 * kTW) k_truncate(MatView M, const Item* __restrict__ items,
                                                 const int32_t* __restrict__ list, int n, int u, int kl, double eps,
                                                 const double* __restrict__ A, const double* __restrict__ B,
                                                 ItemBuffers IB, int* err, int cap) {
  constexpr int RW = MR / kTW;   // rows per virtual warp
  constexpr int LQ = MR + 1;     // leading dimension of V^ and Q in shared memory
  constexpr int VW = Team<NW>::VW;
  extern __shared__ double smem[];
  const int ldg = trunc_ldg(kl);
  const int per = (int)trunc_doubles(MR, kl, 1);
  Team<NW> tm;
  double* Vh;
  const int idx = team_task<NW>(tm, Vh, smem, per, per);
  if (idx >= n) return;
  const int lane = tm.lane;
  double* Qs = Vh + LQ * kl;
  double* Gs = Qs + LQ * kl;      // K x K Gram / Cholesky factor
  double* Xs = Gs + kl * ldg;     // K x K inverse factor / rotations V
  double* dinv = Xs + kl * ldg;   // 32 reciprocal pivots
  const int id = list[idx];
  const Item it = items[id];
  if (!IB.fail[it.update]) return;
  const int side = it.side;
  const int k = it.k;
  const int K = k + u;
  const int kcap = M.kcap;
  if (K > kl) {
    if (tm.lead() && lane == 0) flag(err, kErrCols);
    return;
  }
  int rows = 0;
  int r1 = 0, r2 = 0;
  if (it.flags & kItemLeaf) {
    rows = it.size;
  } else {
    r1 = IB.rank[it.son0];
    r2 = IB.rank[it.son1];
    rows = r1 + r2;
  }
  if (rows > MR) {
    if (tm.lead() && lane == 0) flag(err, kErrRows);
    return;
  }
  // V^_t into shared memory, one column per lane
  if (it.flags & kItemLeaf) {
    const double* V = pick(M.leaf, side) + pick(M.leaf_off, side)[it.cluster];
    const double* F = (side == 0 ? A : B) + it.foff;
    if (lane < K)
      for (int i = tm.wp; i < rows; i += NW)
        Vh[i + lane * LQ] = lane < k ? V[i + lane * rows] : F[(it.rowoff + i) + (size_t)(lane - k) * it.ld];
  } else {
    for (int si = 0; si < 2; ++si) {
      const int sid = si == 0 ? it.son0 : it.son1;
      const Item sn = items[sid];
      const int ks = sn.k;
      const int rs = si == 0 ? r1 : r2;
      const int row0 = si == 0 ? 0 : r1;
      const double* Rt = IB.Rt + (size_t)sid * kSlot;
      const double* E = pick(M.transfer, side) + (size_t)sn.cluster * kcap * kcap;   // ks x k
      if (lane < K)
        for (int p = tm.wp; p < rs; p += NW) {
          double y = 0.0;
          if (lane < k) {
            for (int q = 0; q < ks; ++q) y = fma(Rt[p + q * 32], E[q + lane * kcap], y);
          } else {
            y = Rt[p + (ks + lane - k) * 32];
          }
          Vh[row0 + p + lane * LQ] = y;
        }
    }
  }
  tm.sync();
  // M = V^ B~^*, column `lane` = V^ * row `lane` of B~, scaled by a power
  // of two (exact) so that max |M| lies in [1/2, 1): the squared sums of
  // the Jacobi test cannot overflow and the float copy keeps its range;
  // singular values are unscaled exactly below.
  const double* Bw = IB.Bw + (size_t)id * kSlot;
  double a[VW][RW];
  int ex = 0;
  auto form_m = [&]() {
#pragma unroll
    for (int v = 0; v < VW; ++v)
#pragma unroll
      for (int h = 0; h < RW; ++h) a[v][h] = 0.0;
    if (lane < K)
      for (int q = lane; q < K; ++q) {   // B~ is upper triangular: B~[lane, q] = 0 for q < lane
        const double bq = Bw[lane + q * 32];
#pragma unroll
        for (int v = 0; v < VW; ++v)
#pragma unroll
          for (int h = 0; h < RW; ++h) {
            const int i = trow(h, tm.vw(v));
            if (i < rows) a[v][h] = fma(Vh[i + q * LQ], bq, a[v][h]);
          }
      }
    double mx = 0.0;
#pragma unroll
    for (int v = 0; v < VW; ++v)
#pragma unroll
      for (int h = 0; h < RW; ++h) mx = fmax(mx, fabs(a[v][h]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
    mx = tm.max1(mx);
    ex = 0;
    if (mx > 0.0) frexp(mx, &ex);
#pragma unroll
    for (int v = 0; v < VW; ++v)
#pragma unroll
      for (int h = 0; h < RW; ++h) a[v][h] = ldexp(a[v][h], -ex);
  };
  auto store_rows = [&]() {
    if (lane < K)
#pragma unroll
      for (int v = 0; v < VW; ++v)
#pragma unroll
        for (int h = 0; h < RW; ++h) {
          const int i = trow(h, tm.vw(v));
          if (i < rows) Qs[i + lane * LQ] = a[v][h];
        }
    tm.sync();
  };
  form_m();
  const double thr = 0.25 * eps * eps;
  unsigned long long* cnt = IB.jac + 4 * (size_t)id;
  // certified full-rank path: M^* M - (tau + delta) I positive definite
  bool certified = false;
  if (rows >= K && K >= 1 && (cap <= 0 || K <= cap)) {   // (a rank cap below K truncates)
    store_rows();
    gram_t(Qs, LQ, rows, K, Gs, ldg, tm);
    double trace = 0.0;
    for (int j = 0; j < K; ++j) trace += Gs[j + j * ldg];
    const double tau = ldexp(thr, -2 * ex);
    const double delta = 4.0 * (double)(rows + K * K) * DBL_EPSILON * trace;
    if (chol_t(Gs, K, tau + delta, ldg, tm)) {
      // The certificate's factor L (L L^* = M^* M - (tau + delta) I) is the
      // first Cholesky-QR pass: M L^{-*} deviates from orthonormality only
      // by (tau + delta) |(L L^*)^{-1}|; a polish (or a second full pass)
      // removes the rest.
      apply_inverse_t<RW, NW>(Qs, LQ, a, rows, K, Gs, Xs, dinv, ldg, tm);
      certified = polish_t<RW, NW>(Qs, LQ, a, rows, K, Gs, ldg, tm) ||
                  (cholqr_t<RW, NW>(Qs, LQ, a, rows, K, Gs, Xs, dinv, ldg, tm) &&
                   polish_t<RW, NW>(Qs, LQ, a, rows, K, Gs, ldg, tm));
      if (!certified) form_m();   // a factorisation broke down after the certificate
    }
  }
  int r = 0;
  if (certified) {
    r = K;   // Qs holds an orthonormal basis of range(M)
    if (tm.lead() && lane == 0 && cnt) {
      cnt[0] = 0;
      cnt[1] = 0;
      cnt[2] = 1;
    }
  } else {
    // Float32 preconditioning: rotate a float copy of M to orthogonal
    // columns and keep the rotations V; V is made orthogonal in float64 and
    // M <- M V, which leaves the left singular vectors and singular values
    // of M unchanged and hands the float64 Jacobi nearly orthogonal columns.
    if (K >= 2 && rows > 0) {
      store_rows();
      float af[VW][RW];
      float vf[VW][32 / kTW];
#pragma unroll
      for (int v = 0; v < VW; ++v) {
#pragma unroll
        for (int h = 0; h < RW; ++h) af[v][h] = (float)a[v][h];
#pragma unroll
        for (int jj = 0; jj < 32 / kTW; ++jj) vf[v][jj] = (kTW * jj + tm.vw(v) == lane) ? 1.f : 0.f;
      }
      jacobi32_t<RW, NW>(af, vf, rows, K, tm);
#pragma unroll
      for (int v = 0; v < VW; ++v)
#pragma unroll
        for (int jj = 0; jj < 32 / kTW; ++jj) {
          const int j = kTW * jj + tm.vw(v);
          if (j < K && lane < K) Xs[j + lane * ldg] = (double)vf[v][jj];
        }
      tm.sync();
      orthonormalize_t(Xs, Gs, K, ldg, tm);
#pragma unroll
      for (int v = 0; v < VW; ++v)
#pragma unroll
        for (int h = 0; h < RW; ++h) a[v][h] = 0.0;
      if (lane < K)
        for (int j = 0; j < K; ++j) {
          const double vj = Xs[j + lane * ldg];
#pragma unroll
          for (int v = 0; v < VW; ++v)
#pragma unroll
            for (int h = 0; h < RW; ++h) {
              const int i = trow(h, tm.vw(v));
              if (i < rows) a[v][h] = fma(Qs[i + j * LQ], vj, a[v][h]);
            }
        }
    }
    jacobi_t<RW, NW>(a, rows, K, tm, cnt, err);
    if (tm.lead() && lane == 0 && cnt) cnt[2] = 0;
    // singular values, order, rank
    double s2p[VW];   // this lane's scaled column: squared norm per virtual warp
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      double x = 0.0;
      if (lane < K)
#pragma unroll
        for (int h = 0; h < RW; ++h)
          if (trow(h, tm.vw(v)) < rows) x = fma(a[v][h], a[v][h], x);
      s2p[v] = x;
    }
    const double s2c = tm.sum1(s2p);
    const double s2 = lane < K ? ldexp(s2c, 2 * ex) : -1.0;   // unscaled
    int pos = 0;
    for (int d = 0; d < 32; ++d) {
      const double o = __shfl_sync(kFull, s2, d);
      if (d < K && (o > s2 || (o == s2 && d < lane))) ++pos;
    }
    double tail = 0.0;
    for (int d = 0; d < 32; ++d) {
      const double o = __shfl_sync(kFull, s2, d);
      const int op = __shfl_sync(kFull, pos, d);
      if (d < K && op >= pos) tail += o;
    }
    // the rank rule; with the rank cap option, at most cap columns
    const bool keep = lane < K && rows > 0 && tail > thr && (cap <= 0 || pos < cap);
    r = __popc(__ballot_sync(kFull, keep));
    __syncwarp();   // the warp's rows of M are read before Q overwrites them
    if (keep) {
      const double inv = 1.0 / sqrt(s2c);
#pragma unroll
      for (int v = 0; v < VW; ++v)
#pragma unroll
        for (int h = 0; h < RW; ++h) {
          const int i = trow(h, tm.vw(v));
          if (i < rows) Qs[i + pos * LQ] = a[v][h] * inv;
        }
    }
    tm.sync();
  }
  // R_t = Q^* V^ (r x K): the warps split the rows p
  double* Rt = IB.Rt + (size_t)id * kSlot;
  if (lane < K)
    for (int p = tm.wp; p < 32; p += NW) {
      double y = 0.0;
      if (p < r)
        for (int i = 0; i < rows; ++i) y = fma(Qs[i + p * LQ], Vh[i + lane * LQ], y);
      Rt[p + lane * 32] = y;
    }
  if (tm.lead() && lane == 0) IB.rank[id] = r;
  // outputs: leaf basis or the sons' transfer matrices
  if (it.flags & kItemLeaf) {
    double* Q = IB.Q + it.qoff;
    if (lane < r)
      for (int i = tm.wp; i < rows; i += NW) Q[i + (size_t)lane * rows] = Qs[i + lane * LQ];
  } else {
    double* F1 = IB.F + (size_t)it.son0 * kSlot;
    double* F2 = IB.F + (size_t)it.son1 * kSlot;
    if (lane < r) {
      for (int p = tm.wp; p < r1; p += NW) F1[p + lane * 32] = Qs[p + lane * LQ];
      for (int p = tm.wp; p < r2; p += NW) F2[p + lane * 32] = Qs[r1 + p + lane * LQ];
    }
  }
  if ((it.flags & kItemRoot) && !(it.flags & kItemTreeRoot)) {
    // E_t0 <- R_t0 [E_t0; 0]  (r x kf)
    tm.sync();   // R_t of every warp is written
    const double* E = pick(M.transfer, side) + (size_t)it.cluster * kcap * kcap;   // k x kf
    double* Fo = IB.F + (size_t)id * kSlot;
    if (lane < it.kf)
      for (int p = tm.wp; p < r; p += NW) {
        double y = 0.0;
        for (int q = 0; q < k; ++q) y = fma(Rt[p + q * 32], E[q + lane * kcap], y);
        Fo[p + lane * 32] = y;
      }
  }
}

// ------------------------------------------------------------- step 5
// Reprojection S_b <- R_t S~_b R_s^* for every affected admissible block.
//
// Updates of the certified path have R_t = L_t^* upper triangular: the
// products run over the triangle only, with the 32 lanes spread over the
// entries of the result so that the lanes of one instruction share the
// row (left factor) or the column (right factor) and with it the length of
// the triangular sum.  Operands are staged in shared memory and the result
// leaves through it in coalesced columns.  Updates of the exact path have a
// general r_t x K_t factor and use one lane per column.
// k_reproject: 3 tiles per warp of tc columns and tc + 1 rows (at most 32 + 1)

__device__ __forceinline__ void reproject_general(const MatView& M, const Item* __restrict__ items, const Task& tk,
                                                  int u, const ItemBuffers& IB, const double* S, double* out,
                                                  int lane) {
  const int kcap = M.kcap;
  if (tk.it >= 0 && tk.is >= 0) {
    const int kt = items[tk.it].k, ls = items[tk.is].k;
    const int Kt = kt + u;
    const int rt = IB.rank[tk.it], rs = IB.rank[tk.is];
    const double* Rt = IB.Rt + (size_t)tk.it * kSlot;
    const double* Rs = IB.Rt + (size_t)tk.is * kSlot;
    if (lane < rs) {
      double T[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        double v = 0.0;
        if (i < kt) {
          for (int q = 0; q < ls; ++q) v = fma(S[i + q * kcap], Rs[lane + q * 32], v);
        } else if (i < Kt) {
          v = Rs[lane + (ls + i - kt) * 32];
        }
        T[i] = v;
      }
      for (int p = 0; p < rt; ++p) {
        double y = 0.0;
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i < Kt) y = fma(Rt[p + i * 32], T[i], y);
        out[p + lane * 32] = y;
      }
    }
  } else if (tk.it >= 0) {
    const int kt = items[tk.it].k;
    const int rt = IB.rank[tk.it];
    const double* Rt = IB.Rt + (size_t)tk.it * kSlot;
    const int ls = tk.ls;
    if (lane < ls)
      for (int p = 0; p < rt; ++p) {
        double y = 0.0;
        for (int i = 0; i < kt; ++i) y = fma(Rt[p + i * 32], S[i + lane * kcap], y);
        out[p + lane * 32] = y;
      }
  } else {
    const int ls = items[tk.is].k;
    const int rs = IB.rank[tk.is];
    const int kt = tk.kt;
    const double* Rs = IB.Rt + (size_t)tk.is * kSlot;
    if (lane < rs)
      for (int p = 0; p < kt; ++p) {
        double y = 0.0;
        for (int q = 0; q < ls; ++q) y = fma(S[p + q * kcap], Rs[lane + q * 32], y);
        out[p + lane * 32] = y;
      }
  }
}

__device__ __forceinline__ void reproject_task(const MatView& M, const Item* __restrict__ items, const Task& tk,
                                               int idx, int u, int tc, const BaseWeights& BW, const ItemBuffers& IB,
                                               double* smem, int w, int lane) {
  const int kcap = M.kcap;
  const double* S = M.S + (size_t)tk.slot * kcap * kcap;
  double* out = IB.S_out + (size_t)idx * kSlot;
  const int upd = items[tk.it >= 0 ? tk.it : tk.is].update;
  if (IB.fail[upd]) {
    reproject_general(M, items, tk, u, IB, S, out, lane);
    return;
  }
  const int rld = tc + 1;                          // tiles of at most tc rows
  double* X = smem + (size_t)w * 3 * rld * tc;      // S (k_t x l_s), later T
  double* R = X + rld * tc;                         // triangular factor
  double* O = R + rld * tc;                         // result
  int rows = 0, cols = 0;                    // size of the result
  if (tk.it >= 0 && tk.is >= 0) {
    const int kt = items[tk.it].k, ls = items[tk.is].k;
    const int Kt = kt + u, Ks = ls + u;
    rows = Kt;
    cols = Ks;
    for (int c = 0; c < ls; ++c)
      if (lane < kt) X[lane + c * rld] = S[lane + c * kcap];
    const double* Rs = IB.Rt + (size_t)tk.is * kSlot;
    for (int c = 0; c < Ks; ++c)
      if (lane <= c) R[lane + c * rld] = Rs[lane + c * 32];
    __syncwarp();
    // T = S~ R_s^* (Kt x Ks), column-major over the lanes: rows i < kt sum
    // S[i][q] R_s[j][q] over q = j..ls-1; rows i >= kt pick R_s[j][ls + i - kt]
    for (int e = lane; e < Kt * Ks; e += 32) {
      const int i = e % Kt, j = e / Kt;
      double v = 0.0;
      if (i < kt) {
        for (int q = j; q < ls; ++q) v = fma(X[i + q * rld], R[j + q * rld], v);
      } else {
        const int q = ls + i - kt;
        v = q >= j ? R[j + q * rld] : 0.0;
      }
      O[i + j * rld] = v;
    }
    __syncwarp();
    const double* Rt = IB.Rt + (size_t)tk.it * kSlot;
    for (int c = 0; c < Kt; ++c)
      if (lane <= c) R[lane + c * rld] = Rt[lane + c * 32];
    for (int c = 0; c < Ks; ++c)
      if (lane < Kt) X[lane + c * rld] = O[lane + c * rld];
    __syncwarp();
    // out = R_t T, row-major over the lanes: sum over i = p..Kt-1
    for (int e = lane; e < Kt * Ks; e += 32) {
      const int p = e / Ks, j = e % Ks;
      double v = 0.0;
      for (int i = p; i < Kt; ++i) v = fma(R[p + i * rld], X[i + j * rld], v);
      O[p + j * rld] = v;
    }
  } else if (tk.it >= 0) {
    // R_t [S_b; 0]: rows p < kt sum over i = p..kt-1, rows kt.. are zero;
    // R_t = [[I, C_t], [0, L_S^*]] for an orthonormal V_t gives [S_b; 0]
    const Item it = items[tk.it];
    const int kt = it.k, ls = tk.ls;
    rows = kt + u;
    cols = ls;
    for (int c = 0; c < ls; ++c)
      if (lane < kt) X[lane + c * rld] = S[lane + c * kcap];
    const double* Rt = IB.Rt + (size_t)tk.it * kSlot;
    for (int c = 0; c < kt; ++c)
      if (lane <= c) R[lane + c * rld] = Rt[lane + c * 32];
    __syncwarp();
    for (int e = lane; e < kt * ls; e += 32) {
      const int p = e / ls, j = e % ls;
      double v = 0.0;
      for (int i = p; i < kt; ++i) v = fma(R[p + i * rld], X[i + j * rld], v);
      O[p + j * rld] = v;
    }
    for (int c = 0; c < ls; ++c)
      if (lane >= kt && lane < rows) O[lane + c * rld] = 0.0;
  } else {
    // [S_b, 0] R_s^*: columns j < ls sum over q = j..ls-1, columns ls.. are
    // zero; [S_b, 0] for an orthonormal W_s
    const Item is = items[tk.is];
    const int kt = tk.kt, ls = is.k;
    rows = kt;
    cols = ls + u;
    for (int c = 0; c < ls; ++c)
      if (lane < kt) X[lane + c * rld] = S[lane + c * kcap];
    const double* Rs = IB.Rt + (size_t)tk.is * kSlot;
    for (int c = 0; c < ls; ++c)
      if (lane <= c) R[lane + c * rld] = Rs[lane + c * 32];
    __syncwarp();
    for (int e = lane; e < kt * ls; e += 32) {
      const int p = e % kt, j = e / kt;
      double v = 0.0;
      for (int q = j; q < ls; ++q) v = fma(X[p + q * rld], R[j + q * rld], v);
      O[p + j * rld] = v;
    }
    for (int c = ls; c < cols; ++c)
      if (lane < kt) O[lane + c * rld] = 0.0;
  }
  __syncwarp();
  for (int c = 0; c < cols; ++c)
    if (lane < rows) out[lane + c * 32] = O[lane + c * rld];
}

// The two-sided tasks (list from the host) and the one-sided tasks that
// k_onesided did not flag as copies (list built on the device), with persistent warps:
// warp g takes entries g, g + G, ... (G warps in the grid).
__global__ void k_reproject(MatView M, const Item* __restrict__ items, const Task* __restrict__ tasks,
                            const int32_t* __restrict__ two, int n_two, const int32_t* __restrict__ left,
                            const int32_t* __restrict__ n_left, int u, int tc, BaseWeights BW, ItemBuffers IB) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int G = gridDim.x * (blockDim.x >> 5);
  const int n = n_two + *n_left;
  for (int e = blockIdx.x * (blockDim.x >> 5) + w; e < n; e += G) {
    const int idx = e < n_two ? two[e] : left[e - n_two];
    const Task tk = tasks[idx];
    reproject_task(M, items, tk, idx, u, tc, BW, IB, smem, w, lane);
    __syncwarp();
  }
}

// The one-sided reprojections of certified updates with an orthonormal basis
// keep the coupling: R_t [S_b; 0] = [S_b; 0] and [S_b, 0] R_s^* = [S_b, 0],
// since R_t = [[I, C_t], [0, L_S^*]].  Such a task is flagged (IB.copy) and
// its coupling stays where it is (the packing of the result and the commit
// read it from the unchanged matrix); the other one-sided tasks go to a
// device list for k_reproject.  One thread per task.
__global__ void k_onesided(const Item* __restrict__ items, const Task* __restrict__ tasks, int n, BaseWeights BW,
                           ItemBuffers IB, int32_t* __restrict__ left, int32_t* __restrict__ n_left) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const Task tk = tasks[idx];
  int8_t copy = 0;
  if (tk.it < 0 || tk.is < 0) {
    const int side = tk.it >= 0 ? 0 : 1;
    const Item it = items[side == 0 ? tk.it : tk.is];
    if (IB.fail[it.update] || !pick(BW.orth, side)[it.cluster])
      left[atomicAdd(n_left, 1)] = idx;   // k_reproject computes it
    else
      copy = 1;
  }
  IB.copy[idx] = copy;
}

// Batched copies of column-major matrices (commit of one update); a
// descriptor without source writes zeros.
__global__ void k_copy(const CopyDesc* __restrict__ d, int n) {
  const int idx = blockIdx.x;
  if (idx >= n) return;
  const CopyDesc c = d[idx];
  for (int e = threadIdx.x; e < c.rows * c.cols; e += blockDim.x) {
    const int i = e % c.rows, j = e / c.rows;
    c.dst[i + (size_t)j * c.ldd] = c.src ? c.src[i + (size_t)j * c.lds] : 0.0;
  }
}

// Nearfield G|_b += A|_t B|_s^* for the inadmissible leaves inside b0.
__global__ void k_near_add(const NearDesc* __restrict__ d, int n, int u) {
  const int idx = blockIdx.x;
  if (idx >= n) return;
  const NearDesc c = d[idx];
  for (int e = threadIdx.x; e < c.rows * c.cols; e += blockDim.x) {
    const int i = e % c.rows, j = e / c.rows;
    double v = c.N[i + (size_t)j * c.ldn];
    for (int q = 0; q < u; ++q) v = fma(c.A[i + (size_t)q * c.lda], c.B[j + (size_t)q * c.ldb], v);
    c.N[i + (size_t)j * c.ldn] = v;
  }
}

}  // namespace

// ------------------------------------------------------------ launchers
static constexpr int kWarps = 4;

static int blocks_for(int n) { return (n + kWarps - 1) / kWarps; }

static int sm_count() {
  static std::atomic<int> cached[64];   // host threads may ask at once
  int dev = 0;
  H2_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64) {
    const int c = cached[dev].load(std::memory_order_relaxed);
    if (c) return c;
  }
  int sms = 0;
  H2_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (dev >= 0 && dev < 64) cached[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

// kTW-warp teams while a launch holds at most four tasks per SM (every
// task then has the float64 units of a whole SM, or a quarter at least);
// one warp per task beyond, where the tasks fill the SMs anyway.  Both
// forms compute the same bits.
static bool wide_teams(int n) { return n <= 4 * sm_count(); }

// Launch a fold kernel (template over the team width) for n tasks.
#define H2_LAUNCH_FOLD(kern, n, stream, ...)                                                              \
  do {                                                                                                   \
    if (wide_teams(n))                                                                                   \
      kern<kTW><<<(n), 32 * kTW, fold_doubles(kTW) * sizeof(double), (stream)>>>(__VA_ARGS__);           \
    else                                                                                                 \
      kern<1><<<blocks_for(n), 32 * kWarps, kWarps * fold_doubles(1) * sizeof(double), (stream)>>>(      \
          __VA_ARGS__);                                                                                  \
  } while (0)

// Blocks of a persistent launch: as many as stay resident on the device at
// once (at most `need`).
template <class Kern>
static int persistent_blocks(Kern kern, int threads, size_t smem, int need) {
  int dev = 0, sms = 0, per_sm = 0;
  H2_CUDA(cudaGetDevice(&dev));
  H2_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  H2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
  const int nb = sms * (per_sm > 0 ? per_sm : 1);
  return nb < need ? nb : (need > 0 ? need : 1);
}

template <int MR>
static void launch_truncate_mr(const MatView& M, const Item* items, const int32_t* list, int n, int u, int kl,
                               double eps, const double* A, const double* B, const ItemBuffers& IB, int* err,
                               int cap, cudaStream_t st) {
  static std::atomic<unsigned long long> attr4{0}, attr1{0};
  if (wide_teams(n)) {
    // one block of kTW warps per task
    smem_limit(k_truncate<MR, kTW>, trunc_doubles(MR, kMaxCols, kTW) * sizeof(double), attr4);
    k_truncate<MR, kTW><<<n, 32 * kTW, trunc_doubles(MR, kl, kTW) * sizeof(double), st>>>(M, items, list, n, u,
                                                                                           kl, eps, A, B, IB, err, cap);
  } else {
    // one warp per task, two tasks per block
    constexpr int warps = 2;
    smem_limit(k_truncate<MR, 1>, warps * trunc_doubles(MR, kMaxCols, 1) * sizeof(double), attr1);
    k_truncate<MR, 1><<<(n + warps - 1) / warps, 32 * warps, warps * trunc_doubles(MR, kl, 1) * sizeof(double),
                        st>>>(M, items, list, n, u, kl, eps, A, B, IB, err, cap);
  }
}

static void launch_truncate(const MatView& M, const Item* items, const int32_t* list, int n, int u, int kl,
                            int max_rows, double eps, const double* A, const double* B, const ItemBuffers& IB,
                            int* err, int cap, cudaStream_t st) {
  if (max_rows <= 32)
    launch_truncate_mr<32>(M, items, list, n, u, kl, eps, A, B, IB, err, cap, st);
  else if (max_rows <= 48)
    launch_truncate_mr<48>(M, items, list, n, u, kl, eps, A, B, IB, err, cap, st);
  else
    launch_truncate_mr<64>(M, items, list, n, u, kl, eps, A, B, IB, err, cap, st);
}

void run_pipeline(const Pipeline& P) {
  cudaStream_t st = P.stream;
  cudaStream_t bs = P.side ? P.side : P.stream;   // stream of the weights of the unchanged matrix
  int64_t pl[H2_PHASE_COUNT] = {};
  // phase timing events: recorded as external events while the sequence is
  // captured into a graph, so that they are real records when it runs
  const unsigned rec = P.capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  auto start = [&](int ph, cudaStream_t s) {
    if (P.events) H2_CUDA(cudaEventRecordWithFlags(P.events[2 * ph], s, rec));
  };
  auto stop = [&](int ph, cudaStream_t s) {
    if (P.events) H2_CUDA(cudaEventRecordWithFlags(P.events[2 * ph + 1], s, rec));
  };
  auto fork = [&]() {
    if (!P.side) return;
    H2_CUDA(cudaEventRecord(P.fork, st));
    H2_CUDA(cudaStreamWaitEvent(P.side, P.fork, 0));
  };
  const int L = P.levels;
  const int ni = P.lvl_ptr[L];
  const int ncl = P.cl_ptr[L];
  const bool gram = !P.exact_only;
  bool early_ran = false;
  // per-update path flags and per-cluster marks of the exact path
  if (P.n_updates > 0) H2_CUDA(cudaMemsetAsync(P.IB.fail, gram ? 0 : 1, (size_t)P.n_updates * 4, st));
  H2_CUDA(cudaMemsetAsync(P.n_left, 0, sizeof(int32_t), st));
  for (int sd = 0; sd < 2; ++sd)
    if (P.ncl[sd] > 0) H2_CUDA(cudaMemsetAsync(P.BW.need[sd], gram ? 0 : 1, (size_t)P.ncl[sd] * 4, st));
  if (gram) {
    // certified Gram path: weights of the unchanged matrix on the side
    // stream, overlapping the basis Grams and the norms
    fork();
    start(H2_PHASE_BASE_WEIGHTS, bs);
    cudaStream_t vs = bs;   // stream of the basis Grams
    if (P.side && P.side2) {
      vs = P.side2;
      H2_CUDA(cudaStreamWaitEvent(vs, P.fork, 0));
    }
    if (ncl > 0) {
      launch_gram_orth(P, vs);
      pl[H2_PHASE_BASE_WEIGHTS] += 2;
    }
    if (P.out) {
      // results that the orthonormality flags already fix go to the host
      // while the update runs
      H2_CUDA(cudaEventRecord(P.out->ready, vs));
      H2_CUDA(cudaStreamWaitEvent(P.out->stream, P.out->ready, 0));
      P.out->early(P, *P.out, P.out->stream);
      H2_CUDA(cudaEventRecord(P.out->done, P.out->stream));
      early_ran = true;
    }
    for (int l = L - 1; l >= 0; --l)
      if (P.cl_ptr[l + 1] > P.cl_ptr[l]) {
        launch_gram_vbasis_level(P, l, vs);
        ++pl[H2_PHASE_BASE_WEIGHTS];
      }
    if (vs != bs) H2_CUDA(cudaEventRecord(P.join2, vs));   // flags and V_t^* V_t (needed by the norms)
    if (ncl > 0) {
      launch_gram_base(P, bs);
      ++pl[H2_PHASE_BASE_WEIGHTS];
    }
    for (int l = 0; l < L; ++l)
      if (P.cl_ptr[l + 1] > P.cl_ptr[l]) {
        launch_gram_base_level(P, l, bs);
        ++pl[H2_PHASE_BASE_WEIGHTS];
      }
    if (vs != bs) H2_CUDA(cudaStreamWaitEvent(bs, P.join2, 0));   // the phase ends with both chains
    stop(H2_PHASE_BASE_WEIGHTS, bs);
    if (P.side) H2_CUDA(cudaEventRecord(P.join, P.side));
    start(H2_PHASE_RFACTOR, st);
    for (int l = L - 1; l >= 0; --l)
      if (P.lvl_ptr[l + 1] > P.lvl_ptr[l]) {
        pl[H2_PHASE_RFACTOR] += launch_gram_basis(P, l);
      }
    stop(H2_PHASE_RFACTOR, st);
    // the norms need the orthonormality flags only; the weights need all
    if (P.side) H2_CUDA(cudaStreamWaitEvent(st, vs != bs ? P.join2 : P.join, 0));
    start(H2_PHASE_NORMS, st);
    if (P.n_norms > 0) {
      launch_gram_norms(P);
      ++pl[H2_PHASE_NORMS];
    }
    stop(H2_PHASE_NORMS, st);
    if (P.side) H2_CUDA(cudaStreamWaitEvent(st, P.join, 0));
    start(H2_PHASE_WEIGHTS, st);
    for (int l = 0; l < L; ++l)
      if (P.lvl_ptr[l + 1] > P.lvl_ptr[l]) {
        launch_gram_weights(P, l);
        ++pl[H2_PHASE_WEIGHTS];
      }
    stop(H2_PHASE_WEIGHTS, st);
    start(H2_PHASE_TRUNCATE, st);
    if (ni > 0) {
      launch_gram_certify(P);
      pl[H2_PHASE_TRUNCATE] += 2;   // block-form and general variants
    }
    stop(H2_PHASE_TRUNCATE, st);
    start(H2_PHASE_BASES, st);
    if (ni > 0) {
      launch_gram_outputs(P);
      pl[H2_PHASE_BASES] += 2;
    }
    stop(H2_PHASE_BASES, st);
  }
  // exact path for the updates whose certificate failed (every kernel returns
  // at once for the tasks of the other updates and for unmarked clusters):
  // weights of the unchanged matrix on the side stream, overlapping step 2,
  // the norms and the outside folds of step 3
  start(H2_PHASE_EXACT, st);
  fork();
  if (ncl > 0) {
    H2_LAUNCH_FOLD(k_blockweights, ncl, bs, P.M, P.cl_list, ncl, P.BL, P.BW, P.err);
    ++pl[H2_PHASE_EXACT];
  }
  const int32_t* bl = P.bl_ptr ? P.bl_list : P.cl_list;
  const int32_t* bp = P.bl_ptr ? P.bl_ptr : P.cl_ptr;
  for (int l = 0; l < L; ++l) {
    const int n = bp[l + 1] - bp[l];
    if (!n) continue;
    H2_LAUNCH_FOLD(k_baseweights, n, bs, P.M, bl + bp[l], n, P.BW, P.err);
    ++pl[H2_PHASE_EXACT];
  }
  if (P.side) H2_CUDA(cudaEventRecord(P.join, P.side));
  for (int l = L - 1; l >= 0; --l) {
    const int n = P.lvl_ptr[l + 1] - P.lvl_ptr[l];
    if (!n) continue;
    H2_LAUNCH_FOLD(k_rfactor, n, st, P.M, P.items, P.lvl_list + P.lvl_ptr[l], n, P.u, P.A, P.B, P.IB, P.err);
    ++pl[H2_PHASE_EXACT];
  }
  if (P.n_norms > 0) {
    k_norms<<<blocks_for(P.n_norms), 32 * kWarps, 0, st>>>(P.M, P.items, P.norms, P.n_norms, P.u, P.IB);
    ++pl[H2_PHASE_EXACT];
  }
  if (ni > 0) {
    H2_LAUNCH_FOLD(k_outside, ni, st, P.M, P.items, P.ents, P.lvl_list, ni, P.u, P.IB);
    ++pl[H2_PHASE_EXACT];
  }
  if (P.side) H2_CUDA(cudaStreamWaitEvent(st, P.join, 0));
  for (int l = 0; l < L; ++l) {
    const int n = P.lvl_ptr[l + 1] - P.lvl_ptr[l];
    if (!n) continue;
    H2_LAUNCH_FOLD(k_weights, n, st, P.M, P.items, P.ents, P.lvl_list + P.lvl_ptr[l], n, P.u, P.BW, P.IB, P.err);
    ++pl[H2_PHASE_EXACT];
  }
  for (int l = L - 1; l >= 0; --l) {
    const int n = P.lvl_ptr[l + 1] - P.lvl_ptr[l];
    if (!n) continue;
    launch_truncate(P.M, P.items, P.lvl_list + P.lvl_ptr[l], n, P.u, P.kl, P.lvl_rows[l], P.eps, P.A, P.B, P.IB,
                    P.err, P.max_rank, st);
    ++pl[H2_PHASE_EXACT];
  }
  stop(H2_PHASE_EXACT, st);
  // step 5: reprojection
  start(H2_PHASE_REPROJECT, st);
  if (P.n_tasks > 0) {
    const int tc = P.kl > P.M.kcap ? P.kl : P.M.kcap;
    static std::atomic<unsigned long long> attr{0};
    smem_limit(k_reproject, (size_t)kWarps * 3 * 33 * 32 * sizeof(double), attr);
    // flag the copies, list the one-sided tasks that need products
    k_onesided<<<(P.n_tasks + 255) / 256, 256, 0, st>>>(P.items, P.tasks, P.n_tasks, P.BW, P.IB, P.left, P.n_left);
    const size_t rp_smem = (size_t)kWarps * 3 * (tc + 1) * tc * sizeof(double);
    k_reproject<<<persistent_blocks(k_reproject, 32 * kWarps, rp_smem, blocks_for(P.n_tasks)), 32 * kWarps, rp_smem,
                  st>>>(P.M, P.items, P.tasks, P.two, P.n_two, P.left, P.n_left, P.u, tc, P.BW, P.IB);
    pl[H2_PHASE_REPROJECT] += 2;
  }
  stop(H2_PHASE_REPROJECT, st);
  if (P.out) {
    if (early_ran) H2_CUDA(cudaStreamWaitEvent(st, P.out->packed, 0));
    P.out->late(P, *P.out, st, early_ran);
    if (early_ran) H2_CUDA(cudaStreamWaitEvent(st, P.out->done, 0));
  }
  H2_CUDA(cudaGetLastError());
  if (P.phase_launches)
    for (int ph = 0; ph < H2_PHASE_COUNT; ++ph) P.phase_launches[ph] = pl[ph];
}

void launch_copy(const CopyDesc* d, int n, cudaStream_t st) {
  if (n <= 0) return;
  k_copy<<<n, 128, 0, st>>>(d, n);
}

void launch_near_add(const NearDesc* d, int n, int u, cudaStream_t st) {
  if (n <= 0) return;
  k_near_add<<<n, 128, 0, st>>>(d, n, u);
}

}  // namespace h2
