// Allocation-free variant of the single in-place local low-rank update.
//
// Who needs it: callers that must not allocate device memory while they
// run -- code running under a fixed device-memory budget handed out once at
// start-up (a cudaMalloc in the middle of the run could fail or push another
// part of the program out of its share), or hosts whose device allocator is
// owned by another runtime (a framework's caching allocator that has already
// reserved the free memory).  For them h2_lowrank_update_noalloc
// performs the same update as h2_lowrank_update (same kernels, same results)
// but takes every piece of device scratch (task lists, per-cluster R-factor,
// weight and basis-change tiles, the weights of the unchanged matrix, copy
// descriptors) from one fixed array in this file, and plans on the host in
// fixed static buffers.  It never calls cudaMalloc/cudaFree or any routine
// that allocates device memory, and it never grows the matrix storage.
//
// The array lives for the whole process on every GPU that loads the
// library.  In host code its name is only a stand-in, so its device address
// is fetched with cudaGetSymbolAddress the first time the entry point runs
// on a device (with that device current); that first call therefore has to
// happen before any stream capture.  Every call shares the array (and the
// static host planning buffers): calls whose GPU work overlapped would race
// on it, so each call holds a library-wide lock and waits for its own GPU
// work (it synchronizes the context's stream) before it returns.  The array
// keeps the last call's contents; no part of it has to start at zero: each
// kernel writes every value a later kernel reads.  The cached device address
// belongs to the device's primary context: a caller that destroys that
// context (cudaDeviceReset) must not call this entry point afterwards.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "h2_internal.h"
#include "update_kernels.h"

namespace h2 {
namespace {

// Limits of the fixed scratch (per call).
constexpr int kNaClusters = 512;     // clusters per side of the matrix
constexpr int kNaItems = 256;        // cluster tasks of the update (both sides)
constexpr int kNaEntries = 4096;     // blocks in the weight stacks
constexpr int kNaTasks = 2048;       // couplings to reproject
constexpr int kNaNorms = 256;        // blocks inside the update
constexpr int kNaNear = 1024;        // nearfield leaves inside the block
constexpr int64_t kNaQ = 262144;     // doubles of new leaf bases
constexpr int kNaLevels = 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte layout of the scratch array.
constexpr size_t kOffG = 0;                                                    // G tiles, 2 sides
constexpr size_t kOffB = kOffG + align256(2ull * kNaClusters * kSlot * 8);     // B~ tiles, 2 sides
constexpr size_t kOffRq = kOffB + align256(2ull * kNaClusters * kSlot * 8);
constexpr size_t kOffBw = kOffRq + align256((size_t)kNaItems * kSlot * 8);
constexpr size_t kOffRt = kOffBw + align256((size_t)kNaItems * kSlot * 8);
constexpr size_t kOffF = kOffRt + align256((size_t)kNaItems * kSlot * 8);
constexpr size_t kOffQ = kOffF + align256((size_t)kNaItems * kSlot * 8);
constexpr size_t kOffS = kOffQ + align256((size_t)kNaQ * 8);
constexpr size_t kOffRank = kOffS + align256((size_t)kNaTasks * kSlot * 8);
constexpr size_t kOffOwn = kOffRank + align256((size_t)kNaItems * 4);
constexpr size_t kOffNorm = kOffOwn + align256((size_t)kNaItems * 4);
constexpr size_t kOffJac = kOffNorm + align256((size_t)kNaNorms * 8);
constexpr size_t kOffItems = kOffJac + align256((size_t)kNaItems * 32);
constexpr size_t kOffEnts = kOffItems + align256((size_t)kNaItems * sizeof(Item));
constexpr size_t kOffTasks = kOffEnts + align256((size_t)kNaEntries * sizeof(Entry));
constexpr size_t kOffNT = kOffTasks + align256((size_t)kNaTasks * sizeof(Task));
constexpr size_t kOffLvl = kOffNT + align256((size_t)kNaNorms * sizeof(NormTask));
constexpr size_t kOffCl = kOffLvl + align256((size_t)kNaItems * 4);
constexpr size_t kOffCopy = kOffCl + align256(2ull * kNaClusters * 4);
constexpr size_t kOffNear = kOffCopy + align256((size_t)(2 * kNaItems + kNaTasks) * sizeof(CopyDesc));
constexpr size_t kOffNeed = kOffNear + align256((size_t)kNaNear * sizeof(NearDesc));    // 2 sides
constexpr size_t kOffFail = kOffNeed + align256(2ull * kNaClusters * 4);
constexpr size_t kOffOrth = kOffFail + align256(4);                                       // 2 sides
constexpr size_t kOffTwo = kOffOrth + align256(2ull * kNaClusters * 4);
constexpr size_t kOffLeft = kOffTwo + align256((size_t)kNaTasks * 4);
constexpr size_t kOffNLeft = kOffLeft + align256((size_t)kNaTasks * 4);
constexpr size_t kOffCopyFlag = kOffNLeft + align256(4);
constexpr size_t kScratchBytes = kOffCopyFlag + align256((size_t)kNaTasks);
// The Gram matrices V_t^* V_t of the unchanged bases (2 sides x 512 slots)
// live in the coupling-output region: they are dead before the
// reprojection writes its results there.
static_assert(2ull * kNaClusters * kSlot * 8 <= (size_t)kNaTasks * kSlot * 8, "basis Grams exceed their region");
static_assert(kScratchBytes <= (48u << 20), "scratch above its stated 48 MiB");

static __device__ __align__(256) unsigned char h2_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
unsigned char* g_scratch[kMaxDevices] = {};
std::mutex g_lock;

// Host-side plan in static storage.
struct HostPlan {
  Item items[kNaItems];
  Entry ents[kNaEntries];
  Task tasks[kNaTasks];
  NormTask norms[kNaNorms];
  int32_t lvl_list[kNaItems];
  int32_t lvl_ptr[kNaLevels + 1];
  int32_t lvl_leaves[kNaLevels];
  int32_t lvl_rows[kNaLevels];
  int32_t cl_list[2 * kNaClusters];
  int32_t cl_ptr[kNaLevels + 1];
  int32_t item_of[2][kNaClusters];
  int32_t stack[kNaClusters];
  int32_t sub[2][kNaClusters];
  int32_t nsub[2];
  int32_t rank[kNaItems];
  int8_t copy[kNaTasks];
  int32_t two[kNaTasks];
  int n_two;
  CopyDesc copies[2 * kNaItems + kNaTasks];
  NearDesc nears[kNaNear];
  int32_t bstack[4 * kNaNear + 64];
  int n_items, n_ents, n_tasks, n_norms;
  int64_t qlen;
  int kl;
};
HostPlan g_plan;
char g_msg[512];

h2_status fail(h2_status code, const char* fmt, long long a = 0, long long b = 0) {
  std::snprintf(g_msg, sizeof(g_msg), fmt, a, b);
  return code;
}

#define NA_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      std::snprintf(g_msg, sizeof(g_msg), "%s: %s", #call, cudaGetErrorString(e_));         \
      return H2_ECUDA;                                                                       \
    }                                                                                        \
  } while (0)

h2_status scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return fail(H2_EINVAL, "device id %lld out of range", device);
  if (!g_scratch[device]) {
    void* p = nullptr;
    NA_CUDA(cudaGetSymbolAddress(&p, h2_noalloc_scratch));
    g_scratch[device] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch[device];
  return H2_OK;
}

const ClusterTree& tree(const h2_matrix* Z, int side) { return side == 0 ? Z->rows : Z->cols; }
const DeviceBasis& basis(const h2_matrix* Z, int side) { return side == 0 ? Z->V : Z->W; }

h2_status plan_single(const h2_matrix* Z, int32_t b0, int u, int64_t lda, int64_t ldb) {
  HostPlan& P = g_plan;
  const BlockTree& bt = Z->blocks;
  const int32_t root[2] = {bt.row[b0], bt.col[b0]};
  const int depth = std::max(Z->rows.depth, Z->cols.depth);
  if (depth + 1 > kNaLevels) return fail(H2_EINVAL, "tree depth %lld above %lld", depth, kNaLevels - 1);
  P.n_items = P.n_ents = P.n_tasks = P.n_norms = 0;
  P.qlen = 0;
  for (int sd = 0; sd < 2; ++sd) {
    const ClusterTree& ct = tree(Z, sd);
    const DeviceBasis& bs = basis(Z, sd);
    for (int32_t c = 0; c < ct.count(); ++c) P.item_of[sd][c] = -1;
    int top = 0;
    P.nsub[sd] = 0;
    P.stack[top++] = root[sd];
    while (top > 0) {
      const int32_t c = P.stack[--top];
      if (P.nsub[sd] >= kNaClusters) return fail(H2_EINVAL, "subtree above %lld clusters", kNaClusters);
      P.sub[sd][P.nsub[sd]++] = c;
      if (!ct.leaf(c)) {
        if (top + 2 > kNaClusters) return fail(H2_EINVAL, "subtree above %lld clusters", kNaClusters);
        P.stack[top++] = ct.son1[c];
        P.stack[top++] = ct.son0[c];
      }
    }
    for (int i = 0; i < P.nsub[sd]; ++i) {
      const int32_t c = P.sub[sd][i];
      if (P.n_items >= kNaItems)
        return fail(H2_EINVAL, "the update touches more than %lld cluster tasks (fixed scratch limit)", kNaItems);
      Item it{};
      it.update = 0;
      it.side = sd;
      it.cluster = c;
      it.parent = (c == root[sd]) ? -1 : P.item_of[sd][ct.father[c]];
      it.son0 = it.son1 = -1;
      if (ct.leaf(c)) it.flags |= kItemLeaf;
      if (c == root[sd]) it.flags |= kItemRoot;
      if (ct.father[c] < 0) it.flags |= kItemTreeRoot;
      it.k = bs.rank[c];
      it.kf = ct.father[c] >= 0 ? bs.rank[ct.father[c]] : 0;
      if (it.k + u > Z->kcap)
        return fail(H2_EINVAL, "rank %lld + update rank would exceed the storage capacity %lld "
                    "(this entry point never grows storage)", it.k, Z->kcap);
      it.size = (int32_t)ct.size[c];
      it.rowoff = (int32_t)(ct.off[c] - ct.off[root[sd]]);
      it.ld = (int32_t)(sd == 0 ? lda : ldb);
      it.foff = 0;
      it.qoff = -1;
      if (ct.leaf(c)) {
        it.qoff = P.qlen;
        P.qlen += ct.size[c] * (it.k + u);
        if (P.qlen > kNaQ) return fail(H2_EINVAL, "new leaf bases above %lld doubles", kNaQ);
      }
      P.item_of[sd][c] = P.n_items;
      P.items[P.n_items++] = it;
    }
    for (int i = 0; i < P.nsub[sd]; ++i) {
      const int32_t c = P.sub[sd][i];
      if (!ct.leaf(c)) {
        Item& it = P.items[P.item_of[sd][c]];
        it.son0 = P.item_of[sd][ct.son0[c]];
        it.son1 = P.item_of[sd][ct.son1[c]];
      }
    }
  }
  for (int sd = 0; sd < 2; ++sd) {
    const std::vector<int32_t>& ptr = sd == 0 ? bt.row_ptr : bt.col_ptr;
    const std::vector<int32_t>& adm = sd == 0 ? bt.row_adm : bt.col_adm;
    for (int i = 0; i < P.nsub[sd]; ++i) {
      const int32_t c = P.sub[sd][i];
      const int32_t iid = P.item_of[sd][c];
      Item& it = P.items[iid];
      it.ent_begin = P.n_ents;
      for (int32_t e = ptr[c]; e < ptr[c + 1]; ++e) {
        const int32_t slot = adm[e];
        const int32_t blk = bt.adm[slot];
        const int32_t o = sd == 0 ? bt.col[blk] : bt.row[blk];
        const int32_t oi = P.item_of[1 - sd][o];
        Entry en{slot, oi, o, -1};
        if (oi >= 0) {
          for (int q = 0; q < P.n_norms; ++q)
            if (P.norms[q].slot == slot) en.norm = q;
          if (en.norm < 0) {
            if (P.n_norms >= kNaNorms) return fail(H2_EINVAL, "more than %lld blocks inside the update", kNaNorms);
            P.norms[P.n_norms] = NormTask{slot, sd == 0 ? iid : oi, sd == 0 ? oi : iid, 0};
            en.norm = P.n_norms++;
          }
          it.flags |= kItemInside;
        }
        if (P.n_ents >= kNaEntries) return fail(H2_EINVAL, "weight stacks above %lld blocks", kNaEntries);
        P.ents[P.n_ents++] = en;
        const int kt = Z->V.rank[bt.row[blk]], ls = Z->W.rank[bt.col[blk]];
        if (sd == 0 || oi < 0) {
          if (P.n_tasks >= kNaTasks) return fail(H2_EINVAL, "more than %lld affected couplings", kNaTasks);
          P.tasks[P.n_tasks++] = sd == 0 ? Task{slot, iid, oi, kt, ls} : Task{slot, -1, iid, kt, ls};
        }
      }
      it.ent_end = P.n_ents;
    }
  }
  // items by level, bound on the truncation rows per level
  const int L = depth + 1;
  for (int l = 0; l <= L; ++l) P.lvl_ptr[l] = 0;
  for (int l = 0; l < L; ++l) P.lvl_rows[l] = 0;
  P.kl = 0;
  for (int i = 0; i < P.n_items; ++i) {
    const Item& it = P.items[i];
    P.lvl_ptr[tree(Z, it.side).level[it.cluster] + 1]++;
    P.kl = std::max(P.kl, it.k + u);
  }
  for (int l = 0; l < L; ++l) P.lvl_ptr[l + 1] += P.lvl_ptr[l];
  int fill[kNaLevels];
  for (int l = 0; l < L; ++l) {
    fill[l] = P.lvl_ptr[l];
    P.lvl_leaves[l] = 0;
  }
  for (int pass = 0; pass < 2; ++pass)   // leaves first within a level
    for (int i = 0; i < P.n_items; ++i) {
      const Item& it = P.items[i];
      const bool leaf = it.flags & kItemLeaf;
      if (leaf != (pass == 0)) continue;
      const int lev = tree(Z, it.side).level[it.cluster];
      P.lvl_list[fill[lev]++] = i;
      if (leaf) ++P.lvl_leaves[lev];
      const int rows = leaf ? it.size : P.items[it.son0].k + P.items[it.son1].k + 2 * u;
      P.lvl_rows[lev] = std::max(P.lvl_rows[lev], rows);
    }
  for (int l = 0; l < L; ++l)
    if (P.lvl_rows[l] > 64) return fail(H2_EINVAL, "leaf clusters above 64 indices are not supported");
  // all clusters of both sides by level, for the weights of the unchanged matrix
  for (int l = 0; l <= L; ++l) P.cl_ptr[l] = 0;
  for (int sd = 0; sd < 2; ++sd)
    for (int32_t c = 0; c < tree(Z, sd).count(); ++c) P.cl_ptr[tree(Z, sd).level[c] + 1]++;
  for (int l = 0; l < L; ++l) P.cl_ptr[l + 1] += P.cl_ptr[l];
  for (int l = 0; l < L; ++l) fill[l] = P.cl_ptr[l];
  for (int sd = 0; sd < 2; ++sd)
    for (int32_t c = 0; c < tree(Z, sd).count(); ++c) P.cl_list[fill[tree(Z, sd).level[c]]++] = (sd << 30) | c;
  return H2_OK;
}

h2_status run(h2_ctx* ctx, h2_matrix* Z, int32_t b0, int u, const double* A, int64_t lda, const double* B,
              int64_t ldb, double eps) {
  HostPlan& P = g_plan;
  for (int sd = 0; sd < 2; ++sd)
    if (tree(Z, sd).count() > kNaClusters)
      return fail(H2_EINVAL, "the matrix has %lld clusters per side; this entry point handles at most %lld",
                  tree(Z, sd).count(), kNaClusters);
  h2_status st = plan_single(Z, b0, u, lda, ldb);
  if (st != H2_OK) return st;
  unsigned char* base = nullptr;
  st = scratch_address(ctx->device, &base);
  if (st != H2_OK) return st;
  cudaStream_t s = ctx->stream;
  Item* d_items = reinterpret_cast<Item*>(base + kOffItems);
  Entry* d_ents = reinterpret_cast<Entry*>(base + kOffEnts);
  Task* d_tasks = reinterpret_cast<Task*>(base + kOffTasks);
  NormTask* d_nt = reinterpret_cast<NormTask*>(base + kOffNT);
  int32_t* d_lvl = reinterpret_cast<int32_t*>(base + kOffLvl);
  int32_t* d_cl = reinterpret_cast<int32_t*>(base + kOffCl);
  NA_CUDA(cudaMemcpyAsync(d_items, P.items, P.n_items * sizeof(Item), cudaMemcpyHostToDevice, s));
  if (P.n_ents) NA_CUDA(cudaMemcpyAsync(d_ents, P.ents, P.n_ents * sizeof(Entry), cudaMemcpyHostToDevice, s));
  if (P.n_tasks) NA_CUDA(cudaMemcpyAsync(d_tasks, P.tasks, P.n_tasks * sizeof(Task), cudaMemcpyHostToDevice, s));
  P.n_two = 0;
  for (int t = 0; t < P.n_tasks; ++t)
    if (P.tasks[t].it >= 0 && P.tasks[t].is >= 0) P.two[P.n_two++] = t;
  int32_t* d_two = reinterpret_cast<int32_t*>(base + kOffTwo);
  if (P.n_two) NA_CUDA(cudaMemcpyAsync(d_two, P.two, P.n_two * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (P.n_norms) NA_CUDA(cudaMemcpyAsync(d_nt, P.norms, P.n_norms * sizeof(NormTask), cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaMemcpyAsync(d_lvl, P.lvl_list, P.n_items * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  const int L = std::max(Z->rows.depth, Z->cols.depth) + 1;
  NA_CUDA(cudaMemcpyAsync(d_cl, P.cl_list, P.cl_ptr[L] * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  ItemBuffers IB{};
  IB.Rq = reinterpret_cast<double*>(base + kOffRq);
  IB.Bw = reinterpret_cast<double*>(base + kOffBw);
  IB.Rt = reinterpret_cast<double*>(base + kOffRt);
  IB.F = reinterpret_cast<double*>(base + kOffF);
  IB.Q = reinterpret_cast<double*>(base + kOffQ);
  IB.rank = reinterpret_cast<int32_t*>(base + kOffRank);
  IB.own = reinterpret_cast<int32_t*>(base + kOffOwn);
  IB.norms = reinterpret_cast<double*>(base + kOffNorm);
  IB.S_out = reinterpret_cast<double*>(base + kOffS);
  IB.copy = reinterpret_cast<int8_t*>(base + kOffCopyFlag);
  IB.jac = reinterpret_cast<unsigned long long*>(base + kOffJac);
  // the certified path's Gram matrices are dead before the exact path
  // writes its R-factors and weights into the same tiles
  IB.Gv = IB.Rq;
  IB.Wg = IB.Bw;
  IB.fail = reinterpret_cast<int32_t*>(base + kOffFail);
  BaseWeights BW{};
  for (int sd = 0; sd < 2; ++sd) {
    BW.G[sd] = reinterpret_cast<double*>(base + kOffG) + (size_t)sd * kNaClusters * kSlot;
    BW.B[sd] = reinterpret_cast<double*>(base + kOffB) + (size_t)sd * kNaClusters * kSlot;
    BW.Wo[sd] = BW.G[sd];
    BW.W0[sd] = BW.B[sd];
    BW.need[sd] = reinterpret_cast<int32_t*>(base + kOffNeed) + (size_t)sd * kNaClusters;
    BW.Vg[sd] = reinterpret_cast<double*>(base + kOffS) + (size_t)sd * kNaClusters * kSlot;
    BW.orth[sd] = reinterpret_cast<int32_t*>(base + kOffOrth) + (size_t)sd * kNaClusters;
  }
  MatView M;
  for (int sd = 0; sd < 2; ++sd) {
    const DeviceBasis& bs = basis(Z, sd);
    M.leaf[sd] = bs.d_leaf;
    M.transfer[sd] = bs.d_transfer;
    M.leaf_off[sd] = bs.d_leaf_off;
    M.rank[sd] = bs.d_rank;
  }
  M.father[0] = Z->d_father_r;
  M.father[1] = Z->d_father_c;
  M.subtree[0] = Z->d_subtree_r;
  M.subtree[1] = Z->d_subtree_c;
  M.size[0] = Z->d_row_size;
  M.size[1] = Z->d_col_size;
  M.S = Z->d_S;
  M.kcap = Z->kcap;
  // the same kernels as the allocating path, on the fixed scratch
  Pipeline pp{};
  pp.M = M;
  pp.BL.ptr[0] = Z->d_row_ptr;
  pp.BL.ptr[1] = Z->d_col_ptr;
  pp.BL.adm[0] = Z->d_row_adm;
  pp.BL.adm[1] = Z->d_col_adm;
  pp.BL.other[0] = Z->d_blk_col;
  pp.BL.other[1] = Z->d_blk_row;
  pp.BW = BW;
  pp.IB = IB;
  pp.items = d_items;
  pp.ents = d_ents;
  pp.tasks = d_tasks;
  pp.norms = d_nt;
  pp.lvl_list = d_lvl;
  pp.lvl_ptr = P.lvl_ptr;
  pp.lvl_leaves = P.lvl_leaves;
  pp.lvl_rows = P.lvl_rows;
  pp.cl_list = d_cl;
  pp.cl_ptr = P.cl_ptr;
  pp.levels = L;
  pp.n_updates = 1;
  pp.ncl[0] = Z->rows.count();
  pp.ncl[1] = Z->cols.count();
  pp.exact_only = 0;
  pp.n_tasks = P.n_tasks;
  pp.two = d_two;
  pp.n_two = P.n_two;
  pp.left = reinterpret_cast<int32_t*>(base + kOffLeft);
  pp.n_left = reinterpret_cast<int32_t*>(base + kOffNLeft);
  pp.n_norms = P.n_norms;
  pp.u = u;
  pp.kl = P.kl;
  pp.eps = eps;
  pp.A = A;
  pp.B = B;
  pp.err = ctx->d_error;
  pp.stream = s;
  pp.side = nullptr;
  pp.fork = nullptr;
  pp.join = nullptr;
  pp.side2 = nullptr;
  pp.join2 = nullptr;
  pp.events = nullptr;
  pp.phase_launches = nullptr;
  pp.out = nullptr;
  run_pipeline(pp);
  NA_CUDA(cudaGetLastError());
  // commit (Section 5): new bases, transfers, couplings, nearfield inside b0
  NA_CUDA(cudaMemcpyAsync(P.rank, IB.rank, P.n_items * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (P.n_tasks) NA_CUDA(cudaMemcpyAsync(P.copy, IB.copy, P.n_tasks * sizeof(int8_t), cudaMemcpyDeviceToHost, s));
  NA_CUDA(cudaStreamSynchronize(s));
  int err = 0;
  NA_CUDA(cudaMemcpy(&err, ctx->d_error, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    NA_CUDA(cudaMemset(ctx->d_error, 0, sizeof(int)));
    return fail(H2_EDEVICE, "device reported an internal limit (code %lld)", err);
  }
  int nc = 0;
  const int kcap = Z->kcap;
  for (int i = 0; i < P.n_items; ++i) {
    const Item& it = P.items[i];
    const DeviceBasis& db = basis(Z, it.side);
    const ClusterTree& ct = tree(Z, it.side);
    const int r = P.rank[i];
    if ((it.flags & kItemLeaf) && r > 0)
      P.copies[nc++] = CopyDesc{IB.Q + it.qoff, db.d_leaf + db.leaf_off[it.cluster], it.size, r, it.size, it.size};
    if (!(it.flags & kItemTreeRoot)) {
      const int rf = (it.flags & kItemRoot) ? db.rank[ct.father[it.cluster]] : P.rank[it.parent];
      if (r > 0 && rf > 0)
        P.copies[nc++] = CopyDesc{IB.F + (size_t)i * kSlot, db.d_transfer + (size_t)it.cluster * kcap * kcap, r, rf,
                                  32, kcap};
    }
  }
  for (int t = 0; t < P.n_tasks; ++t) {
    const Task& tk = P.tasks[t];
    const int rt = tk.it >= 0 ? P.rank[tk.it] : tk.kt;
    const int rs = tk.is >= 0 ? P.rank[tk.is] : tk.ls;
    if (rt <= 0 || rs <= 0) continue;
    double* d = Z->d_S + (size_t)tk.slot * kcap * kcap;
    if (P.copy[t]) {
      // [S_b; 0] or [S_b, 0] in place: only the zero rows or columns
      if (tk.it >= 0)
        P.copies[nc++] = CopyDesc{nullptr, d + tk.kt, rt - tk.kt, rs, 0, kcap};
      else
        P.copies[nc++] = CopyDesc{nullptr, d + (size_t)tk.ls * kcap, rt, rs - tk.ls, 0, kcap};
      continue;
    }
    P.copies[nc++] = CopyDesc{IB.S_out + (size_t)t * kSlot, d, rt, rs, 32, kcap};
  }
  const BlockTree& bt = Z->blocks;
  int nn = 0, top = 0;
  P.bstack[top++] = b0;
  while (top > 0) {
    const int32_t b = P.bstack[--top];
    if (bt.kind[b] == kSub) {
      for (int i = 3; i >= 0; --i)
        if (bt.son4[4 * b + i] >= 0) {
          if (top >= (int)(sizeof(P.bstack) / sizeof(P.bstack[0])))
            return fail(H2_EINVAL, "block subtree too large for the fixed scratch");
          P.bstack[top++] = bt.son4[4 * b + i];
        }
    } else if (bt.kind[b] == kNear) {
      if (nn >= kNaNear) return fail(H2_EINVAL, "more than %lld nearfield leaves inside the block", kNaNear);
      const int32_t t = bt.row[b], sc = bt.col[b];
      NearDesc d{};
      d.N = Z->d_N + Z->near_off[bt.slot[b]];
      d.A = A + (Z->rows.off[t] - Z->rows.off[bt.row[b0]]);
      d.B = B + (Z->cols.off[sc] - Z->cols.off[bt.col[b0]]);
      d.rows = (int)Z->rows.size[t];
      d.cols = (int)Z->cols.size[sc];
      d.ldn = d.rows;
      d.lda = (int)lda;
      d.ldb = (int)ldb;
      P.nears[nn++] = d;
    }
  }
  CopyDesc* d_copy = reinterpret_cast<CopyDesc*>(base + kOffCopy);
  NearDesc* d_near = reinterpret_cast<NearDesc*>(base + kOffNear);
  if (nc) NA_CUDA(cudaMemcpyAsync(d_copy, P.copies, nc * sizeof(CopyDesc), cudaMemcpyHostToDevice, s));
  if (nn) NA_CUDA(cudaMemcpyAsync(d_near, P.nears, nn * sizeof(NearDesc), cudaMemcpyHostToDevice, s));
  launch_copy(d_copy, nc, s);
  launch_near_add(d_near, nn, u, s);
  NA_CUDA(cudaGetLastError());
  for (int i = 0; i < P.n_items; ++i) {
    const Item& it = P.items[i];
    DeviceBasis& db = it.side == 0 ? Z->V : Z->W;
    db.rank[it.cluster] = P.rank[i];
  }
  NA_CUDA(cudaMemcpyAsync(Z->V.d_rank, Z->V.rank.data(), Z->V.rank.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaMemcpyAsync(Z->W.d_rank, Z->W.rank.data(), Z->W.rank.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice, s));
  NA_CUDA(cudaStreamSynchronize(s));
  return H2_OK;
}

}  // namespace
}  // namespace h2

extern "C" h2_status h2_lowrank_update_noalloc(h2_ctx* ctx, h2_matrix* Z, int64_t block, int u, const double* A,
                                               int64_t lda, const double* B, int64_t ldb, double eps) {
  using namespace h2;
  if (!ctx || !Z || !A || !B) return H2_EINVAL;
  std::lock_guard<std::mutex> hold(g_lock);
  h2_status st = H2_OK;
  g_msg[0] = 0;
  if (block < 0 || block >= Z->blocks.count()) {
    st = fail(H2_EINVAL, "block %lld out of range", block);
  } else if (u < 1 || u >= kMaxCols) {
    st = fail(H2_EINVAL, "update rank %lld must be in 1..31", u);
  } else if (!Z->d_S && !Z->blocks.adm.empty()) {
    st = fail(H2_EINVAL, "matrix has no device storage");
  } else if (lda < Z->rows.size[Z->blocks.row[block]] || ldb < Z->cols.size[Z->blocks.col[block]]) {
    st = fail(H2_EINVAL, "leading dimension too small");
  } else if (lda > INT32_MAX || ldb > INT32_MAX) {
    // the kernels index the caller's factors with 32-bit leading dimensions
    st = fail(H2_EINVAL, "leading dimension above 2^31 - 1");
  } else if (!std::isfinite(eps) || eps < 0) {
    st = fail(H2_EINVAL, "eps must be finite and >= 0");
  } else {
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) {
      st = fail(H2_ECUDA, "cudaSetDevice failed");
    } else {
      try {
        st = run(ctx, Z, (int32_t)block, u, A, lda, B, ldb, eps);
      } catch (const std::exception& e) {
        std::snprintf(g_msg, sizeof(g_msg), "%s", e.what());
        st = H2_ECUDA;
      }
      if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    }
  }
  if (st != H2_OK) ctx->last_error = std::string("h2_lowrank_update_noalloc: ") + g_msg;
  return st;
}
