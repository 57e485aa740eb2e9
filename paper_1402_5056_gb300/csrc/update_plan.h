// Device-side plan of a batch of local low-rank updates (shared by the
// host planner in api.cu and the kernels in update_kernels.cu).
#pragma once

#include <cstdint>

namespace h2 {

// Item flags.
constexpr int32_t kItemLeaf = 1;       // cluster is a leaf of the cluster tree
constexpr int32_t kItemRoot = 2;       // cluster is the root of the update's subtree
constexpr int32_t kItemInside = 4;     // some block of row(t)/col(s) lies inside the update
constexpr int32_t kItemTreeRoot = 8;   // cluster is the root of the cluster tree

// Device error codes (OR-ed into the context's error word).
constexpr int kErrRows = 1;      // a matrix has more rows than the kernel's register tile
constexpr int kErrCols = 2;      // more than 32 columns
constexpr int kErrJacobi = 4;    // one-sided Jacobi did not converge in the sweep limit
constexpr int kErrRank = 8;      // inconsistent ranks
constexpr int kErrPivot = 256;   // zero pivot in a leaf LU (H^2-LR)
constexpr int kErrDefinite = 512;   // pivot not positive in a leaf Cholesky

// One cluster of one side of one update ("cluster task").
struct Item {
  int32_t update;      // index of the update in the batch
  int32_t side;        // 0 row basis V (factor A), 1 column basis W (factor B)
  int32_t cluster;
  int32_t parent;      // item of the father inside the subtree, -1 for the subtree root
  int32_t son0, son1;  // items of the sons, -1 for leaves
  int32_t flags;
  int32_t k;           // rank of the cluster before the update
  int32_t kf;          // rank of the father before the update (0 for the tree root)
  int32_t size;        // #t
  int32_t rowoff;      // offset of t's rows inside the update's factor
  int32_t ld;          // rows of the update's factor (#t0 or #s0)
  int32_t ent_begin, ent_end;  // entries (blocks of row(t) or col(s))
  int64_t foff;        // element offset of the update's factor
  int64_t qoff;        // element offset of the new leaf basis (leaves), -1 otherwise
};

// One admissible block of row(t) (row-side item) or col(s) (column-side item).
struct Entry {
  int32_t slot;        // coupling slot of the block
  int32_t other;       // item of the other cluster if it lies in the other subtree, else -1
  int32_t other_cluster;
  int32_t norm;        // slot of ||Z~|_b||_F for inside blocks, -1 otherwise
};

// One coupling to reproject: S_b <- R_t S~_b R_s^*.
struct Task {
  int32_t slot;
  int32_t it;          // row-side item or -1 (row cluster outside T_t0)
  int32_t is;          // column-side item or -1
  int32_t kt, ls;      // ranks of the row and column cluster before the update
};

// Inside block whose norm ||R_t S~_b R_s^*||_F is needed by the weights.
struct NormTask {
  int32_t slot;
  int32_t it, is;
  int32_t pad;
};

// Pointers a kernel needs from the matrix (read-only during execution).
struct MatView {
  const double* leaf[2];
  const double* transfer[2];
  const int64_t* leaf_off[2];
  const int32_t* rank[2];
  const int32_t* father[2];
  const int32_t* subtree[2];   // clusters in the subtree (1 for leaves; sons of c: c + 1 and
                               // c + 1 + subtree[c + 1], clusters being numbered in preorder)
  const int32_t* size[2];      // #t
  const double* S;
  int kcap;
};

// Global weights of the unchanged matrix (both sides), per cluster.
struct BaseWeights {
  double* G[2];        // R-factor of the weighted blocks of row(t)/col(s), ld 32
  double* B[2];        // R-factor of the full weight stack B~_t, ld 32
  // Gram matrices of the same stacks for the certified path (Wo = G^* G,
  // W0 = B^* B).  They are dead once the certified path has finished and
  // may share storage with G and B, which only the exact path writes.
  double* Wo[2];
  double* W0[2];
  int32_t* need[2];    // per cluster: 1 if the exact path needs G and B of it
  // Gram matrix V_t^* V_t of every cluster basis of the unchanged matrix and
  // a flag: 1 when it equals the identity within 1e-13 (orthonormal basis)
  double* Vg[2];
  int32_t* orth[2];
};

// Per-item workspace and outputs; every matrix slot is 32 x 32, ld 32.
struct ItemBuffers {
  double* Rq;          // basis R-factor (step 2)
  double* Bw;          // weight matrix B~_t (step 3)
  double* Rt;          // R_t = Q_t^* V~_t (step 4)
  double* F;           // new transfer matrix of the item's cluster
  double* Q;           // new leaf bases (at Item::qoff, ld = size)
  int32_t* rank;       // new rank
  int32_t* own;        // 1 if the item folds its outside blocks itself (step 3)
  double* norms;       // per NormTask
  // certified path: Gram matrices G_t = V~_t^* V~_t and W_t = B~_t^* B~_t.
  // They are dead before the exact path runs and may share storage with Rq
  // and Bw (the exact path only writes the tasks of updates that failed).
  double* Gv;
  double* Wg;
  int32_t* fail;       // per update: 1 if the exact path computes it
  double* S_out;       // per Task, 32 x 32 slots
  int8_t* copy;        // per Task: 1 when the new coupling is the old one padded with zeros
                       // ([S_b; 0] or [S_b, 0]); S_out is not written then
  unsigned long long* jac;   // per item: Jacobi pairs checked, rotations applied, 1 if the
                             // full-rank certificate held (no Jacobi), reserved (4 counters)
};

constexpr int kSlot = 32 * 32;

}  // namespace h2
