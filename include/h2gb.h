/*
 * h2gb -- H^2-matrix local low-rank updates on one NVIDIA GB300 (sm_103a).
 *
 * C ABI of libh2gb.so.  Method: Boerm & Reimer, "Efficient arithmetic
 * operations for rank-structured matrices based on hierarchical low-rank
 * updates" (arXiv:1402.5056).  Section references below are to that paper.
 *
 * Conventions (every entry point):
 *  - No exceptions cross the ABI; every call returns h2_status.  A non-OK
 *    status leaves a message retrievable with h2_last_error(ctx).
 *  - Argument errors (null pointer, id out of range, negative size, ...)
 *    return H2_EINVAL and modify nothing.
 *  - Host pointers are read or written synchronously before the call
 *    returns.  Device pointers are used asynchronously on the context's
 *    stream; the caller keeps ownership of every pointer it passes.
 *  - Matrices are column-major float64 unless stated otherwise.
 *  - Rows of a cluster basis and of update factors follow the TREE order of
 *    the cluster's index set (h2_tree_permutation maps tree positions to
 *    the caller's original point numbers).
 *  - Cluster bases must be orthonormal (V_t^* V_t = I), as Section 4
 *    assumes for the recompression; bases produced by this library are.
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef H2GB_H
#define H2GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  H2_OK = 0,
  H2_EINVAL = 1,       /* invalid argument                                   */
  H2_ENOMEM = 2,       /* device or host allocation failed                   */
  H2_ECUDA = 3,        /* a CUDA runtime call failed                         */
  H2_ETIMEOUT = 4,     /* a bounded device wait ran out                      */
  H2_EDEVICE = 5,      /* a kernel reported an internal limit (see message)  */
  H2_EINTERNAL = 6     /* unexpected internal error                          */
} h2_status;

typedef struct h2_ctx h2_ctx;         /* device + stream + device error word  */
typedef struct h2_matrix h2_matrix;   /* trees + device storage of one H^2 matrix */
typedef struct h2_batch h2_batch;     /* plan and outputs of a batch of updates */

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t to run on (NULL = the legacy default stream); the caller
 * keeps ownership of the stream. */
h2_status h2_ctx_create(int device, void* cuda_stream, h2_ctx** out);
void h2_ctx_destroy(h2_ctx* ctx);
/* Message of the last non-OK status on this context (never NULL). */
const char* h2_last_error(const h2_ctx* ctx);
/* Block until the context's stream is idle; returns H2_EDEVICE if any
 * kernel since the last check reported an internal limit, H2_ECUDA on a
 * CUDA error. */
h2_status h2_ctx_synchronize(h2_ctx* ctx);

/* ------------------------------------------------------------- structure */

/* Build the cluster tree and block tree (Section 2, Defs. "Cluster tree" and
 * "Block tree") for n points of dimension dim (host, row-major n x dim) and
 * allocate device storage for an H^2 matrix with row and column bases of
 * rank 0.
 *  - cluster tree: geometric bisection of the points' bounding box along its
 *    longest axis (ties: lowest axis) at the midpoint while a cluster has
 *    more than leaf_size points; coordinates below the midpoint go to the
 *    first son; clusters numbered in depth-first preorder, root 0;
 *  - admissibility of (t,s): dist > 0 and max(diam t, diam s) <= eta * dist
 *    with Euclidean box diameters/distance, boxes padded by `pad` per side;
 *  - block tree: a block is subdivided while inadmissible and both clusters
 *    have sons; blocks numbered in depth-first preorder, sons ordered
 *    (t1,s1),(t1,s2),(t2,s1),(t2,s2).
 * `kcap` (1..32) is the rank capacity of the storage; it grows on demand. */
h2_status h2_matrix_create(h2_ctx* ctx, const double* points, int64_t n, int dim,
                           int leaf_size, double eta, double pad, int kcap, h2_matrix** out);
void h2_matrix_free(h2_matrix* Z);
/* Deep copy (trees shared by value, device storage copied). */
h2_status h2_matrix_clone(h2_ctx* ctx, const h2_matrix* Z, h2_matrix** out);

/* Counts of the structure. Any output pointer may be NULL. */
h2_status h2_tree_sizes(const h2_matrix* Z, int64_t* n, int64_t* n_clusters, int64_t* n_blocks,
                        int64_t* n_admissible, int64_t* n_inadmissible, int* depth);
/* Per-cluster arrays (length n_clusters, host): offset and size of the
 * cluster's index range in tree order, father (-1 for the root), sons (-1
 * for leaves), level (root 0), #T_t (clusters in its subtree). */
h2_status h2_tree_clusters(const h2_matrix* Z, int64_t* offset, int64_t* size, int32_t* father,
                           int32_t* son0, int32_t* son1, int32_t* level, int32_t* subtree);
/* Per-block arrays (length n_blocks, host): row cluster, column cluster,
 * kind (0 subdivided, 1 admissible leaf, 2 inadmissible leaf), father. */
h2_status h2_tree_blocks(const h2_matrix* Z, int32_t* row, int32_t* col, int32_t* kind,
                         int32_t* father);
/* perm[i] = original point number of tree position i (host, length n). */
h2_status h2_tree_permutation(const h2_matrix* Z, int64_t* perm);

/* ------------------------------------------------------------------ data */

/* Canonical host layouts (column-major per matrix, concatenated):
 *   basis  : ranks[n_clusters]; leaf_data = V_t (size_t x k_t) for every
 *            leaf in cluster order; transfer_data = E_t (k_t x k_father) for
 *            every non-root cluster in cluster order (Eq. (nested)).
 *   couplings: S_b (k_t x l_s) for every admissible leaf in block order
 *            (Eq. (vsw)).
 *   nearfield: G|_b (size_t x size_s) for every inadmissible leaf in block
 *            order.
 * side 0 = row basis V, side 1 = column basis W.  Setting a basis with new
 * ranks invalidates the couplings (set them again afterwards). */
h2_status h2_set_basis(h2_ctx* ctx, h2_matrix* Z, int side, const int32_t* ranks,
                       const double* leaf_data, const double* transfer_data);
h2_status h2_set_couplings(h2_ctx* ctx, h2_matrix* Z, const double* data);
h2_status h2_set_nearfield(h2_ctx* ctx, h2_matrix* Z, const double* data);
/* Element counts of the canonical layouts for the current ranks. */
h2_status h2_data_sizes(const h2_matrix* Z, int side, int64_t* leaf_len, int64_t* transfer_len,
                        int64_t* coupling_len, int64_t* nearfield_len);
h2_status h2_get_ranks(const h2_matrix* Z, int side, int32_t* ranks);
h2_status h2_get_basis(h2_ctx* ctx, const h2_matrix* Z, int side, double* leaf_data,
                       double* transfer_data);
h2_status h2_get_couplings(h2_ctx* ctx, const h2_matrix* Z, double* data);
h2_status h2_get_nearfield(h2_ctx* ctx, const h2_matrix* Z, double* data);
/* Single matrices (host outputs, column-major, leading dimension = rows):
 * leaf basis of a leaf cluster (size_t x k_t), transfer of a non-root
 * cluster (k_t x k_father), coupling of an admissible block (k_t x l_s). */
h2_status h2_get_leaf(h2_ctx* ctx, const h2_matrix* Z, int side, int64_t cluster, double* out);
h2_status h2_get_transfer(h2_ctx* ctx, const h2_matrix* Z, int side, int64_t cluster, double* out);
h2_status h2_get_coupling(h2_ctx* ctx, const h2_matrix* Z, int64_t block, double* out);

/* --------------------------------------------------------------- updates */

/* Plan a batch of `count` local low-rank updates
 *     Z|_{t0 x s0} <- trunc_eps(Z|_{t0 x s0} + A_j B_j^*)      (Section 5)
 * on the blocks blocks[j] (any block-tree node, host array) with update
 * rank u (1..31, k_t + u <= 32 for every cluster touched).  The plan holds
 * the level-by-level task lists (clusters of the subtrees T_{t0}, T_{s0},
 * every admissible block whose row lies in T_{t0} or whose column lies in
 * T_{s0}) and the device workspace.  It reads the structure and ranks of Z
 * at creation; Z must not change ranks before the plan is executed. */
h2_status h2_batch_create(h2_ctx* ctx, const h2_matrix* Z, int64_t count, const int64_t* blocks,
                          int u, h2_batch** out);
void h2_batch_free(h2_batch* batch);
/* Rows of update j's factors: A_j is rows_A x u, B_j is rows_B x u, stored
 * at element offsets off_A, off_B of the concatenated factor arrays. */
h2_status h2_batch_factor_layout(const h2_batch* batch, int64_t j, int64_t* rows_A,
                                 int64_t* off_A, int64_t* rows_B, int64_t* off_B);
h2_status h2_batch_factor_sizes(const h2_batch* batch, int64_t* len_A, int64_t* len_B);

/* Execute the batch in ISOLATED mode: every update reads the same Z (the one
 * given at planning) and writes its own result (new ranks, bases, transfer
 * matrices and couplings) into the batch's output buffers; Z is not changed.
 * A and B are DEVICE pointers to the concatenated factors (layout from
 * h2_batch_factor_layout).  Truncation: block-relative accuracy eps
 * (Sections 4 and 7), every admissible block keeps
 * ||Z~|_b - Z_new|_b||_F <= eps/sqrt(2) ||Z~|_b||_F.  Asynchronous. */
h2_status h2_batch_execute(h2_ctx* ctx, h2_batch* batch, const double* A, const double* B,
                           double eps);
/* Same, from HOST factor arrays: copies them in, executes, and copies the
 * updates' new ranks, bases, transfer matrices and couplings back to the
 * host buffer `result` (length from h2_batch_result_size, layout from
 * h2_batch_result_offsets), then synchronizes.  When `result` is
 * page-locked (cudaHostAlloc / cudaHostRegister) most of it is copied while
 * the update runs. */
h2_status h2_batch_execute_host(h2_ctx* ctx, h2_batch* batch, const double* A_host,
                                const double* B_host, double eps, double* result);
/* Same with a compact result: copied[b] (one byte per block task, host
 * array of n_block_tasks entries) is set to 1 where the update keeps the
 * coupling -- the new coupling of block task b is the unchanged S_b of the
 * planned matrix padded with zero rows ([S_b; 0], row cluster changed) or
 * zero columns ([S_b, 0]), which happens for the one-sided blocks of a
 * certified update whose changed cluster keeps its orthonormal basis as the
 * leading part of the new one (Section 5 with the block form of the Gram
 * path) -- and to 0 elsewhere.  With a page-locked `result` those pieces are
 * not copied to the host (their contents in `result` are unspecified; read
 * S_b from the planned matrix, h2_get_coupling); every other piece is as in
 * h2_batch_execute_host.  With a pageable `result` every piece is written.
 * copied may be NULL only for a batch without block tasks. */
h2_status h2_batch_execute_host_compact(h2_ctx* ctx, h2_batch* batch, const double* A_host,
                                        const double* B_host, double eps, double* result,
                                        int8_t* copied);
/* Bytes the last h2_batch_execute_host(_compact) copied host -> device (the
 * factors) and device -> host (result pieces, chunk flags, pieces sent
 * again, copy flags). */
h2_status h2_batch_host_bytes(const h2_batch* batch, int64_t* h2d, int64_t* d2h);
h2_status h2_batch_result_size(const h2_batch* batch, int64_t* len);
/* Layout of that result (host arrays of n_cluster_tasks and n_block_tasks
 * entries, h2_batch_stats).  result[i] = new rank r_i of cluster task i
 * (h2_batch_item_info).  At item_off[i]: for a leaf cluster its new basis
 * (#t x r_i, column-major, ld #t), then, unless the cluster is the root of
 * its tree, its new transfer matrix (r_i x r_f, ld r_i; r_f = the new rank
 * of the father's task, or for the subtree root t0 the unchanged rank of
 * its father: the committed E_t0 of Section 5).  At task_off[b]: the new
 * coupling of block task b (h2_batch_task_info), r_t x r_s, ld r_t, with
 * r_t the new rank of its row cluster's task or, when the row cluster is
 * outside the update's subtrees, its unchanged rank (r_s likewise). */
h2_status h2_batch_result_offsets(const h2_batch* batch, int64_t* item_off, int64_t* task_off);
/* Block task b of a batch (a coupling the update changes, Section 5):
 * info[0] update index, info[1] block (block-tree index), info[2] the
 * cluster task of its row cluster or -1 (row cluster unchanged), info[3]
 * that of its column cluster or -1, info[4], info[5] the ranks of the row
 * and column cluster before the update. */
h2_status h2_batch_task_info(const h2_batch* batch, int64_t task, int32_t* info);
/* Commit update j's result into dst (Section 5: replace the bases in the
 * subtrees, the transfer matrices E_{t0}, E_{s0} and every affected
 * coupling; add A|_t B|_s^* to the inadmissible leaves inside the block --
 * this last part reads A, B again, so pass the same device factors).  dst
 * must have the structure of the planned matrix and, outside the touched
 * subtrees, its ranks; its storage grows if a new rank exceeds capacity.
 * The couplings that the update keeps ([S_b; 0] and [S_b, 0] of a certified
 * update whose basis keeps the old one as its leading part) are not stored
 * by the execution: they are read here from the planned matrix, which must
 * not have changed since (dst may be that matrix itself). */
h2_status h2_batch_apply(h2_ctx* ctx, const h2_batch* batch, int64_t j, const double* A,
                         const double* B, h2_matrix* dst);
/* Statistics of the last execution (host, synchronizes): number of cluster
 * tasks, block tasks, kernel launches, and the algorithmic float64 flop
 * count of the executed path (rotations of the one-sided Jacobi counted as
 * executed). */
h2_status h2_batch_stats(h2_ctx* ctx, const h2_batch* batch, int64_t* n_cluster_tasks,
                         int64_t* n_block_tasks, int64_t* n_launches, double* flops);

/* Phases of an execution, for h2_batch_phase_stats.  Phases 0-4 and 7 are
 * the certified Gram path (every update), phase 6 the exact path (the
 * updates whose certificate failed, see h2_batch_set_mode), phase 5 the
 * reprojection of every update. */
typedef enum {
  H2_PHASE_BASE_WEIGHTS = 0,  /* Gram matrices of the weights of the unchanged
                                 matrix (all clusters)                           */
  H2_PHASE_RFACTOR = 1,       /* step 2: basis Gram matrices R_t^* R_t           */
  H2_PHASE_NORMS = 2,         /* ||Z~|_b||_F of the blocks inside the update     */
  H2_PHASE_WEIGHTS = 3,       /* step 3: weight Gram matrices B~_t^* B~_t        */
  H2_PHASE_TRUNCATE = 4,      /* step 4: full-rank certificate, R_t              */
  H2_PHASE_REPROJECT = 5,     /* step 5: reprojection of the couplings           */
  H2_PHASE_EXACT = 6,         /* steps 2-4 by Householder R-factors and one-sided
                                 Jacobi SVD for the updates the certificate
                                 did not cover (with the weights of the
                                 unchanged matrix they need)                     */
  H2_PHASE_BASES = 7,         /* step 4: new leaf bases and transfer matrices of
                                 the certified updates, commit of E_t0           */
  H2_PHASE_COUNT = 8
} h2_phase;

/* Path selection of later executions of this batch.
 *   H2_MODE_AUTO (default): every update first takes the certified Gram
 *     path.  Its certificate proves, with a margin covering rounding, that
 *     the rank rule of step 4 keeps the full extended rank k_t + u at every
 *     cluster of the update; then every orthonormal basis of range(V~_t)
 *     gives the same truncated matrix as the singular vectors, and the path
 *     builds one from the Gram matrix of V~_t.  Updates for which any
 *     cluster fails the certificate are recomputed by the exact path.
 *   H2_MODE_EXACT: every update takes the exact path (Householder R-factors,
 *     one-sided Jacobi SVD; Sections 4 and 5 step by step).
 * Both produce the truncation the rank rule defines; bases may differ by an
 * orthogonal change of basis. */
typedef enum { H2_MODE_AUTO = 0, H2_MODE_EXACT = 1 } h2_mode;
h2_status h2_batch_set_mode(h2_batch* batch, int mode);
/* Per update of the last execution (host array of `count` entries): 1 if
 * the exact path computed it, 0 if the certified path did.  Synchronizes. */
h2_status h2_batch_paths(h2_ctx* ctx, const h2_batch* batch, int32_t* exact);

/* Enable (on = 1) or disable (on = 0) CUDA-event timing of each phase in
 * later executions of this batch (events on the context's stream).  on = 2
 * times the phases with every phase on the context's stream (the side
 * streams of the certified path unused), so that a phase's time is that of
 * its own kernels without overlap; the results are the same. */
h2_status h2_batch_set_timing(h2_batch* batch, int on);
/* Launches, device time in ms (last execution, only with timing enabled,
 * else -1) and algorithmic float64 flops of one phase.  Synchronizes. */
h2_status h2_batch_phase_stats(h2_ctx* ctx, const h2_batch* batch, int phase, int64_t* launches,
                               double* ms, double* flops);

/* Intermediate results of one cluster task of the last execution, for
 * step-by-step parity checks.  info (host, 8 entries): update index, side,
 * cluster, rank before, new rank, flags (1 leaf, 2 subtree root, 4 inside
 * blocks, 8 tree root), 0, 0.  which: 0 Gram matrix R^* R of the basis
 * R-factor (step 2), 1 Gram matrix B~_t^* B~_t of the weights (step 3), 2
 * R_t = Q_t^* V~_t (step 4); out = the 32 x 32 tile (column-major, ld 32,
 * zero outside the (k+u) x (k+u) or r x (k+u) part).  Synchronizes. */
h2_status h2_batch_item_info(const h2_batch* batch, int64_t item, int32_t* info);
h2_status h2_batch_item_tile(h2_ctx* ctx, const h2_batch* batch, int64_t item, int which,
                             double* out);
/* Cluster tasks of update j occupy items [first, last). */
h2_status h2_batch_update_items(const h2_batch* batch, int64_t j, int64_t* first, int64_t* last);

/* Size and rank statistics of an H^2 matrix (host data only; no device
 * access, no synchronisation).  out (host, 12 entries): 0 n, 1 clusters per
 * tree, 2 block-tree nodes, 3 admissible leaves, 4 inadmissible leaves,
 * 5 depth of the cluster tree, 6 rank capacity of the storage, 7 largest
 * row-basis rank, 8 largest column-basis rank, 9 bytes of device storage of
 * the bases, transfers, couplings and nearfield (at the rank capacity; 0
 * for a structure without device storage),
 * 10 bytes of the values the representation holds at its ranks (leaf bases
 * #t x k_t, transfers k_t x k_{t+}, couplings k_t x l_s, nearfield
 * #t x #s), 11 sum of the row-basis ranks.  max_rank_per_level (host,
 * depth + 1 entries, or NULL): the largest row-basis rank on each level of
 * the cluster tree.  Floating-point work is reported per batch
 * (h2_batch_stats, h2_batch_phase_stats) and per factorisation
 * (h2_lr_factor's stats). */
h2_status h2_stats(const h2_matrix* Z, int64_t* out, int32_t* max_rank_per_level);

/* Y <- alpha Z X + beta Y for nrhs right-hand sides (Section 2: Eq. (vsw)
 * on the admissible leaves with the nested bases of Eq. (nested), dense
 * inadmissible leaves; the product the multiplication of Section 3 applies
 * where a factor block is a leaf, Section 6 Case 2).  X (n_cols x nrhs, ld ldx) and Y (n_rows x nrhs, ld ldy)
 * are column-major DEVICE arrays with rows in TREE order
 * (h2_tree_permutation); they must not overlap; Y is not read when
 * beta = 0.  Forward transformation over the column tree, the couplings,
 * backward transformation over the row tree and the nearfield, each value
 * of the matrix read once.  Asynchronous on the context's stream (its
 * workspace is stream-ordered). */
h2_status h2_matvec(h2_ctx* ctx, const h2_matrix* Z, int64_t nrhs, double alpha, const double* X,
                    int64_t ldx, double beta, double* Y, int64_t ldy);

/* The dense block Z|_{t x s} of any block-tree node (Section 2: the
 * admissible leaves V_t S_b W_s^*, the dense inadmissible leaves, and the
 * sub-blocks of a subdivided node), into the DEVICE array out (#t x #s,
 * column-major, ld >= #t, rows and columns in tree order).  Computed as the
 * rows t of Z times the unit columns of s (h2_matvec with #s right-hand
 * sides): a check and a diagnostic, not a fast path.  Asynchronous. */
h2_status h2_block_to_dense(h2_ctx* ctx, const h2_matrix* Z, int64_t block, double* out, int64_t ld);

/* count updates Z|_{b_j} <- trunc_eps(Z|_{b_j} + A_j B_j^*) applied to Z in
 * place in the order j = 0, 1, ... (sequential semantics; Section 5 applied
 * repeatedly): the result is that of calling h2_lowrank_update for each in
 * turn.  Updates whose footprints do not meet -- what one writes (the bases
 * of its subtrees T_t0, T_s0, the couplings of blocks with row in T_t0 or
 * column in T_s0) the other does not read (the bases of its subtrees and
 * their ancestors, the couplings in their block rows and columns) -- run
 * together as one isolated batch (a wave); inside a wave every update reads
 * the matrix as it was before the wave and the commits follow in order.
 * A, B: DEVICE pointers to the concatenated factors: A_j (#t_j x u,
 * column-major) starts at element sum_{i<j} #t_i u of A, B_j likewise with
 * the column clusters.  waves (host, optional): the number of waves.
 * Synchronizes. */
h2_status h2_lowrank_update_sequence(h2_ctx* ctx, h2_matrix* Z, int64_t count, const int64_t* blocks,
                                     int u, const double* A, const double* B, double eps,
                                     int64_t* waves);
/* The waves h2_lowrank_update_sequence would use (host only, no device
 * work): wave[j] (host, count entries) = the wave of update j, n_waves
 * (optional) = their number. */
h2_status h2_sequence_waves(const h2_matrix* Z, int64_t count, const int64_t* blocks, int32_t* wave,
                            int64_t* n_waves);
/* One update applied to Z in place (sequential semantics; Section 5).
 * A (rows of block's row cluster x u, ld lda) and B (rows of column cluster
 * x u, ld ldb) are DEVICE pointers. */
h2_status h2_lowrank_update(h2_ctx* ctx, h2_matrix* Z, int64_t block, int u, const double* A,
                            int64_t lda, const double* B, int64_t ldb, double eps);

/* Allocation-free variant of h2_lowrank_update (the paper has no
 * counterpart; this is an interface for callers that must not allocate
 * device memory while they run: code living in a fixed device-memory budget
 * reserved at start-up, where an allocation in the middle of the run could
 * fail or take memory another part of the program counts on, and hosts
 * whose device allocator belongs to another runtime, e.g. a framework's
 * caching allocator that has reserved the free memory).  Same arguments,
 * same update, same
 * results as h2_lowrank_update, but every piece of device scratch comes
 * from one fixed 48 MiB array inside the library (held on every GPU that
 * loads the library until the process exits), host planning uses static
 * buffers, and no cudaMalloc/cudaFree or other allocating routine is
 * called.  Limits, rejected with H2_EINVAL and a message naming the limit:
 * at most 512 clusters per side in the matrix, 256 cluster tasks, 2048
 * affected couplings, 4096 weight-stack blocks, 256 blocks inside the
 * update, 1024 nearfield leaves inside the block, leading dimensions up to
 * 2^31 - 1; and k_t + u must fit the matrix's current rank capacity, because
 * this entry point never grows storage.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress, with that device
 * current) and keeps it for the process: make that first call before any
 * stream capture, and do not call this entry point on a device whose
 * primary context was destroyed (cudaDeviceReset) after that.  All calls
 * share the array and the host planning buffers, and the array keeps the
 * last call's contents; calls whose GPU work overlapped would race on them,
 * so each call holds a library-wide lock and synchronizes the context's
 * stream before it returns. */
h2_status h2_lowrank_update_noalloc(h2_ctx* ctx, h2_matrix* Z, int64_t block, int u, const double* A,
                                    int64_t lda, const double* B, int64_t ldb, double eps);

/* ------------------------------------------------ H^2-LR (Section 3, 7) */

/* Arithmetic of the factorisation.  H2_FP64: every step in float64. */
typedef enum { H2_FP64 = 0, H2_MIXED_FP32 = 1 } h2_precision;

/* Options of the FEM matrix and its factorisation.
 *  eps       block-relative truncation accuracy of every local update
 *            (Sections 4, 5 and 7; the rank rule of h2_batch_execute) and
 *            of the temporaries of the product (see h2_lr_factor);
 *  eta       admissibility parameter, max(diam t, diam s) <= eta dist(t, s);
 *  leaf_size clusters with more points are split;
 *  precision h2_precision;
 *  trunc_norm, weighting: 0 (Frobenius norm, block-relative weights) --
 *            the only supported values;
 *  max_rank  0: no rank cap (the paper's method: the rank rule alone);
 *            1..31: every local update of h2_lr_factor and h2_inverse
 *            keeps at most max_rank columns per new cluster basis (its
 *            leading singular directions), so that ranks stay within the
 *            32-column limit of the update kernels on problems whose
 *            ranks would exceed it.  The paper sets no cap; a cap changes
 *            the result wherever it binds.  Other values: H2_EINVAL. */
typedef struct {
  double eps;
  double eta;
  int leaf_size;
  int precision;
  int trunc_norm;
  int weighting;
  int max_rank;
} h2_options;

/* The P1 finite-element stiffness matrix of -div(sigma grad u) = f on the
 * unit square (dim 2) or cube (dim 3) with u = 0 on the boundary (the model
 * problem of Section 7), as an H^2 matrix.  `cells` cells per side; every
 * cell split into two triangles along its (i,j)-(i+1,j+1) diagonal (2D) or
 * into Kuhn's six tetrahedra around its main diagonal (3D); the unknowns
 * are the interior nodes (i/cells, j/cells[, k/cells]), numbered x fastest
 * (h2_tree_permutation maps tree positions to these numbers).  sigma (host,
 * checker^dim positive values, x fastest) is piecewise constant on a
 * checker x checker (x checker) grid; an element takes the value at its
 * centroid.  Cluster tree and block tree as in h2_matrix_create with the
 * points' support boxes (padding 1/cells): every admissible block of the
 * stiffness matrix is then zero, the bases have rank 0 and the nonzeros
 * sit in the inadmissible leaves.  Uses opt->leaf_size and opt->eta. */
h2_status h2_build_fem(h2_ctx* ctx, int dim, int64_t cells, int64_t checker, const double* sigma,
                       const h2_options* opt, h2_matrix** out);

/* In-place H^2-LR factorisation Z = L R (Section 3): on return the
 * strictly lower part of Z holds L (unit diagonal implied) and the upper
 * part R, as one H^2 matrix sharing its cluster bases.  Recursion: a leaf
 * (t, t) by Gaussian elimination without pivoting; otherwise factorise
 * (t1, t1), solve L11 R12 = A12 and L21 R11 = A21 by block forward
 * substitution, A22 <- A22 - L21 R12 by the product recursion (Section 3,
 * Cases 1 and 2 of Section 6), factorise (t2, t2).  Low-rank terms enter Z
 * through the local low-rank update with accuracy opt->eps.  Readings of
 * what the paper leaves open: a product's terms are computed from the
 * matrix as it is when the product starts; an admissible target of two
 * subdivided factors receives up to four temporaries, each the stacked
 * terms below it truncated by SVD (sum of the discarded sigma_i^2 <=
 * (eps/2)^2 of the total) and added by one update; forward substitution on
 * an admissible leaf V_t S W_s^* replaces it by (L^-1 V_t S) W_s^* through
 * an update; updates are applied in column groups of at most 32 - (largest
 * rank in the two subtrees) columns.  Z must be square with one tree and
 * its LU without pivoting must exist (SPD matrices).  stats (host, 15
 * entries, optional): local updates, product terms, largest rank, then the
 * wall time in microseconds spent on the local updates, on computing the
 * product terms, on the temporaries (truncation), on the dense solves
 * through diagonal blocks, on the leaf LU launches, and, within the local
 * updates, on host planning, on enqueueing their kernels, on waiting for
 * the GPU before each commit, and in total; then the microseconds spent
 * waiting for the truncation rank of the temporaries, their number and
 * their stacked columns.  Synchronizes. */
h2_status h2_lr_factor(h2_ctx* ctx, h2_matrix* Z, const h2_options* opt, int64_t* stats);

/* The product of Section 3, Z|_{t x r} <- Z|_{t x r} + alpha X|_{t x s}
 * Y|_{s x r}, for blocks bx = (t, s), by = (s, r), bz = (t, r) of the block
 * tree X, Y and Z share (same points, leaf size and eta; X or Y may be Z
 * itself).  The recursion of Section 3 over the sons (the eight
 * sub-products, Case 1 of Section 6); where X or Y is a leaf the term is
 * low rank, (X|_{t x s} V_s) S W_r^* or V_t S (Y|_{s x r}^* W_s)^* (Case 2),
 * or dense; low-rank terms enter Z through the local low-rank update with
 * accuracy eps, dense ones are added to inadmissible leaves; a target that
 * is an admissible leaf of two subdivided factors receives up to four
 * truncated temporaries.  Every term is computed from the matrices as they
 * are when the call starts.  X and Y are not modified (unless one is Z).
 * updates (host, optional): local updates made.  Synchronizes. */
h2_status h2_mul(h2_ctx* ctx, double alpha, const h2_matrix* X, int64_t bx, const h2_matrix* Y, int64_t by,
                 h2_matrix* Z, int64_t bz, double eps, int64_t* updates);

/* h2_lr_factor of count independent matrices at once (Section 3 for each;
 * batches of problems of different sizes): `threads` host threads (0: one
 * per hardware thread, at most count) take the matrices in turn, each on a
 * stream and context of its own on ctx's device, so that the few-task
 * launches of the factorisations run side by side.  Every result equals
 * h2_lr_factor of that matrix alone.  The matrices must be distinct; ctx's
 * stream is synchronized first.  stats (host, 3 entries per matrix, or
 * NULL): local updates, product terms, largest rank.  Synchronizes; on
 * failure the status of the first failing matrix (in index order) with its
 * index in the message, the other matrices factorised or not. */
h2_status h2_lr_factor_many(h2_ctx* ctx, h2_matrix* const* Z, int64_t count, const h2_options* opt, int threads,
                            int64_t* stats);

/* X <- R^-1 L^-1 X for a factor from h2_lr_factor: block forward and
 * backward substitution (Section 3).  X: DEVICE n x nrhs, column-major, ld
 * ldx, rows in TREE order.  Synchronizes. */
h2_status h2_lr_solve(h2_ctx* ctx, const h2_matrix* LR, int64_t nrhs, double* X, int64_t ldx);

/* Conjugate gradients for A x = b preconditioned by the factor LR (NULL =
 * none), from x = 0, stopped when ||b - A x||_2 <= tol ||b||_2 (the
 * recursively updated residual) or after maxit steps (Section 7).  A: the
 * matrix (not factorised; applied by h2_matvec); b, x: DEVICE vectors in
 * tree order.  iterations, relres (host, optional): steps taken, final
 * relative residual.  Synchronizes. */
h2_status h2_pcg(h2_ctx* ctx, const h2_matrix* A, const h2_matrix* LR, const double* b, double* x, double tol,
                 int maxit, int* iterations, double* relres);

/* ||I - LR^-1 A||_2 estimated by the power iteration (Section 7, column
 * Err): iters steps v <- w / ||w||, w = v - LR^-1 A v, from the DEVICE
 * start vector v (n entries, tree order; overwritten); err (host) = the
 * last ||w||.  Synchronizes. */
h2_status h2_lr_error(h2_ctx* ctx, const h2_matrix* A, const h2_matrix* LR, double* v, int iters, double* err);

/* Approximate inverse by block Gauss elimination (Section 3, Remark on
 * inversion).  For a diagonal block with sons t1, t2: C11 = A11^-1
 * (recursively), B12 = C11 A12, B21 = A21 C11, S = A22 - A21 B12,
 * C22 = S^-1 (recursively), C12 = -B12 C22, C21 = -C22 B21,
 * C11 <- C11 - C12 B21; a leaf is inverted by LU without pivoting and two
 * triangular solves with the identity.  Every product is the product of
 * Section 3 (as h2_mul, accuracy opt->eps) into a matrix that starts at
 * zero.  *out receives a new H^2 matrix with A's trees (free it with
 * h2_matrix_free).  A is consumed: its blocks below and right of the first
 * son hold Schur complements on return (clone A to keep it).  stats (host,
 * 3 entries, or NULL): local updates, product terms, largest rank of the
 * inverse.  Synchronizes.  H2_EINVAL if A is not square with one tree; on
 * any failure *out is NULL and A may have changed. */
h2_status h2_inverse(h2_ctx* ctx, h2_matrix* A, const h2_options* opt, h2_matrix** out, int64_t* stats);

/* h2_pcg with the approximate inverse C from h2_inverse as the
 * preconditioner (z = C r by h2_matvec); same arguments and results. */
h2_status h2_pcg_inverse(h2_ctx* ctx, const h2_matrix* A, const h2_matrix* C, const double* b, double* x, double tol,
                         int maxit, int* iterations, double* relres);

/* Approximate Cholesky factorisation A ~ L L^* of a symmetric positive
 * definite H^2 matrix in place (Section 7's preconditioner, built with the
 * algorithms of Section 3): on a diagonal block with sons t1, t2,
 * L11 = chol(A11) (recursively), L21 = A21 L11^-* (block substitution over
 * the sons of the column cluster; an admissible leaf V_t S W_s^* becomes
 * V_t (L^-1 W_s S^*)^*, added by one local update), A22 <- A22 - L21 L21^*
 * (the product of Section 3 with its second factor read transposed, only
 * the blocks on or below the diagonal of a diagonal target), L22 =
 * chol(A22); a leaf by dense Cholesky, its strictly upper part zeroed.
 * On return the lower triangle of Z (with the diagonal) holds L; the
 * strictly upper nearfield is never read and the strictly upper admissible
 * blocks hold no part of the factor.  Z must be square with one tree;
 * opt as for h2_lr_factor (max_rank included).  stats (host, 3 entries,
 * optional): local updates, product terms, largest rank.  Synchronizes;
 * H2_EDEVICE if a leaf pivot is not positive (A not positive definite to
 * the accuracy reached). */
h2_status h2_chol_factor(h2_ctx* ctx, h2_matrix* Z, const h2_options* opt, int64_t* stats);

/* h2_chol_factor of count independent matrices side by side, with the
 * threads, streams, statistics and failure rules of h2_lr_factor_many;
 * every result equals h2_chol_factor of that matrix alone. */
h2_status h2_chol_factor_many(h2_ctx* ctx, h2_matrix* const* Z, int64_t count, const h2_options* opt, int threads,
                              int64_t* stats);

/* X <- L^-* L^-1 X for a factor from h2_chol_factor (block forward and
 * backward substitution with L and its transpose).  X: DEVICE n x nrhs,
 * column-major, ld ldx, rows in TREE order.  Synchronizes. */
h2_status h2_chol_solve(h2_ctx* ctx, const h2_matrix* F, int64_t nrhs, double* X, int64_t ldx);

/* h2_pcg with the Cholesky factor F from h2_chol_factor as the
 * preconditioner (z = L^-* L^-1 r: symmetric positive definite, so CG is
 * the method it is built for); same arguments and results. */
h2_status h2_pcg_chol(h2_ctx* ctx, const h2_matrix* A, const h2_matrix* F, const double* b, double* x, double tol,
                      int maxit, int* iterations, double* relres);

/* h2_lr_error for a factor from h2_chol_factor: ||I - (L L^*)^-1 A||_2 by
 * the power iteration (Section 7, column Err); same arguments. */
h2_status h2_chol_error(h2_ctx* ctx, const h2_matrix* A, const h2_matrix* F, double* v, int iters, double* err);

/* ----------------------------------------------------------- diagnostics */

/* The float64 reciprocal the factorisation kernels use for their pivots
 * (the paper has no counterpart; a check of the arithmetic the certificate's
 * margin relies on): out[i] = the PTX estimate rcp.approx.ftz.f64 of 1/d[i]
 * refined by one cubic Newton-Raphson step, within one ulp of the correctly
 * rounded quotient.  Defined for normal d > 0 with a normal reciprocal.
 * d, out: DEVICE arrays of n doubles.  Asynchronous. */
h2_status h2_check_reciprocal(h2_ctx* ctx, const double* d, int64_t n, double* out);

/* Test hook for the error paths (no counterpart in the paper): the n-th
 * device allocation the library makes from now on, in any context and
 * thread, fails as if the device were out of memory, so that the call making
 * it returns H2_ENOMEM; n = 0 switches the hook off, and it is off again
 * once it has fired.  A local update allocates everything it needs before
 * its first write to the matrix, so an H2_ENOMEM from h2_lowrank_update or
 * h2_batch_apply leaves the matrix unchanged (its rank capacity may have
 * grown) and frees what the call allocated; after one from
 * h2_lowrank_update_sequence every update of the sequence is either applied
 * whole or not at all.  h2_lr_factor and h2_mul may have changed the matrix
 * when they fail.  Returns H2_EINVAL for n < 0. */
h2_status h2_debug_fail_allocation(int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* H2GB_H */
