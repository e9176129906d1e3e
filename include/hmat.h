/*
 * hmat.h -- C ABI of the GB300 (sm_103a) H-matrix library: truncated
 * low-rank updates in the accumulated form of
 *   S. Boerm, "Hierarchical matrix arithmetic with accumulated updates"
 *   (arXiv:1703.09085),
 * used inside the H-LU factorisation of finite-difference matrices.
 *
 * Conventions for every entry point:
 *  - Return value: an hmat_status (HMAT_OK = 0).  No call aborts or throws
 *    across this boundary; hmat_last_error() gives the message of the last
 *    failure on the calling thread.
 *  - Matrices are column-major FP64.  "host" arguments are ordinary host
 *    pointers, "device" arguments are pointers into device memory of the
 *    context's GPU.  Buffers passed in stay owned by the caller; the library
 *    copies host inputs and uses device buffers in place where stated.
 *  - Objects (contexts, trees, H-matrices) are opaque, owned by the library
 *    and released by the matching *_destroy call.  An H-matrix lives in the
 *    context's device memory.
 *  - Calls taking a context run asynchronously on the context's CUDA stream
 *    unless stated otherwise; *_build, *_nodes, *_perm and hmat_stats are
 *    synchronous host calls.
 */
#ifndef HMAT_H
#define HMAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HMAT_OK = 0,
  HMAT_ERR_ARG = 1,        /* invalid argument or unsupported input          */
  HMAT_ERR_NOMEM = 2,      /* device or host allocation failed               */
  HMAT_ERR_SINGULAR = 3,   /* zero pivot in a dense leaf LU                   */
  HMAT_ERR_NONFINITE = 4,  /* NaN or Inf produced or met                      */
  HMAT_ERR_RANK = 5,       /* a truncated rank exceeded the block capacity    */
  HMAT_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up              */
  HMAT_ERR_CUDA = 7,       /* a CUDA runtime call failed                      */
  HMAT_ERR_INTERNAL = 9
} hmat_status;

typedef struct hmat_ctx hmat_ctx;
typedef struct hmat_ctree hmat_ctree;
typedef struct hmat_btree hmat_btree;
typedef struct hmat hmat;
typedef struct hmat_mlp hmat_mlp;

/* Options of the arithmetic.
 *  eps        truncation tolerance: every truncation keeps the smallest rank k
 *             with sum_{i>k} sigma_i^2 <= eps^2 sum_i sigma_i^2 (relative
 *             Frobenius, per block); the paper leaves "choose new rank k"
 *             open (Fig. rkadd).  eps = 0 keeps every nonzero singular value.
 *  max_rank   capacity of every low-rank block and accumulator (<= 0: 64).
 *             A truncation whose rank exceeds it keeps the first max_rank
 *             singular triplets and reports HMAT_ERR_RANK.
 *  precision  HMAT_FP64 or HMAT_MIXED (see hmat_lu).
 *  spin_limit iterations of a bounded device-side dependency wait before it
 *             gives up with HMAT_ERR_TIMEOUT (<= 0: library default).
 *  reuse_schedule  non-zero: hmat_lu keeps the task schedule it builds (host
 *             list, device copy and scratch arena) with the first matrix and
 *             reuses it when called again on the same matrices with the same
 *             trees, initial zero pattern, max_rank and precision (the
 *             schedule never depends on the values).  The kept schedule is
 *             freed with the matrix.
 *  predictor  rank predictor (hmat_mlp_*) sizing the randomised truncation's
 *             first sketch in HMAT_MIXED: max(predicted rank + 3, kz + 2)
 *             columns, kz the larger input rank; NULL: max(kz + 6, 8).  A
 *             sketch that misses too much is
 *             widened and, at its limit, replaced by the exact QR + SVD.
 *  record_training  non-zero: every exact truncation records its features
 *             and rank (see hmat_lu_training_data).
 *  seed       seed of the randomised sketches' Rademacher signs (0: a fixed
 *             default); results are reproducible for a given seed.
 *  mode       HMAT_ACCUMULATED (0, default): products collected in
 *             accumulators and truncated once per block and flush (Section 4,
 *             Figs. addproduct, split, flush); HMAT_STANDARD (1): every
 *             product of a leaf pair applied at once by rkupdate (Section 4,
 *             the multiplication before "Accumulated updates"; the remark
 *             after the complexity theorem), for hmat_lu, hmat_lu_batched
 *             and hmat_addmul.
 *  rank_rule  HMAT_REL_FRO (0, default): the Frobenius rule above;
 *             HMAT_REL_SPEC (1): the smallest k with sigma_{k+1} <= eps
 *             sigma_1, available with precision HMAT_FP64 (HMAT_ERR_ARG with
 *             HMAT_MIXED, whose checks bound the Frobenius residual). */
enum { HMAT_FP64 = 0, HMAT_MIXED = 1 };
enum { HMAT_ACCUMULATED = 0, HMAT_STANDARD = 1 };
enum { HMAT_REL_FRO = 0, HMAT_REL_SPEC = 1 };
typedef struct {
  double eps;
  int64_t max_rank;
  int precision;
  int64_t spin_limit;
  int reuse_schedule;
  const hmat_mlp* predictor;
  int record_training;
  uint64_t seed;
  int mode;
  int rank_rule;
} hmat_opts;

typedef struct {
  int64_t n;              /* matrix dimension                                   */
  int64_t blocks;         /* block-tree nodes                                   */
  int64_t dense_leaves;
  int64_t lowrank_leaves;
  int64_t max_rank;       /* largest rank among admissible leaves               */
  double mean_rank;
  int64_t tasks;          /* device tasks of the last hmat_lu schedule          */
  int64_t truncations;    /* rank-revealing factorisations of the last hmat_lu  */
  double flops;           /* FP64 operations counted by the tasks of the last hmat_lu */
  double factor_seconds;  /* device time of the last hmat_lu numeric phase      */
  double schedule_seconds;/* host time of the last hmat_lu symbolic phase       */
  int64_t device_bytes;   /* device memory held by the H-matrix and its arena   */
  int status;             /* device status word of the last hmat_lu             */
  int64_t levels;         /* longest dependency chain of the schedule (tasks)   */
  double critical_flops;  /* estimated flops on the longest dependency chain    */
  double est_flops;       /* estimated flops of all tasks (static ranks)        */
  double type_seconds[16];/* summed CTA time per task type of the last hmat_lu  */
  int64_t type_count[16]; /* tasks run per task type                            */
  double wait_seconds;    /* summed CTA time waiting on predecessors            */
  int schedule_reused;    /* 1 if the last hmat_lu reused a kept schedule       */
  int64_t rand_truncations; /* truncations done by the randomised path (MIXED)  */
  int64_t rand_fallbacks;   /* randomised attempts that fell back to QR + SVD   */
  int64_t sketch_attempts;  /* sketches tried by the randomised truncations     */
  int64_t sketch_columns;   /* columns sketched over all those attempts         */
  int64_t training_pairs;   /* pairs recorded by the last hmat_lu               */
  /* Filled when the environment sets HMAT_PROFILE_TASKS=1: the measured
   * critical path (longest chain of task durations) and its make-up
   * (HMAT_PROFILE_PATH=<file> also writes the path's tasks as CSV). */
  double cp_seconds;
  double cp_type_seconds[16];
  int64_t cp_type_count[16];
  double flops32;           /* FP32 operations of the mixed path (flops: FP64)    */
  double bytes;             /* algorithmic bytes the tasks must move: stacked
                               factors read and truncated factors written
                               (8 [(m + n) l + (m + n) k] per truncation),
                               dense leaves and thin blocks read and written */
  int64_t gang_truncations; /* truncations of large blocks run by a gang of CTAs
                               (TSQR over row blocks; mixed form)             */
} hmat_stats;

/* Message of the last failure on this thread, copied into buf (NUL-terminated,
 * truncated to size).  Returns the full length. */
size_t hmat_last_error(char* buf, size_t size);

/* Context on CUDA device `device`, issuing work on `cuda_stream` (a
 * cudaStream_t, NULL for the legacy default stream).  The stream stays owned by
 * the caller and must outlive the context. */
hmat_status hmat_ctx_create(int device, void* cuda_stream, hmat_ctx** out);
hmat_status hmat_ctx_destroy(hmat_ctx* ctx);

/* Cluster tree (Section 2, Definition "Cluster tree") of n points in d = 2 or
 * 3 dimensions by geometric bisection: a cluster with more than leaf_size
 * points is split at the midpoint of its tight bounding box along the longest
 * side (first side on ties); points below the midpoint go to the first son,
 * order kept.  coords: host, n x d row-major.  Synchronous. */
hmat_status hmat_clustertree_build(hmat_ctx* ctx, const double* coords, int64_t n, int d,
                                   int64_t leaf_size, hmat_ctree** out);
/* perm[i] = original index of permuted index i (host, caller-owned, n). */
hmat_status hmat_clustertree_perm(const hmat_ctree* ct, int64_t* perm);
int64_t hmat_clustertree_size(const hmat_ctree* ct);
/* Per node (pre-order, root 0): first permuted index, size, level, parent
 * (-1 for the root), number of sons.  Host arrays of hmat_clustertree_size. */
hmat_status hmat_clustertree_nodes(const hmat_ctree* ct, int64_t* off, int64_t* size, int* level,
                                   int* parent, int* nsons);
hmat_status hmat_ctree_destroy(hmat_ctree* ct);

/* Block tree (Section 2, Definition "Block tree"): (t, s) is an admissible
 * leaf iff dist(t, s) > 0 and max(diam t, diam s) <= eta dist(t, s) (Euclidean
 * box diameter and distance); otherwise an inadmissible leaf if t or s is a
 * leaf, otherwise subdivided into sons(t) x sons(s).  Synchronous. */
hmat_status hmat_blocktree_build(hmat_ctx* ctx, const hmat_ctree* rows, const hmat_ctree* cols,
                                 double eta, hmat_btree** out);
int64_t hmat_blocktree_size(const hmat_btree* bt);
/* Per node (pre-order, root 0): row cluster, column cluster, level, parent,
 * kind (0 subdivided, 1 inadmissible/dense leaf, 2 admissible/low-rank leaf). */
hmat_status hmat_blocktree_nodes(const hmat_btree* bt, int* t, int* s, int* level, int* parent, int* kind);
hmat_status hmat_btree_destroy(hmat_btree* bt);

/* H-matrix on bt from a sparse matrix in CSR form in the ORIGINAL ordering
 * (host arrays rowptr[n+1], colidx[nnz], val[nnz]); the library permutes.
 * Admissible blocks start at rank 0; an entry inside an admissible block is
 * rejected with HMAT_ERR_ARG (finite-difference stencils have none there,
 * Section 3 opening paragraph).  The CSR arrays are copied to the device and
 * scattered into the dense leaves by a kernel. */
hmat_status hmat_create_from_csr(hmat_ctx* ctx, const hmat_btree* bt, int64_t n, const int64_t* rowptr,
                                 const int64_t* colidx, const double* val, hmat** out);
hmat_status hmat_destroy(hmat* H);

/* dst <- src, leaf values and ranks, for two H-matrices created on the same
 * block tree (device-to-device copy on the context stream).  Lets a caller
 * keep an unfactored matrix and factor fresh copies of it. */
hmat_status hmat_copy_values(hmat_ctx* ctx, hmat* dst, const hmat* src);

/* Dense copy of H in the permuted ordering into out (device, n x n, ld n). */
hmat_status hmat_to_dense(hmat_ctx* ctx, const hmat* H, double* out);

/* Y <- Y + alpha H X (trans = 0) or Y <- Y + alpha H^T X (trans = 1): the
 * multiplication by a thin dense matrix of Fig. addeval / addevaltrans.
 * X, Y: device, n x ncol, leading dimension n, permuted ordering. */
hmat_status hmat_addeval(hmat_ctx* ctx, const hmat* H, double alpha, int trans, int64_t ncol,
                         const double* X, double* Y);

/* In-place H-LU with accumulated updates: afterwards H holds the unit lower
 * factor L (strictly lower part) and the upper factor U.  The recursion is the
 * block LU with Schur complement of Section 6, accumulators split as in
 * Fig. invert, products added by Fig. addproduct, flushed by Fig. flush.
 * A host-side symbolic pass turns the recursion into a dependency-ordered task
 * list that one persistent kernel executes.  precision HMAT_FP64 runs every
 * task in FP64.  HMAT_MIXED with eps >= 1e-5 runs the truncations (QR of the
 * stacked factor, the projected block, pivoted-QR and Jacobi core, sketches
 * where used) and the leaf products and triangular solves in FP32 and keeps
 * FP64 for the leaf LU of the diagonal blocks, the stored factors and the
 * sums that decide the rank rule; every result still satisfies the rule of
 * hmat_opts.eps (a failed check falls back to the exact FP64 truncation).
 * HMAT_MIXED with eps < 1e-5 keeps FP64 truncations with FP32 sketches only.
 * Returns the device status (HMAT_ERR_SINGULAR, _RANK, _TIMEOUT, _NONFINITE)
 * after synchronising the stream. */
hmat_status hmat_lu(hmat_ctx* ctx, hmat* H, const hmat_opts* opts);

/* hmat_lu of count independent H-matrices (different trees and sizes allowed,
 * same context) in one schedule and ONE persistent kernel launch, so that the
 * instances fill the GPU together.  Each matrix is factored in place exactly
 * as by hmat_lu; the statistics of every instance report the batch's totals. */
hmat_status hmat_lu_batched(hmat_ctx* ctx, hmat** G, int count, const hmat_opts* opts);

/* H-matrix multiplication Z <- blocktrunc(Z + alpha X Y) (Section 4) with
 * accumulated updates (Section 4, Figs. addproduct, split, flush): the
 * product of the root blocks is entered
 * into an accumulator by addproduct (the four leaf cases produce low-rank
 * factors or dense blocks), split down the block tree of Z and flushed into
 * Z's leaves, so that every leaf of Z is truncated once per pending product
 * sum rather than once per product.  X, Y and Z must be distinct matrices of
 * this context built on block trees of ONE cluster tree (same index set and
 * ordering); X and Y are read only.  opts: eps (relative Frobenius rule per
 * truncation), precision, max_rank (capped by Z's leaf capacity), predictor,
 * spin_limit, record_training.  Runs as one persistent kernel launch and
 * synchronises the stream; Z's statistics describe the call.  Errors:
 * HMAT_ERR_ARG for aliasing or mismatched trees, device statuses as hmat_lu. */
hmat_status hmat_addmul(hmat_ctx* ctx, double alpha, const hmat* X, const hmat* Y, hmat* Z, const hmat_opts* opts);

/* In-place H-matrix inversion with accumulated updates (Section 6, Fig.
 * invert): G <- G^{-1}, by the recursion on the binary cluster tree with the
 * Schur complement S = G_22 - G_21 G_11^{-1} G_12, the updates of every block
 * held in accumulators (split, addproduct, flush) and each block truncated
 * once per flush.  Dense diagonal leaves are inverted by no-pivot LU (at most
 * 67 x 67; larger leaves give HMAT_ERR_INTERNAL).  The auxiliary blocks H_12,
 * H_21 live in an H-matrix allocated for the call.  opts as hmat_lu.  Runs as
 * one persistent kernel launch and synchronises the stream; G's statistics
 * describe the call.  Errors: HMAT_ERR_ARG for an admissible diagonal block or
 * a cluster with more than two sons, device statuses as hmat_lu. */
hmat_status hmat_invert(hmat_ctx* ctx, hmat* G, const hmat_opts* opts);

/* In-place H-Cholesky with accumulated updates for a symmetric positive
 * definite G (Section 6: treated like the inversion): chol(t1); L21 =
 * G21 L11^{-T}; L21^T mirrored into the (1,2) block; the Schur update
 * -L21 L21^T accumulated for the (2,2) block; chol(t2).  Afterwards the lower
 * blocks and the lower triangles of the diagonal leaves hold L (G = L L^T),
 * the upper ones L^T.  Dense diagonal leaves up to 96 x 96 (larger give
 * HMAT_ERR_INTERNAL); a non-positive pivot gives HMAT_ERR_SINGULAR.  opts as
 * hmat_lu; one persistent launch; synchronises the stream. */
hmat_status hmat_cholesky(hmat_ctx* ctx, hmat* G, const hmat_opts* opts);

/* Host-only analysis of the schedule hmat_lu would run for this matrix (no
 * device is touched): fills tasks, truncations (the schedule's truncation
 * tasks; at run time those of zero products are skipped), levels (longest
 * dependency chain),
 * critical_flops / est_flops (static estimates with rank 8 for unknown
 * ranks), schedule_seconds and the workspace size in device_bytes. */
hmat_status hmat_analyze_lu(const hmat_btree* bt, int64_t n, const int64_t* rowptr, const int64_t* colidx,
                            const double* val, const hmat_opts* opts, hmat_stats* out);

/* B <- (LU)^{-1} B (trans = 0) or (LU)^{-T} B (trans = 1) with the factors of
 * hmat_lu; B: device, n x nrhs, leading dimension ldb, permuted ordering. */
hmat_status hmat_solve(hmat_ctx* ctx, const hmat* LU, int trans, int64_t nrhs, double* B, int64_t ldb);

/* Preconditioned conjugate gradients for A X = B with the factors of
 * hmat_lu as the preconditioner z = (LU)^{-1} r (the paper measures the
 * factors' quality by ||I - (LU)^{-1} A||_2, Section 7; the CG count on an
 * SPD stiffness matrix is the practical form of that measure; Hestenes and
 * Stiefel's method, not in the paper).  A: the matrix the factors approximate,
 * host CSR in the ORIGINAL ordering (rowptr[n+1], colidx, val, copied).
 * B, X: device, n x nrhs column-major (ld n), original ordering; x_0 = 0.
 * Every column runs until ||r|| <= rtol ||b|| or maxit steps; iters and
 * relres (host, nrhs) receive the steps taken and the true relative residual
 * ||b - A x|| / ||b|| at the end.  The solves reuse one task schedule.
 * (LU)^{-1} of an SPD matrix is symmetric up to the truncation error, which
 * CG tolerates as long as that error is small.  Synchronous. */
hmat_status hmat_pcg(hmat_ctx* ctx, const hmat* LU, int64_t n, const int64_t* rowptr, const int64_t* colidx,
                     const double* val, int64_t nrhs, const double* B, double* X, double rtol, int64_t maxit,
                     int64_t* iters, double* relres);

/* Truncation of one low-rank matrix in place (Section 3, "Truncation"): with
 * R = U V^T, U (m x k, ldu) and V (n x k, ldv) in device memory, overwrite the
 * first k_new columns with the best approximation of the rank chosen by eps:
 * U <- left singular vectors, V <- right singular vectors times the singular
 * values (as Fig. rkadd returns C and D).  *k_new is written on the host after
 * the stream is synchronised.  k <= 512. */
hmat_status trunc_lowrank(hmat_ctx* ctx, int64_t m, int64_t n, int64_t k, double* U, int64_t ldu, double* V,
                          int64_t ldv, double eps, int64_t* k_new);

/* Batched truncation: count independent problems, problem i with sizes
 * m[i], n[i], k[i] (host arrays, k[i] <= 256) and factors at the device
 * pointers U[i] (ld m[i]) and V[i] (ld n[i]) (host array of device pointers).
 * k_new is a DEVICE array of count entries receiving the new ranks.  One CTA
 * per problem; the call synchronises the context stream before returning.
 * precision HMAT_MIXED (eps >= 1e-5, m n <= 2^20) first tries the FP32
 * randomised range finder of hmat_lu's mixed form (sketch, projection,
 * pivoted-QR and Jacobi core in FP32, the residual summed in FP64), keeping
 * the same Frobenius rule (its rank may exceed the optimal one by what the
 * sketch missed); a problem whose sketch misses too much falls back to the
 * exact QR + SVD.  *randomised (host, may be NULL) receives how many problems
 * the randomised path finished. */
hmat_status trunc_lowrank_batched(hmat_ctx* ctx, int64_t count, const int64_t* m, const int64_t* n,
                                  const int64_t* k, double* const* U, double* const* V, double eps,
                                  int64_t* k_new, int precision, int64_t* randomised);

/* trunc_lowrank without any memory allocation (the paper has no counterpart:
 * this serves callers that cannot let the library allocate device memory,
 * e.g. real-time hosts that reserve all device memory up front, where an
 * allocation mid-run could fail or stall, or applications whose own pool owns
 * the GPU and would lose track of memory taken behind its back).  Same
 * arguments, result and ld rules as trunc_lowrank (row count <= ld <=
 * 2^31 - 1 here; eps must be a number >= 0, else HMAT_ERR_ARG).  Its scratch
 * is a fixed 16 MiB device array compiled into the library, held by every GPU
 * that loads the library until exit; problems needing more than 2^21 - 32
 * doubles of scratch ((2m + n) k + 2 k^2) are rejected with HMAT_ERR_ARG.
 * The first call on a device looks the array's address up
 * (cudaGetSymbolAddress) and should come before any stream capture begins
 * on that device.  All calls share the array, so calls that overlap on the
 * GPU race: serialise them.  The call synchronises the context stream to
 * return *k_new. */
hmat_status trunc_lowrank_noalloc(hmat_ctx* ctx, int64_t m, int64_t n, int64_t k, double* U, int64_t ldu, double* V,
                                  int64_t ldv, double eps, int64_t* k_new);

/* Training pairs recorded by the last hmat_lu with record_training (kept with
 * the batch's first matrix): X (host, max x 6 floats, row-major) receives the
 * predictor's features of the block t x r (log2 #t / 10, log2 #r / 10,
 * log(dbar / (dist + 1e-3 dbar)) / 4 with dbar the mean of the clusters'
 * diameters, dimension / 3, l / 16 with l the rank of the sum before
 * truncation, log10(eps) / 4),
 * y (host, max) log(1 + rank);
 * *count = number of pairs held (copies min(max, count)). */
hmat_status hmat_lu_training_data(const hmat* H, int64_t max, float* X, float* y, int64_t* count);

/* Rank predictor: 3-layer MLP (6 -> 64 -> 64 -> 1, ReLU), BF16 weights and FP32
 * accumulation, predicting log(1 + truncated rank) from the features above.
 * Parameters: 4673 FP32 masters (W1[64][6], b1[64], W2[64][64], b2[64],
 * w3[64], b3), evaluated through their BF16 copy.  Created with He-uniform
 * weights from a counter-based generator seeded by seed. */
hmat_status hmat_mlp_create(hmat_ctx* ctx, uint64_t seed, hmat_mlp** out);
hmat_status hmat_mlp_destroy(hmat_mlp* M);
hmat_status hmat_mlp_get_params(const hmat_mlp* M, float* out);
hmat_status hmat_mlp_set_params(hmat_mlp* M, const float* in);
/* y[i] = network(X[i]) for count feature rows (host arrays). */
hmat_status hmat_mlp_forward(const hmat_mlp* M, int64_t count, const float* X, float* y);
/* Mean squared error over the rows and its gradient (4673 floats, host) by
 * the library's backward kernel. */
hmat_status hmat_mlp_grad(hmat_mlp* M, int64_t count, const float* X, const float* y, float* loss, float* grad);
/* Adam (lr, beta 0.9 / 0.999) on minibatches of size batch, epochs passes over
 * a seeded shuffle; *final_loss (may be NULL) = MSE on the whole set after. */
hmat_status hmat_mlp_train(hmat_mlp* M, int64_t count, const float* X, const float* y, int epochs, int batch,
                           float lr, uint64_t seed, float* final_loss);

/* Statistics of H and of its last hmat_lu (synchronous). */
hmat_status hmat_stats_get(const hmat* H, hmat_stats* out);

/* Per block-tree node: rank of an admissible leaf, -1 otherwise (host array). */
hmat_status hmat_ranks(const hmat* H, int64_t* ranks);

#ifdef __cplusplus
}
#endif
#endif /* HMAT_H */
