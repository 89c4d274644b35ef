/*
 * iaskit.h - C ABI of the GB300 INV-ASKIT library (libiaskit.so).
 *
 * INV-ASKIT (Yu, March, Xiao, Biros, arXiv 1602.01376) factorizes lambda*I + K~,
 * where K~ = D + UV is ASKIT's hierarchical approximation of the Gaussian kernel
 * matrix K_ij = exp(-||x_i - x_j||^2 / (2 h^2)) (Sec. I, eq. gaussian; Sec. II-A,
 * II-B), and then solves (lambda*I + K~) w = u in O(N log N) (Sec. II-C, Alg.
 * "Factorize" and Alg. "Solve").  The calls follow the paper's problem statement
 * (Sec. II-C, first paragraph): given the points, the bandwidth h, the
 * regularization lambda, the leaf size m and the skeleton budget, build the tree,
 * K~ and its factorization; then apply (lambda*I + K~)^{-1} to right-hand sides.
 *
 * Conventions shared by every call
 *  - Every step runs on the current CUDA device in this library's kernels; there
 *    is no CPU fallback.  If no device is usable the call returns IASKIT_ERR_CUDA.
 *  - All int-returning calls return IASKIT_OK (0) or a negative error code and
 *    never abort; iaskit_last_error() describes the last failure.
 *  - Matrices are column-major FP64.  Points are row-major: point i occupies
 *    points[i*d .. i*d + d - 1].  Right-hand sides and solutions are N x nrhs
 *    column-major in the ORIGINAL point order (the tree permutation is internal).
 *  - One implicit factorization is held by the library.  It is owned by the
 *    library until iaskit_free() or the next iaskit_factor* (iaskit_refactor
 *    replaces its lambda-dependent part in place); the library never keeps a
 *    caller pointer after a call returns.
 *  - Calls are synchronous: they return after the device work they enqueued has
 *    finished.  Work is enqueued on the stream set by iaskit_set_stream (default:
 *    the legacy default stream).
 *  - Not thread-safe: serialize calls from several host threads.
 */
#ifndef IASKIT_H
#define IASKIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define IASKIT_OK 0
#define IASKIT_ERR_ARG (-1)           /* invalid argument (sizes, h <= 0, lambda < 0, ...) */
#define IASKIT_ERR_INPUT (-2)         /* non-finite point or right-hand-side entry */
#define IASKIT_ERR_NOMEM (-3)         /* device allocation failed or memory cap exceeded */
#define IASKIT_ERR_SINGULAR (-4)      /* exact zero pivot in a leaf LU or a reduced system */
#define IASKIT_ERR_NOT_FACTORED (-5)  /* solve/apply before a successful factor */
#define IASKIT_ERR_NOT_CONVERGED (-6) /* iterative refinement hit its sweep cap */
#define IASKIT_ERR_TIMEOUT (-7)       /* a bounded device-side wait expired */
#define IASKIT_ERR_CUDA (-8)          /* CUDA runtime error; see iaskit_last_error() */
#define IASKIT_ERR_UNSUPPORTED (-9)   /* valid request outside what this build supports */

/*
 * Build the tree, the kNN lists, the skeletons (ASKIT, Sec. II-B) and the
 * INV-ASKIT factorization (Sec. II-C, Alg. "Factorize") for N points in d
 * dimensions.
 *   points   HOST pointer, N*d doubles, row-major; copied to the device.
 *   N >= 2, d >= 1, h > 0, lambda >= 0, leaf_m >= 2 (leaf size m: the tree has
 *            L = min{l : ceil(N/2^l) <= m} levels below the root, Sec. II-A),
 *   s_max >= 1 (skeleton budget per node),
 *   tol      > 0: adaptive rank, the smallest s with |R_ss| <= tol*|R_00| in the
 *            column-pivoted QR of the sampled block (Sec. II-B "chosen adaptively");
 *            <= 0: fixed rank s = min(s_max, columns, sampled rows).
 * Errors: IASKIT_ERR_ARG, _INPUT (non-finite point), _NOMEM, _SINGULAR, _CUDA.
 * On error the previous factorization is released.
 */
int iaskit_factor(const double* points, int64_t N, int d, double h, double lambda,
                  int leaf_m, int s_max, double tol);

/* As iaskit_factor with a DEVICE pointer (caller-owned, e.g. a torch tensor). */
int iaskit_factor_device(const double* d_points, int64_t N, int d, double h, double lambda,
                         int leaf_m, int s_max, double tol);

/*
 * Factor nprob independent problems together (each with its own points, N, h and
 * lambda; shared d, leaf_m, s_max, tol).  Each problem gets exactly the tree, kNN
 * lists (searched among its own points), skeletons and factorization it would get
 * alone; the work of all problems at the same height above the leaves runs in the
 * same launches.  This is a batching of the paper's per-problem method (Sec. II-C);
 * the paper itself factors one problem at a time.
 *   points   HOST pointers, points[q] is N[q] x d row-major.
 * The kNN lists use kappa = min("kappa", min_q N[q] - 1) for every problem.
 * Errors as iaskit_factor.
 */
int iaskit_factor_batched(int nprob, const double* const* points, const int64_t* N, int d,
                          const double* h, const double* lambda, int leaf_m, int s_max, double tol);

/* As iaskit_factor_batched with one DEVICE array holding the problems' points one
 * after the other (sum_q N[q] rows of d doubles). */
int iaskit_factor_batched_device(int nprob, const double* d_points, const int64_t* N, int d,
                                 const double* h, const double* lambda, int leaf_m, int s_max,
                                 double tol);

/* Number of problems of the current factorization, or a negative error. */
int iaskit_num_problems(void);

/*
 * Refactor for new regularizations (Sec. II-C: the skeletons and P do not depend on
 * lambda, so a new lambda recomputes only the leaf LUs, W and Z).  Keeps the tree, the
 * kNN lists, the samples, the skeletons and the P matrices of the current
 * factorization (single or batched) and forms lambda[q] I + K~ for each problem q
 * again: the leaf blocks and their LU, the U blocks, W and the reduced systems Z.  The
 * form ("precision") of the kept factorization is kept; the mixed form re-chooses each
 * problem's FP32/FP64 factorization and operator precision from its condition estimate
 * 1 + r_q / lambda[q] (r_q: the largest sampled kernel row sum).  The result is the
 * factorization iaskit_factor(_batched) would give for the same points and the new
 * lambdas.
 *   lambda   HOST pointer, nprob values >= 0, one per problem in batch order.
 *   nprob    must equal iaskit_num_problems().
 * Errors: IASKIT_ERR_NOT_FACTORED; _ARG (null pointer, wrong count, a negative or
 * non-finite value: the current factorization stays usable); _SINGULAR, _NOMEM,
 * _CUDA (the factorization is released).
 */
int iaskit_refactor(const double* lambda, int nprob);

/*
 * Solve (lambda*I + K~) w = u in place (Sec. II-C, Alg. "Solve").
 *   rhs      HOST pointer, N x nrhs column-major, original point order; on return
 *            it holds w.  nrhs >= 1.
 * With refinement on (option "refine" > 0, or the mixed precision), the solve refines
 * against the FP64 hierarchical operator: residuals r = u - (lambda I + K~) w in FP64,
 * corrections from restarted flexible GMRES on A z = r right-preconditioned by the
 * stored factorization M^-1, w += Z y with Z the kept vectors M^-1 v_j (FGMRES-IR).
 * A column is done when ||r||/||u|| <= "refine_tol", or when a cycle whose GMRES
 * estimate met 0.1 "refine_tol" lowered the recomputed residual by less than half, or
 * left it more than 100 times above that estimate: the rounding floor of the residual
 * (about 1e-16 ||A|| ||w|| / ||u|| in FP64) is then above the target; iaskit_stats
 * reports such columns as "refine_stagnated", each with its residual and that floor
 * estimate in "stagnated", and the last residuals in "refine_history".
 * "refine" bounds the total GMRES iterations; when they are spent with a column still
 * open the call returns IASKIT_ERR_NOT_CONVERGED and w holds the last iterate.
 * Errors: IASKIT_ERR_NOT_FACTORED, _ARG, _INPUT, _NOT_CONVERGED, _NOMEM, _CUDA.
 */
int iaskit_solve(double* rhs, int nrhs);

/* As iaskit_solve with a DEVICE pointer (N x nrhs, column-major, ld = N).  After a
 * batched factorization, d_rhs holds the problems' N[q] x nrhs column-major blocks one
 * after the other. */
int iaskit_solve_device(double* d_rhs, int nrhs);

/* Solve every problem of a batched factorization: rhs[q] is a HOST N[q] x nrhs
 * column-major block, overwritten with the solution.  Refinement, when on, runs
 * until every column of every problem meets "refine_tol". */
int iaskit_solve_batched(double* const* rhs, int nrhs);

/* As iaskit_solve_batched with one DEVICE array of all blocks one after the other. */
int iaskit_solve_batched_device(double* d_rhs, int nrhs);

/*
 * u = (lambda*I + K~) w by the FP64 hierarchical MatVec (Sec. II-B: the steps of
 * "Skeletonize" that depend on w, then "Evaluate" with the separation i not in alpha).
 *   w, u     HOST pointers, N x nrhs column-major, original point order; u is
 *            overwritten.  The pointers may not alias.
 * With option "near_field" = 1 the operator is lambda I + K~ + S (eq. askit): the nodes
 * of a target's Evaluate list that hold one of its nearest neighbours are evaluated
 * exactly instead of through their skeletons.
 * Errors: IASKIT_ERR_NOT_FACTORED, _ARG, _NOMEM, _CUDA.
 */
int iaskit_apply(const double* w, double* u, int nrhs);

/* As iaskit_apply with DEVICE pointers. */
int iaskit_apply_device(const double* d_w, double* d_u, int nrhs);

/*
 * Exact kernel sums at test points (Sec. III, "Kernel regression for binary
 * classification": a test point x gets the label sign(K(x, X) w), K(x, X) the exact
 * kernel row over all training points; at training points the same sums give the exact
 * K w of the error eps_M, eq. (error)):
 *   scores(i, r) = sum_j exp(-|test_i - x_j|^2 / (2 h^2)) w(j, r)
 * over every point x_j of the factored problem (the one selected by option "problem"
 * in a batch), with that problem's h.  Not an approximation: no skeletons are used.
 *   test     HOST pointer, M x d row-major FP64 (d of the factorization), caller-owned.
 *   w        HOST pointer, N x nrhs column-major, the problem's original point order
 *            (e.g. the weights returned by iaskit_solve).
 *   scores   HOST pointer, M x nrhs column-major, overwritten.
 * FP64 in the Gram form |x|^2 + |y|^2 - 2 x.y (relative error of a kernel value about
 * 2^-52 (|x|^2 + |y|^2) / (2 h^2)); chunk partial sums are added in a fixed order, so
 * repeated calls return identical scores.  M = 0 is a no-op.  1 <= nrhs <= 4096.
 * Errors: IASKIT_ERR_NOT_FACTORED, _ARG, _INPUT (non-finite test point or weight),
 * _NOMEM, _CUDA.
 */
int iaskit_predict(const double* test, int64_t M, const double* w, int nrhs, double* scores);

/* As iaskit_predict with DEVICE pointers (test M x d, w N x nrhs, scores M x nrhs). */
int iaskit_predict_device(const double* d_test, int64_t M, const double* d_w, int nrhs, double* d_scores);

/*
 * Options (set before iaskit_factor* unless noted):
 *   "kappa"        neighbours per point for sampling (default 16)
 *   "samp_factor"  sampled rows per node = samp_factor * s_max, capped at N - |node| (2)
 *   "seed"         seed of the uniform-fill random stream (0)
 *   "refine"       max GMRES-IR iterations in iaskit_solve* (0 = plain solve in FP64,
 *                  200 in the mixed precision) [any time]
 *   "refine_tol"   relative residual target of refinement (1e-10) [any time]
 *   "mem_cap_gb"   refuse factorizations whose device footprint exceeds this (0 = none)
 *   "profile"      1: time every kernel class with CUDA events (reported by iaskit_stats)
 *                  and reset the counters; 0: stop timing [any time]
 *   "precision"    0: plain FP64 (default); 1: mixed - FP32 factorization with FP64 pivot
 *                  comparisons, FP64 operator, solves refined to "refine_tol".  In the
 *                  mixed precision a problem whose estimated condition number
 *                  1 + max_i sum_j K(x_i, x_j) / lambda (64 sampled rows i) exceeds
 *                  "mixed_cond_max" is factored in FP64 instead
 *   "mixed_cond_max" condition estimate above which the mixed precision factors a
 *                  problem in FP64 (1e6, >= 1)
 *   "sampling"     0: kNN + uniform rows (Sec. II-B, default); 1: learned proposal
 *                  judged per node against the plain sample (needs weights)
 *   "cand_factor"  learned candidates per sampled row (8, 2..64)
 *   "keep_candidates" 1: keep candidates, features and scores for iaskit_get_learned (0)
 *   "train_batch"  rows per Adam step of iaskit_sampler_train (4096)
 *   "learned_temp" Gumbel temperature of the learned selection (0 = top scores, default)
 *   "gemm_tc"      1: FP32 products with more than 16 columns run on the tensor cores as
 *                  three TF32 products (hi.hi + hi.lo + lo.hi), about FP32 accuracy
 *                  (default); 0: FP32 CUDA-core tiles [any time]
 *   "pair_cond_max" mixed precision: the operator blocks (leaf blocks, U, P) are
 *                  evaluated and applied as FP32 pairs (hi + lo, about 2^-44 relative
 *                  per entry), except for problems whose condition estimate exceeds
 *                  this, which keep them in FP64 (default 1e5: measured pair floors
 *                  were below 4e-13 at estimate 1.9e4 and 4.6e-9 at 4.5e5, against
 *                  the default 1e-10 target; problems factored in FP64 are above it).  When a solve's
 *                  refinement stops at the pair operator's rounding floor above
 *                  "refine_tol", those problems' blocks are re-evaluated in FP64 and the
 *                  solve is refined again ("operator_upgrades" in iaskit_stats) [>= 1]
 *   "cpqr_cluster" 1: FP32 IDs of blocks up to 512 x 512 run on a cluster of up to 8
 *                  thread blocks per node, the columns held in registers (default);
 *                  0: one thread block per node.  Same arithmetic either way.
 *   "lu_inverse"   mixed precision: FP32 LUs inverted once after they are factored
 *                  (GETRI, A^-1 = U^-1 L^-1 P), their solves in Alg. "Solve" (in W =
 *                  D^-1 U and in iaskit_solve) then multiply by the inverses: FP32
 *                  products on the tensor cores instead of triangular solves, 4 more
 *                  bytes per inverted entry.  2: the leaf blocks lambda I + K_aa and the
 *                  reduced systems Z up to height "lu_inverse_zh" (default); 1: the leaf
 *                  blocks only; 0: LU solves throughout.  Products by an FP32 inverse
 *                  are not backward stable: inverses of the Zs above height 1 raised the
 *                  refinement's iterations (10 -> 16 on the manifold in d 64).  All are
 *                  FP32 solves whose error the refinement removes [before iaskit_factor]
 *   "lu_inverse_zh" with lu_inverse 2: the greatest height whose reduced systems are
 *                  inverted (1; leaves are height 0) [before iaskit_factor]
 *   "near_field"   1: the operator is the kNN-separated lambda I + K~ + S of eq. (askit)
 *                  (Sec. II-B): for each target i, a node that the Evaluate step reaches
 *                  for i (the sibling of an ancestor of i's leaf) and that holds one of
 *                  i's kappa nearest neighbours is evaluated exactly, K_{i a} w_a,
 *                  instead of through its skeletons.  iaskit_apply applies it and the
 *                  refinement's GMRES solves with it, preconditioned by the stored
 *                  factorization of lambda I + K~ (the paper's use of INV-ASKIT for
 *                  K~ + S); set "refine" > 0 for the plain form, whose direct solve
 *                  alone inverts lambda I + K~ only.  0: lambda I + K~ (default)
 *                  [any time after a factorization]
 *   "problem"      which problem of a batch the introspection calls report (0) [any time]
 *   "knn_prune"    1: the kNN lists are searched with the points in the order of a
 *                  tree with leaves of at most 128 points: each block of 128 queries
 *                  scans the 8 tiles whose bounding boxes lie nearest its own, then
 *                  only the tiles whose boxes come within its queries' largest kappa-th
 *                  distance so far; the skipped tiles enter the certification of the
 *                  exact re-rank (default).  0: every pair is scanned.  The lists are
 *                  identical either way [any time]
 *   "inner_pair"   mixed precision, problems with FP64 operator blocks: 1 the operator
 *                  applies inside each GMRES cycle form their FP64 products on FP32 pairs
 *                  (about 2^-44 relative) and a cycle aims at 1e-7 of its starting
 *                  residual, while every cycle's residual is recomputed with FP64
 *                  products, so the solution is the FP64 operator's; 0 (default): every
 *                  apply in FP64 (splitting FP64-stored blocks into pairs costs FP64
 *                  instructions: no faster on C4) [any time]
 *   "op_slices"    mixed precision, problems with FP64 operator blocks: 1 (default) the
 *                  operator's products run on the BF16 tensor cores by exact slicing
 *                  (Ozaki's error-free splitting): each block row and right-hand-side
 *                  column is scaled by a power of two and split into 8 signed 8-bit
 *                  digits (63 bits, |error| <= 2^-64 of the row's or column's largest
 *                  value), digit products are summed exactly in FP32 on the tensor cores
 *                  over segments of 128 values and recombined in 64-bit integers and
 *                  FP64; the digits of the operator blocks and of P are kept beside the
 *                  FP64 ones (16 bytes per entry) and built at the first apply after a
 *                  factorization; 0: FP64 products on the FP64 pipe.  Not used by the
 *                  inner applies of "inner_pair" [any time]
 *   "kernel"       the kernel of the next factorization: 0 the Gaussian of eq.
 *                  (gaussian), exp(-|x - y|^2 / (2 h^2)) (default); 1 the polynomial
 *                  kernel (x . y / h^2 + "poly_c")^"poly_p" (Sec. IV reports tests with a
 *                  polynomial kernel and gives no degree or constants; these are this
 *                  library's).  The factorization keeps its kernel: apply, solve,
 *                  predict and refactor use it whatever the option says later.  Learned
 *                  sampling is built for the Gaussian and returns IASKIT_ERR_UNSUPPORTED
 *                  with the polynomial kernel [0, 1]
 *   "poly_p"       polynomial degree (2) [1 .. 16]
 *   "poly_c"       polynomial constant (1.0) [>= 0]
 *   "inject_status" failure-path test hook: device status flags (1 zero pivot, 2
 *                  non-finite input, 4 internal bound, 8 expired bounded wait) that the
 *                  host ORs into the library's device status word just before its next
 *                  status read, exactly where a kernel would have set them; the call in
 *                  progress then returns the matching error (8: IASKIT_ERR_TIMEOUT).
 *                  One-shot: cleared once injected.  No kernel is made to fail [0..15]
 * Errors: IASKIT_ERR_ARG for an unknown key or an invalid value.
 */
int iaskit_set_option(const char* key, double value);
int iaskit_get_option(const char* key, double* value);

/* Stream for all later work (a cudaStream_t passed as void*; NULL = default). */
int iaskit_set_stream(void* cuda_stream);

/*
 * JSON with timings per phase (ms), the rank profile, algorithmic flop and byte
 * counts, the last refinement history (worst relative residual after each cycle), GMRES
 * iterations, columns stopped at the rounding floor, each problem's condition estimate
 * how many problems were factored in FP64 and how many kept their operator blocks in
 * FP64 (mixed precision).  Writes at most len bytes including the
 * terminating NUL; returns the full length needed (>= 0) or a negative error.
 */
int iaskit_stats(char* json_buf, size_t len);

/* Human-readable description of the last error (static storage, never NULL). */
const char* iaskit_last_error(void);

/* Release the factorization and all device memory held by the library. */
void iaskit_free(void);

/*
 * Introspection of the current factorization (tests compare these with the
 * oracle), for the problem selected by the option "problem".  Node (l, i) has heap
 * id 2^l + i, l = 0 .. depth.  Indices and positions are local to that problem.  All
 * outputs are HOST buffers.  Errors: IASKIT_ERR_NOT_FACTORED, _ARG (bad node or
 * short buffer).
 */
int iaskit_depth(void);                                 /* L, or a negative error */
int iaskit_get_perm(int32_t* perm);                     /* N: perm[pos] = original index */
int iaskit_get_knn(int32_t* knn, int kappa_cap);        /* N x kappa row-major, original ids */
int iaskit_get_ranks(int32_t* ranks, int count);        /* per heap id (count = 2^(L+1)); root = 0 */
/* Skeletons of node (l, i) as permuted positions in pivot order; returns s or error. */
int iaskit_get_skeleton(int level, int index, int32_t* skel, int cap);
/* Sampled rows of node (l, i) as ascending permuted positions; returns the count. */
int iaskit_get_samples(int level, int index, int32_t* samp, int cap);
/* Nested P of node (l, i): s x n_cols column-major; returns n_cols. */
int iaskit_get_P(int level, int index, double* P, int64_t cap);

/*
 * One kernel block, by default the Gaussian K(x_rows, x_cols) = exp(-|x_i - x_j|^2 / (2 h^2))
 * (Sec. I), plus diag where the row and column point are the same, evaluated by the
 * library's kernel-block kernels (independent of any factorization):
 *   form 0  FP64, Gram form |x|^2 + |y|^2 - 2 x.y (the plain form's blocks)
 *   form 1  FP32 pairs, difference form, exp on pairs (the mixed form's operator
 *           blocks); returned as hi + lo
 *   form 2  FP32, difference form (the mixed form's sampled blocks)
 *   form 3  FP64 Gram form with the dot products on the BF16 tensor cores from 8-digit
 *           slices of the coordinates and a table-driven FP64 exp (about 1 ulp) (the mixed
 *           form's FP64 operator blocks under "op_slices"); Gaussian kernel and d <= 64
 *           only (else IASKIT_ERR_UNSUPPORTED)
 * With option "kernel" = 1 the block is the polynomial kernel's, (x_i . x_j / h^2 +
 * "poly_c")^"poly_p", from the dot product in the first three precisions.
 * points: HOST N x d row-major; rows[nr], cols[nc]: HOST point indices in [0, N);
 * out: HOST nr x nc column-major.  Errors: IASKIT_ERR_ARG (null pointer, bad size,
 * index or form), IASKIT_ERR_INPUT (non-finite coordinate), IASKIT_ERR_UNSUPPORTED
 * (form 3 outside its range), IASKIT_ERR_TIMEOUT (an expired bounded wait of form 3).
 */
int iaskit_kernel_block(const double* points, int64_t N, int d, double h, const int32_t* rows, int nr,
                        const int32_t* cols, int nc, double diag, int form, double* out);

/*
 * Learned row proposal for skeletonization.  The paper samples the rows of
 * K_{[1:N] alpha} with nearest-neighbour information plus uniform draws (Sec. II-B);
 * with option "sampling" = 1 each node whose sample is not its whole complement
 * also gets a learned sample, and keeps whichever of the two IDs has the smaller
 * held-out error (below).  Not in the paper.
 *   candidates  n_cand = min(cand_factor * n_samp, N - n) rows: at most n_cand / 2 kNN
 *               candidates in the plain order (hits descending, position ascending),
 *               then uniform draws without replacement from the complement on the
 *               node's LEARN stream;
 *   features    8 per candidate, from the column subset Y (at most 32 evenly spaced
 *               ID columns, mean mu, radius r = max ||y - mu||): log(1 + hits) /
 *               log(1 + kappa), ||x - mu|| / h, max and mean K(x, Y), level / L,
 *               log2 n / log2 N, min(||x - mu|| / r, 1e3), 0;
 *   score       MLP 8 -> 128 -> 128 -> 1, ReLU, BF16 operands, FP32 accumulation;
 *   selection   the n_samp highest keys (ties to the lower position), ascending; key =
 *               score + learned_temp * g, g = -log(-log(u)), u = ((r >> 11) + 1/2) 2^-53
 *               for draw r of the candidate's index on the node's GUMBEL stream (salt
 *               0x47554D42): a sample without replacement ~ exp(score / learned_temp);
 *   judge       64 stratified rows H on the HOLD stream (below); the ID of sample v
 *               (skeletons S_v, interpolation P_v) has error sum_h w_h ||K(h, cols) -
 *               K(h, S_v) P_v||^2 / sum_h w_h ||K(h, cols)||^2 (FP64); the learned ID
 *               is kept when its error is not larger than the plain one's.
 * Stream of a node: s0 = splitmix64(splitmix64(seed ^ salt) ^ (2^l + i)), draw q =
 * r_q = splitmix64(s0 + q * 0x9E3779B97F4A7C15); salts LEARN 0x4C4541524E, HOLD
 * 0x484F4C44, GRAM 0x4752414D.  Candidate draws take j = r mod (N - n) as position j
 * (j < offset) or j + n.  A stratified draw of c rows takes its first c/2 (all of them
 * when the parent is the root) from the sibling, position sib_offset + r mod |sib|,
 * and the rest from outside the parent, j = r mod (N - |parent|) taken as j or
 * j + |parent|; a row weighs its stratum's size over the stratum's draws.
 * Weights: 17793 FP32 values in the order W1 [128][8] (row = hidden unit), b1 [128],
 * W2 [128][128] (row = output unit), b2 [128], w3 [128], b3.
 */

/* Trains the proposal on one problem (host points, N x d row-major): factors it in
 * FP64 with plain sampling (lambda = 1; that factorization becomes the current one),
 * labels every candidate of every node with its ridge leverage b^T (G + mu I)^{-1} b
 * (b = K(x, cols), G = B^T diag(w) B over 4096 stratified GRAM-stream rows B with
 * weights w, mu = tol^2 trace G), standardizes the log labels per node, then runs
 * `epochs` epochs of
 * Adam (beta 0.9, 0.999, eps 1e-8, step lr) on the mean squared error in batches of
 * option "train_batch" shuffled rows.  Starts from the current weights if any, else a
 * He-uniform draw.  Errors: IASKIT_ERR_ARG, _INPUT, _NOMEM, _SINGULAR, _CUDA. */
int iaskit_sampler_train(const double* points, int64_t N, int d, double h, int leaf_m, int s_max,
                         double tol, int epochs, double lr);
/* Replace (n = 17793, host FP32) or read the weights; setting clears Adam's state. */
int iaskit_sampler_set_weights(const float* w, int n);
int iaskit_sampler_get_weights(float* w, int n);
/* Scores of n host feature rows (n x 8 FP32, rounded to BF16 on upload). */
int iaskit_mlp_forward(const float* feats, int64_t n, float* scores);
/* One training step on n host rows: forward, gradient of the mean squared error
 * (written to grad, 17793 floats, if not NULL; loss to *loss if not NULL), then one
 * Adam update with step lr. */
int iaskit_mlp_train_step(const float* feats, const float* targets, int64_t n, double lr, float* grad,
                          float* loss);
/* Candidates of node (l, i) kept by the last factorization or training (option
 * "keep_candidates" = 1): positions (permuted, problem-local), features (n x 8, the
 * BF16 values) and the selection keys (factorization) or training targets; info[4] = {plain
 * held-out error, learned held-out error, 1 if the learned ID was kept (0 if not, -1
 * when not judged), n_samp}.  Returns the candidate count (0 if the node had none). */
int iaskit_get_learned(int level, int index, int32_t* cand, float* feat, float* value, int cap,
                       double* info);

/*
 * Autotuning of the grouped GEMM (the batched products of the factorization, the solve
 * and the operator apply; the paper has no counterpart: a tile-shape table of this
 * library).  Its CUDA-core tile shapes, 0 = 64 x 64, 1 = 256 x 16, 3 = 128 x 32 and
 * 4 = 512 x 8 (FP32 only), all sum each output over k in the same order, so a shape
 * changes the speed of a launch and never its result.  A launch that is not on the
 * tensor cores or on FP32 pairs takes the shape of its bucket:
 *   fp64      1 for FP64 products, 0 for FP32;
 *   n_bucket  0 .. 5: the launch's largest column count N in (8 << (b-1), 8 << b]
 *             (bucket 0 up to 8, bucket 5 above 128);
 *   m_bucket  0 .. 4: its largest row count M in (128 << (b-1), 128 << b]
 *             (bucket 0 up to 128, bucket 4 above 1024).
 * iaskit_gemm_tile installs `shape` for a bucket (-1 removes the entry; without an
 * entry the default rule holds: 256 x 16 up to 16 columns, else 64 x 64).
 * iaskit_tune_gemm times one grouped launch of `count` M x N x K problems (zero data,
 * library scratch) with `shape`: *ms = mean milliseconds over `reps` launches after
 * one warm-up.  The binding's autotune module sweeps every bucket with it and writes
 * the table that the binding installs when it loads the library.
 * Errors: IASKIT_ERR_ARG (bad bucket, a shape this type lacks, sizes above 4 GB),
 * _NOMEM, _CUDA.
 */
int iaskit_gemm_tile(int fp64, int n_bucket, int m_bucket, int shape);
int iaskit_tune_gemm(int fp64, int M, int N, int K, int count, int shape, int reps, double* ms);

/*
 * The kNN lists of iaskit_factor (same order, same ties, bit for bit) for callers
 * that must not allocate device memory: for example a serving process whose
 * device memory is entirely handed out by its own pool allocator, or a caller
 * that cannot accept the device-wide synchronization that cudaMalloc/cudaFree may
 * imply.  The paper has no counterpart; this is a library convenience.
 *   d_points  DEVICE pointer, N x d row-major FP64 (caller-owned).
 *   d_knn     DEVICE pointer, N x kappa row-major int32 output (original indices).
 *   cuda_stream  stream to run on (NULL = default stream); the call returns after
 *             the work has finished.
 * Limits: 2 <= N <= 32768, 1 <= d <= 64, N*d <= 1048576, 1 <= kappa <= min(24, N-1);
 * anything larger returns IASKIT_ERR_ARG with the limit in iaskit_last_error().
 * Scratch: one static device array of about 37.3 MiB, which every GPU that loads
 * this library holds until the process exits.  The call makes no device
 * allocation.  Its first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) once, under a lock, so host threads may make that first
 * call concurrently.  The call copies from host memory, reads a count back and
 * synchronizes the stream before it returns, so it cannot be recorded into a CUDA
 * graph.  All calls share the array, so calls that overlap on the GPU (other
 * streams or threads) race; serialize them.
 * Errors: IASKIT_ERR_ARG, _UNSUPPORTED, _CUDA.
 */
int iaskit_knn_noalloc(const double* d_points, int64_t N, int d, int kappa, int32_t* d_knn,
                       void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* IASKIT_H */
