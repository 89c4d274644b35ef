// Host launchers of the INV-ASKIT device kernels.  Each launcher enqueues work on
// `st` and returns immediately; errors of the launch itself throw iaskit::Error.
#pragma once
#include <initializer_list>

#include "common.cuh"
#include "kspec.cuh"

namespace iaskit {

// The kernel spec of the translation units that evaluate kernel values (kspec.cuh);
// the solver sets all of them together.
void kspec_set_dense(const KernelSpec& k, cudaStream_t st);
void kspec_set_near(const KernelSpec& k, cudaStream_t st);
void kspec_set_predict(const KernelSpec& k, cudaStream_t st);

// ------------------------------------------------------------------ tree (a1)
// Scratch buffers of the tree build.
struct TreeScratch {
  DevBuf keys, vals, alt_keys, alt_vals, hist, scan_tmp, flags, pre, minmax, dims, perm2, offs;
  void release() {
    for (DevBuf* b : {&keys, &vals, &alt_keys, &alt_vals, &hist, &scan_tmp, &flags, &pre, &minmax,
                      &dims, &perm2, &offs})
      b->release();
  }
};

// One step of the tree build: nodes covering [0, N) in order; node j owns
// [off[j], off[j+1]).  A split node sends the kleft[j] = floor(n/2) points that come
// first in (x_c, original index) order to its left child; a node that is not split
// has kleft[j] = n and keeps its points in place.
struct TreeLevel {
  std::vector<int> off;
  std::vector<int> kleft;
  std::vector<char> split;
};

// Median split on the coordinate of largest spread, one step per level (Sec. II-A).
// X: N x d row-major (original order, device).  Writes perm (device, N):
// perm[pos] = original index.
void build_tree(const double* X, int N, int d, const std::vector<TreeLevel>& levels, int* perm,
                TreeScratch& s, cudaStream_t st);

// iperm[perm[p]] = p and Xp[p] = X[perm[p]] (rows of d doubles).
void permute_points(const double* X, const int* perm, int N, int d, int* iperm, double* Xp,
                    cudaStream_t st);

// ------------------------------------------------------------------- kNN (a2)
struct KnnScratch {
  DevBuf x32, qnorm, part, mean, rmax, probs, cand_d, cand_i, flagged, counter, tiles, status, seed_tiles, seeds,
      first, box, tau, tq, cnt, toff, tlist, rec, tnorm, bits, boxT, sbox, fgrp, grps;
  void release() {
    for (DevBuf* b : {&x32, &qnorm, &part, &mean, &rmax, &probs, &cand_d, &cand_i, &flagged, &counter,
                      &tiles, &status, &seed_tiles, &seeds, &first, &box, &tau, &tq, &cnt, &toff, &tlist, &rec,
                      &tnorm, &bits, &boxT, &sbox, &fgrp, &grps})
      b->release();
  }
};

// Rows per prefilter tile of the kNN search (and leaf size of its search-order tree).
constexpr int KNN_TILE = 128;

// What the pruned search scanned: point tiles after the seed windows, query-point
// pairs scanned in all, and the pairs of a brute-force search.
struct KnnPruneStats {
  int64_t tiles_scanned = 0;
  double pairs_scanned = 0.0, pairs_all = 0.0;
};

// Work tile of the kNN kernels: queries [q0, q0 + qn) against the points
// [rb, rb + rn) of their problem `prob`.
struct KnnTile {
  int q0, qn, rb, rn, prob;
};

// kappa nearest neighbours of every point by (squared distance, index), self
// excluded, distance = sum_k (x_k - y_k)^2 in FP64 with every operation rounded
// (no contraction), k in order; neighbours are searched among the points of the
// same problem only.  X is N x d row-major FP64 (original order, all problems
// concatenated); problems lists (first point, point count).  knn: N x kappa int32
// (original indices).  Returns the number of queries that needed the exact
// fallback scan.
int knn_bruteforce(const double* X, int N, int d, int kappa, int* knn,
                   const std::vector<std::pair<int, int>>& problems, KnnScratch& s,
                   cudaStream_t st);

// The same lists (bit for bit) from points held in tree order, Xp = X[perm] (perm[r] =
// original index of row r, problems as row ranges of Xp), by the tensor-core prefilter
// over each 128-query block's seed tiles (the 8 tiles whose bounding boxes lie nearest
// its own), then only over the tiles whose boxes come within the block's bound (an
// exact upper bound on its queries' kappa-th distances); the skipped tiles enter the
// certification of the exact re-rank.  Returns the number of queries redone by the
// exact scan.
int knn_tree(const double* Xp, const int* perm, int N, int d, int kappa, int* knn,
             const std::vector<std::pair<int, int>>& problems, KnnScratch& s, cudaStream_t st,
             KnnPruneStats* pstats = nullptr);

// ------------------------------------------------------------- sampling (a3)
struct SampleScratch {
  DevBuf keys, alt_keys, alt_vals, hist, scan_tmp, flags, idx, run_start, run_end, run_key,
      keys2, vals2, node_cnt, node_start, status;
  void release() {
    for (DevBuf* b : {&keys, &alt_keys, &alt_vals, &hist, &scan_tmp, &flags, &idx, &run_start,
                      &run_end, &run_key, &keys2, &vals2, &node_cnt, &node_start, &status})
      b->release();
  }
};

// knn_pos[p*kappa + k] = iperm[knn[perm[p]*kappa + k]].
void knn_to_positions(const int* knn, const int* perm, const int* iperm, int N, int kappa,
                      int* knn_pos, cudaStream_t st);

// Per node of a sampling step: the node's problem (first point pb, point count pn),
// its heap id 2^l + i in its own tree, where its sample starts in `samp`, and
// whether it is sampled (0: points of a problem with no node at this step).
struct SampleNodeInfo {
  int pb, pn, uid, samp_off, active;
};

// Sampled rows of the nodes of one step (see the sampling rule in sampling.cu).
// off: device offsets (nn + 1) covering [0, N); n_samp of an active node =
// min(samp_cap, pn - size).
void sample_level(const int* knn_pos, int N, int kappa, const int* off_dev,
                  const SampleNodeInfo* info_dev, const std::vector<int>& off_host,
                  const std::vector<SampleNodeInfo>& info_host, int samp_cap, uint64_t seed,
                  int* samp, int* dev_status, SampleScratch& s, cudaStream_t st);

// ------------------------------------------------------- dense batched kernels
// All dense kernels are templated on the storage/arithmetic type T (double for
// the plain FP64 path, float for the mixed-precision form).

// Kernel block K(x_rows, x_cols) (+ diag where the row and column positions agree),
// column-major into out.  Rows: rows ? rows[i] : row0 + i.  Columns: colsA ?
// (j < nA ? colsA[j] : colsB[j - nA]) : col0 + j.  Points are positions in Xp.
// T = double evaluates in FP64 (Gram form with the precomputed squared norms);
// T = float evaluates distances (difference form) and exp in FP32.
// scale = -1 / (2 h^2) of the block's problem.
template <typename T>
struct KDescT {
  const int* rows;
  const int* colsA;
  const int* colsB;
  T* out;
  int row0, nrows, col0, nA, ncols, ld;
  double diag;
  double scale;
};
// xnorm: squared norms of the rows of Xp (FP64 blocks use them; may be null for FP32).
template <typename T>
void kernel_blocks(const double* Xp, const double* xnorm, int d, const KDescT<T>* descs_dev, int ndesc,
                   int64_t max_entries_per_desc, cudaStream_t st);
// The same blocks evaluated on FP32 pairs (coordinates Xpair = split Xp, d per point)
// and written as pairs: relative error a few 2^-48 per entry.
void kernel_blocks_pair(const float2* Xpair, int d, const KDescT<float2>* descs_dev, int ndesc,
                        int64_t max_entries, cudaStream_t st);
// out[i] = sum_k Xp[i][k]^2 in FP64, coordinates in order.
void point_norms(const double* Xp, int N, int d, double* out, cudaStream_t st);

// Column-pivoted Householder QR of each block (the ID's T follows with
// trsm_upper_batched).
// A (nrows x ncols, ld) is overwritten: its first s rows hold, in pivoted column
// order, R11 and T = R11^{-1} R12 in place of R12.  piv receives the column
// permutation; rank[0] receives s.  Column norms are accumulated in FP64 for both
// T, so pivot decisions are taken in FP64.
template <typename T>
struct CpqrDescT {
  T* A;
  int* piv;
  int* rank;
  int ld, nrows, ncols;
};
// cluster: FP32 blocks of up to 512 x 512 may run on a cluster of up to 8 blocks per
// node (the same arithmetic, columns held in registers across the cluster).
template <typename T>
void cpqr_id(const CpqrDescT<T>* descs_dev, int ndesc, int max_rows, int max_cols, int s_max,
             double tol, cudaStream_t st, bool cluster = false);

// Builds P (s x ncols, ld = s, FP64) from a cpqr_id result and the skeleton list
// skel[k] = cols[piv[k]] with cols as in KDescT (colsA/colsB/col0).
template <typename T>
struct PDescT {
  const T* A;  // cpqr output (ld)
  const int* piv;
  const int* colsA;
  const int* colsB;
  double* P;
  int* skel;
  int ld, ncols, s, nA, col0;
};
template <typename T>
void assemble_P(const PDescT<T>* descs_dev, int ndesc, int max_cols, cudaStream_t st);

// LU with partial pivoting (ties to the lowest row) of each n x n block in place,
// blocked (panel width 32, register-tiled trailing update), one CTA per matrix.
template <typename T>
struct LuDescT {
  T* A;
  int* ipiv;
  int n, ld;
  // optional (FP32): receives, per 32 x 32 diagonal block b, the inverse of L's unit
  // lower block and of U's upper block (row-major, 2 x 1024 values at 2048 b), then
  // the row permutation of the pivots as n ints (perm[i] = source row of row i).
  T* dinv;
};
// Values of a dinv area for an n x n LU (see LuDescT).
inline int64_t lu_dinv_size(int n) { return (int64_t)2048 * ((n + 31) / 32) + n; }
// inv: every descriptor carries a dinv area (FP32 only), filled after the LU.
template <typename T>
void getrf_batched(const LuDescT<T>* descs_dev, int ndesc, int max_n, int* dev_status,
                   cudaStream_t st, bool inv = false);

// B <- A^{-1} B from getrf output, for each descriptor; B is n x ncols (ldb).
template <typename T>
struct LuSolveDescT {
  const T* LU;
  const int* ipiv;
  T* B;
  int n, ldlu, ldb, ncols;
  const T* dinv;  // the LU's dinv area (see LuDescT), for getrs_batched(..., inv = true)
};
// inv: every descriptor carries its dinv area (FP32 only): the solve multiplies by the
// diagonal blocks' inverses instead of substituting through them.
// pair (FP64 only): the updates outside the 32 x 32 diagonal blocks run on FP32 pairs
// (about 2^-44 relative per 32-term sum); the diagonal substitutions stay in FP64.
template <typename T>
void getrs_batched(const LuSolveDescT<T>* descs_dev, int ndesc, int max_n, int max_cols,
                   cudaStream_t st, bool inv = false, bool pair = false);
// GETRI of FP32 LUs factored with their dinv areas: B (n x n, ldb) <- A^-1 for each
// descriptor (ncols is n; B must not overlap the LU).  Singular U gives non-finite
// entries, as the solve would.
void getri_batched(const LuSolveDescT<float>* descs_dev, int ndesc, int max_n, cudaStream_t st);
// B <- U^{-1} B with U the upper triangle of the n x n block at LU (ipiv unused): the
// ID's T = R11^{-1} R12 after cpqr_id.  A zero diagonal entry gives a zero row.
template <typename T>
void trsm_upper_batched(const LuSolveDescT<T>* descs_dev, int ndesc, int max_n, int max_cols,
                        cudaStream_t st);

// C <- alpha * A * B + beta * C (column-major, no transposes) for each descriptor.
template <typename T>
struct GemmDescT {
  const T* A;
  const T* B;
  T* C;
  int M, N, K, lda, ldb, ldc;
  double alpha, beta;
};
// Work items (descriptor index, tile row, tile column).  Tile shapes: 64 x 64
// (GEMM_SQUARE), 256 x 16 (GEMM_SKINNY), 128 x 128 (GEMM_TC), 128 x 32 (GEMM_WIDE) and
// 512 x 8 (GEMM_NARROW, FP32 only).  Every CUDA-core shape sums each output over k in
// the same order, so they give identical results; the autotuner picks among them.
struct GemmTile {
  int desc, tm, tn;
};
// GEMM_TC: 128 x 128 tiles on the tensor cores (tcgen05, 3xTF32), FP32 products only.
enum GemmShape { GEMM_SQUARE = 0, GEMM_SKINNY = 1, GEMM_TC = 2, GEMM_WIDE = 3, GEMM_NARROW = 4 };
constexpr int GEMM_NSHAPES = 5;
inline int gemm_tile_m(GemmShape s) {
  return s == GEMM_SKINNY ? 256 : s == GEMM_TC ? 128 : s == GEMM_WIDE ? 128 : s == GEMM_NARROW ? 512 : 64;
}
inline int gemm_tile_n(GemmShape s) {
  return s == GEMM_SKINNY ? 16 : s == GEMM_TC ? 128 : s == GEMM_WIDE ? 32 : s == GEMM_NARROW ? 8 : 64;
}
// A CUDA-core shape the grouped GEMM of this element type supports.
inline bool gemm_shape_valid(GemmShape s, bool fp64) {
  return s == GEMM_SQUARE || s == GEMM_SKINNY || s == GEMM_WIDE || (s == GEMM_NARROW && !fp64);
}
// Autotuned CUDA-core tile shapes, keyed by element type and the launch's largest N and
// M (buckets 0 .. GT_NB-1 of ceil(log2) above 8 resp. 128); -1 = no entry.
constexpr int GT_NB = 6, GT_MB = 5;
inline int gemm_n_bucket(int n) {
  int b = 0;
  while (b < GT_NB - 1 && n > (8 << b)) ++b;
  return b;
}
inline int gemm_m_bucket(int m) {
  int b = 0;
  while (b < GT_MB - 1 && m > (128 << b)) ++b;
  return b;
}
int& gemm_tuned(int fp64, int nb, int mb);
// dev_status: device status word; a tensor-core tile whose bounded wait expires sets
// DEV_TIMEOUT there and leaves its C tile unwritten.
template <typename T>
void gemm_grouped(const GemmDescT<T>* descs_dev, const GemmTile* tiles_dev, int ntiles,
                  GemmShape shape, cudaStream_t st, int* dev_status);

// dst (rows x cols, ldd) <- src (rows x cols, lds), batched.
template <typename T>
struct CopyDescT {
  const T* src;
  T* dst;
  int rows, cols, lds, ldd;
};
template <typename T>
void copy_batched(const CopyDescT<T>* descs_dev, int ndesc, int64_t max_entries, cudaStream_t st);

// Z'' = [[I, C_l], [C_r, I]] of size (s_l + s_r), ld = s_l + s_r.
template <typename T>
struct ZDescT {
  const T* Cl;  // s_l x s_r, ld s_l
  const T* Cr;  // s_r x s_l, ld s_r
  T* Z;
  int sl, sr;
};
template <typename T>
void form_Z(const ZDescT<T>* descs_dev, int ndesc, int64_t max_entries, cudaStream_t st);

using KDesc = KDescT<double>;
using CpqrDesc = CpqrDescT<double>;
using PDesc = PDescT<double>;
using LuDesc = LuDescT<double>;
using LuSolveDesc = LuSolveDescT<double>;
using GemmDesc = GemmDescT<double>;
using CopyDesc = CopyDescT<double>;
using ZDesc = ZDescT<double>;

// Elementwise conversions between FP64 and FP32 buffers.
void convert_d2f(const double* in, float* out, int64_t n, cudaStream_t st);
void convert_f2d(const float* in, double* out, int64_t n, cudaStream_t st);

// FP64 values as pairs of FP32 values: x = hi + lo with hi = fl32(x), lo = fl32(x - hi),
// so |x - hi - lo| <= 2^-48 |x| (for |x| inside the FP32 normal range).  out may alias
// in (element i of the pair array occupies the bytes of element i of the FP64 array).
void split_pairs(const double* in, float2* out, int64_t n, cudaStream_t st);

// C = alpha A B + beta C with A stored as FP32 pairs (M x K, column-major, lda in
// pairs) and B, C in FP64: every product is formed exactly (FMA error term) and the
// sums are kept as FP32 pairs (two-sum), so the result carries about 2^-44 relative
// error for K up to a few thousand, on the FP32 pipes.  Tiles of 256 x 16.
struct GemmDescPair {
  const float2* A;
  const double* B;
  double* C;
  int M, N, K, lda, ldb, ldc;
  double alpha, beta;
};
constexpr int GEMM_PAIR_TM = 256, GEMM_PAIR_TN = 16;
void gemm_pair_grouped(const GemmDescPair* descs_dev, const GemmTile* tiles_dev, int ntiles, cudaStream_t st);
// The same products with A in FP64 (split into pairs as it is loaded): FP64 inputs and
// output at about 2^-44 relative, on the FP32 pipes.  Tiles of gemm_tile_m(shape) x
// gemm_tile_n(shape) for GEMM_SKINNY (256 x 16) and GEMM_SQUARE (64 x 64).
void gemm_pair64_grouped(const GemmDesc* descs_dev, const GemmTile* tiles_dev, int ntiles, GemmShape shape,
                         cudaStream_t st);

// Row permutation of an N x ncols column-major block: out[p] = in[perm[p]] (gather)
// or out[perm[p]] = in[p] (scatter).
template <typename T>
void permute_rows(const T* in, int ldi, T* out, int ldo, const int* perm, int N, int ncols,
                  bool scatter, cudaStream_t st);

// u_rows += K(x_rows, x_cols) * y for each descriptor, kernel values recomputed in
// FP64 in the Gram form of kernel_blocks (xnorm: squared norms of the rows of Xp).  y is ncols x nrhs (ldy), u is nrows x nrhs (ldu) with rows starting at row0.
struct KMatvecDesc {
  const int* cols;
  const double* y;
  double* u;
  int row0, nrows, col0, ncols, ldy, ldu;
  double scale;  // -1 / (2 h^2)
};
void kernel_matvec(const double* Xp, const double* xnorm, int d, int nrhs, const KMatvecDesc* descs_dev,
                   int ndesc, int max_rows, cudaStream_t st);

// Exact kernel sums at M test points (Sec. III, kernel regression):
//   out[i + r ldo] = sum_j exp(-|t_i - x_j|^2 / (2 h^2)) w[orig(j) + r ldw]
// over the N points of one problem (Xp rows pbase .. pbase + N - 1, permuted order,
// xnorm their squared norms, perm[pbase + j] - pbase the original index of j), w in
// the problem's original order.  T: M x d row-major (device).  part: scratch of
// predict_scratch_doubles(M, N, nrhs) doubles.  FP64, Gram form; the kernel of the
// factorization (kspec), scale the problem's.
void predict_chunks(int M, int N, int& chunk, int& nchunk);
size_t predict_scratch_doubles(int M, int N, int nrhs);
void kernel_predict(const double* T, int M, const double* Xp, const double* xnorm, const int* perm, int pbase,
                    int N, int d, double scale, const double* w, int ldw, int nrhs, double* part, double* out,
                    int ldo, cudaStream_t st);

// Near-field correction of the kNN-separated operator (eq. askit, Sec. II-B).  For
// every target position p and every node alpha of p's interaction list (the sibling of
// each ancestor of p's leaf) that holds at least one of p's kappa nearest neighbours,
//   u_p += K(x_p, X_alpha) w_alpha - K(x_p, X_skel(alpha)) w~_alpha,
// i.e. the skeleton evaluation of alpha is replaced by the exact one (FP64, Gram form
// of the squared distance as kernel_blocks), grouped by node and tiled.
struct NearProb {
  int pbase, N, L, nbase;
  double scale;  // -1 / (2 h^2)
};
// masks[p] bit l (1 <= l <= L): the level-l node of target p's Evaluate list (the
// sibling of p's level-l ancestor) holds one of p's kappa nearest neighbours.
void near_masks(const int* knn_pos, int kappa, const int* pid, const NearProb* probs, int Ntot, unsigned* masks,
                cudaStream_t st);
// One tile of the exact-minus-skeleton sums: targets tgt[r0 .. r0 + 63] (global
// positions, n in all) against columns cols[0 .. ncols) (or col0 .. col0 + ncols - 1),
// weights y[j + r ldy]; part[t + 64 r] = sign * sum_j K(x_t, x_j) y_j,r.
struct NearItem {
  const int* tgt;
  int n, r0;
  const int* cols;
  int col0, ncols;
  const double* y;
  int ldy;
  double sign, scale;
  double* part;
};
// The partials of one node's list: tile t / 64 holds nchunks consecutive 64 x nrhs
// blocks at part; U[ubase + tgt[t] - pbase + r ldu] += their sum.
struct NearReduce {
  const int* tgt;
  int n, nchunks;
  const double* part;
  size_t ubase;
  int pbase, ldu;
};
int near_tile_rows();
int near_max_rhs();
void near_tiles(const double* Xp, const double* xn, int d, int nrhs, const NearItem* items_dev, int nitems,
                const NearReduce* lists_dev, int nlists, int max_list, double* U, cudaStream_t st);

// Conditioning probe: out[q * KROWSUM_ROWS + r] = sum_j K(x_i, x_j) over the N points of
// problem q (evaluated in FP32), for KROWSUM_ROWS rows i spread evenly over the
// problem's tree order.  The
// largest of them bounds ||K||_2 from below for a near-constant kernel and estimates it.
constexpr int KROWSUM_ROWS = 64;
struct RowSumDesc {
  int pbase, N;
  double scale;  // -1 / (2 h^2)
};
void kernel_rowsums(const double* Xp, int d, const RowSumDesc* descs_dev, int nprob, int max_n,
                    double* out, cudaStream_t st);

// ------------------------------------------- sliced FP64 operator products (a10)
// FP64 operator blocks applied on the BF16 tensor cores by exact slicing: every value
// is split into OZ_S signed 8-bit digits under a per-row (per-column for the right-hand
// sides) power of two, the digit products are summed exactly in FP32 on the tensor
// cores and recombined in integers and FP64 (ozaki.cu).
constexpr int OZ_S = 8;                              // digits per value (63 bits)
constexpr int OZ_TM = 128;                           // rows per tile (MMA M)
constexpr int OZ_KC = 16;                            // columns per chunk (one MMA K step)
constexpr int OZ_NR = 16;                            // right-hand sides per pass
constexpr int OZ_AREC = OZ_S * OZ_TM * OZ_KC * 2;   // bytes of one block chunk (32,768)
constexpr int OZ_BREC = OZ_S * OZ_NR * OZ_KC * 2;   // bytes of one right-hand-side chunk (4,096)
// One FP64 block (rows x cols, column-major, ld) into digit records: tiles of 128 rows
// x chunks of 16 columns x OZ_AREC bytes at rec, row exponents at rexp; tile0 = the
// first tile of this block among the launch's tiles (blocks in tile order).
struct OzSplitDesc {
  const double* src;
  int ld, rows, cols;
  unsigned char* rec;
  int* rexp;
  int tile0;
};
// One K x nrhs block of right-hand sides (column-major, ldw; nrhs <= OZ_NR) into digit
// records (chunks x OZ_BREC bytes) and OZ_NR column exponents.
struct OzVecDesc {
  const double* w;
  int ldw, K, nrhs;
  unsigned char* rec;
  int* cexp;
};
// out[r + c ldo] (+)= sum_k A[r, k] w[k, c] for r < rows, c < nrhs (add = 0: overwrite):
// A's records (all its tiles) and row exponents, w's records and column exponents; nch
// chunks of 16 columns.
struct OzApplyDesc {
  const unsigned char* arec;
  const int* rexp;
  const unsigned char* brec;
  const int* cexp;
  double* out;
  int ldo, rows, nch, nrhs, tile0, add;
};
// Gaussian kernel blocks with the dot products on the tensor cores (digits of every
// point's coordinates: XD, OZ_S x oz_dpad(d) BF16 per point, and XE, built by oz_points):
// out[i + j ld] = exp(scale (|x_r|^2 + |x_c|^2 - 2 x_r.x_c)) (+ diag when r == c) for the
// rows r = row0 + i (i < nrows) and the columns c = colsA[j] (j < nA), colsB[j - nA], or
// col0 + j without lists; tile0 = the first 128-row tile of this block in the launch.
// The diagonal shift goes where ident[r] == ident[c] (r == c without ident).
struct OzKDesc {
  const int* colsA;
  const int* colsB;
  double* out;
  int row0, nrows, col0, nA, ncols, ld;
  double diag, scale;
  int tile0;
  const int* ident;
};
int oz_dpad(int d);  // coordinates per point in XD (d rounded up to 16), 0 above 64
void oz_points(const double* X, int N, int d, uint16_t* XD, int* XE, cudaStream_t st);
void oz_kblocks(const uint16_t* XD, const int* XE, const double* xn, int d, const OzKDesc* descs_dev, int ndesc,
                int ntiles, int* status, cudaStream_t st);
size_t oz_arec_bytes(int rows, int cols);
size_t oz_brec_bytes(int K);
void oz_split_blocks(const OzSplitDesc* descs_dev, int ndesc, int ntiles, cudaStream_t st);
void oz_split_vecs(const OzVecDesc* descs_dev, int ndesc, cudaStream_t st);
void oz_apply(const OzApplyDesc* descs_dev, int ndesc, int ntiles, int* status, cudaStream_t st);

// ------------------------------------------------------ learned sampling (a11)
// MLP 8 -> 128 -> 128 -> 1 (ReLU).  FP32 master parameters, in this order:
// W1 [128][8] (row = hidden unit), b1 [128], W2 [128][128] (row = output unit), b2 [128],
// w3 [128], b3 [1]; BF16 copies of W1, W2, W2^T and w3 feed the tensor-core kernels.
constexpr int MLP_F = 8, MLP_W = 128;
constexpr int MLP_OFF_W1 = 0, MLP_OFF_B1 = 1024, MLP_OFF_W2 = 1152, MLP_OFF_B2 = 17536,
              MLP_OFF_W3 = 17664, MLP_OFF_B3 = 17792, MLP_NPARAM = 17793;
constexpr uint64_t LEARN_SALT = 0x4C4541524Eull, HOLD_SALT = 0x484F4C44ull, GRAM_SALT = 0x4752414Dull,
                   GUMBEL_SALT = 0x47554D42ull;
constexpr int NHOLD = 64;    // held-out rows per judged node
constexpr int NGRAM = 4096;  // Gram-estimate rows per labelled node
struct MlpDev {
  float* master;
  uint16_t *W1, *W2, *W2T, *w3;  // BF16 bit patterns
};
// Per node of a sampling step (same indexing as SampleNodeInfo): where its candidates
// start, how many (0: no learned sample), and its n_samp.
struct LearnNodeInfo {
  int cand_off, n_cand, n_samp;
};
struct LearnFeatDesc {
  const int* colsA;
  const int* colsB;
  int col0, nA, ncols;
  const int* cand;      // n_cand positions (already offset)
  const float* hits;    // n_cand hit counts (already offset)
  int n_cand, cand_off; // rows of the feature array start at cand_off
  float f4, f5, inv_h, inv_log1p_kappa;
  double scale;         // -1 / (2 h^2)
};
// Stratified row draw of a node (offsets inside its problem): the first cs rows from
// the sibling [sib_o, sib_o + sib_n), the others from outside the parent [par_o, par_o +
// par_n); cs = count / 2, or count when the parent is the whole problem.
struct StreamDesc {
  int pb, pn, uid, out_off, sib_o, sib_n, par_o, par_n;
};
struct JudgeDesc {
  const int* H;       // nh held-out positions, the first nh_s from the sibling
  int nh_s;
  double w_s, w_r;    // weights of a sibling row and of a row outside the parent
  const int* colsA;
  const int* colsB;
  int col0, nA, ncols;
  const int* skel;    // s positions
  int s;
  const double* P;    // s x ncols, column-major
  double scale;
};
struct ColsDesc {
  const int* colsA;
  const int* colsB;
  int col0, nA, ncols, out_off;
};
struct RidgeDesc {
  double* G;
  int n;
};
struct LevDesc {
  const double* Bc;   // nc x n_cand K(cols, cand)
  const double* Xs;   // nc x n_cand (G + mu I)^{-1} K(cols, cand)
  int nc, n_cand, out_off;
};
void learned_candidates(const uint32_t* cand_sorted, const uint64_t* keys_sorted, const int* node_start,
                        const int* node_cnt, int cnt_bits, const int* off, const SampleNodeInfo* info,
                        const LearnNodeInfo* linfo, int nn, uint64_t seed, int max_cand, int* cand,
                        float* hits, int* status, cudaStream_t st);
void learned_features(const double* Xp, int d, const LearnFeatDesc* descs, int nd, int max_cand,
                      uint16_t* feat, cudaStream_t st);
void mlp_forward(const uint16_t* X, int64_t n, const MlpDev& w, float* y, uint16_t* H1, uint16_t* H2,
                 cudaStream_t st);
void mlp_backward(const uint16_t* X, const uint16_t* H1, const uint16_t* H2, const float* y,
                  const float* t, int64_t n, double inv_batch, const MlpDev& w, float* grad,
                  float* loss, cudaStream_t st);
void mlp_adam(const MlpDev& w, float* grad, float* m, float* v, int step, double lr, double beta1,
              double beta2, double eps, cudaStream_t st);
void mlp_refresh_copies(const MlpDev& w, cudaStream_t st);
// score[c] <- score[c] + temp * g_c with g_c = -log(-log(u_c)) a Gumbel draw, u_c =
// ((r_c >> 11) + 1/2) 2^-53 from draw c of the node's GUMBEL stream (FP64, rounded to
// FP32): the top n_samp of the perturbed scores sample without replacement with
// probabilities proportional to exp(score / temp).
void perturb_scores(float* score, const LearnNodeInfo* linfo, const SampleNodeInfo* info, int nn,
                    int max_cand, uint64_t seed, double temp, cudaStream_t st);
void learned_select(const float* score, const int* cand, const LearnNodeInfo* linfo,
                    const SampleNodeInfo* info, int nn, int max_cand, int* samp, cudaStream_t st);
void stream_rows(const StreamDesc* descs, int nd, int count, uint64_t seed, uint64_t salt, int* out,
                 cudaStream_t st);
void id_judge(const double* Xp, int d, const JudgeDesc* descs, int nd, int nh, int max_s, double* out,
              cudaStream_t st);
void gather_cols(const ColsDesc* descs, int nd, int* out, cudaStream_t st);
void add_ridge(const RidgeDesc* descs, int nd, double tol2, cudaStream_t st);
void leverage_targets(const LevDesc* descs, int nd, double* lev, float* target, cudaStream_t st);
// B[r, :] *= (r < split ? w0 : w1) for the rows of each block (column-major, ld)
struct RowScaleDesc {
  double* B;
  int rows, cols, ld, split;
  double w0, w1;
};
void scale_rows(const RowScaleDesc* descs, int nd, cudaStream_t st);
// Training batch: of[i] = feat row idx[i] (8 BF16), ot[i] = tgt[idx[i]].
void gather_train(const uint16_t* feat, const float* tgt, const int* idx, int n, uint16_t* of, float* ot,
                  cudaStream_t st);

// Any entry non-finite -> atomicOr(status, DEV_BADINPUT).
void check_finite(const double* x, int64_t n, int* dev_status, cudaStream_t st);

}  // namespace iaskit
