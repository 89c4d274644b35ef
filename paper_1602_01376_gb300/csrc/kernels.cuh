// Host launchers of the INV-ASKIT device kernels.  Each launcher enqueues work on
// `st` and returns immediately; errors of the launch itself throw iaskit::Error.
#pragma once
#include <initializer_list>

#include "common.cuh"

namespace iaskit {

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
  DevBuf x32, cand_d, cand_i, flagged, counter, maxabs, tiles;
  void release() {
    for (DevBuf* b : {&x32, &cand_d, &cand_i, &flagged, &counter, &maxabs, &tiles}) b->release();
  }
};

// Work tile of the kNN kernels: queries [q0, q0 + qn) against the points
// [rb, rb + rn) of their problem.
struct KnnTile {
  int q0, qn, rb, rn;
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
// T = double evaluates in FP64; T = float evaluates distances and exp in FP32.
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
template <typename T>
void kernel_blocks(const double* Xp, int d, const KDescT<T>* descs_dev, int ndesc,
                   int64_t max_entries_per_desc, cudaStream_t st);

// Column-pivoted Householder QR + interpolative decomposition of each block.
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
template <typename T>
void cpqr_id(const CpqrDescT<T>* descs_dev, int ndesc, int max_rows, int max_cols, int s_max,
             double tol, cudaStream_t st);

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
};
template <typename T>
void getrf_batched(const LuDescT<T>* descs_dev, int ndesc, int max_n, int* dev_status,
                   cudaStream_t st);

// B <- A^{-1} B from getrf output, for each descriptor; B is n x ncols (ldb).
template <typename T>
struct LuSolveDescT {
  const T* LU;
  const int* ipiv;
  T* B;
  int n, ldlu, ldb, ncols;
};
template <typename T>
void getrs_batched(const LuSolveDescT<T>* descs_dev, int ndesc, int max_n, int max_cols,
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
// Work items (descriptor index, tile row, tile column).  Tile shape: 64 x 64
// (GEMM_SQUARE) or 256 x 16 (GEMM_SKINNY, every problem with N <= 16).
struct GemmTile {
  int desc, tm, tn;
};
enum GemmShape { GEMM_SQUARE = 0, GEMM_SKINNY = 1 };
inline int gemm_tile_m(GemmShape s) { return s == GEMM_SKINNY ? 256 : 64; }
inline int gemm_tile_n(GemmShape s) { return s == GEMM_SKINNY ? 16 : 64; }
template <typename T>
void gemm_grouped(const GemmDescT<T>* descs_dev, const GemmTile* tiles_dev, int ntiles,
                  GemmShape shape, cudaStream_t st);

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

// Row permutation of an N x ncols column-major block: out[p] = in[perm[p]] (gather)
// or out[perm[p]] = in[p] (scatter).
template <typename T>
void permute_rows(const T* in, int ldi, T* out, int ldo, const int* perm, int N, int ncols,
                  bool scatter, cudaStream_t st);

// u_rows += K(x_rows, x_cols) * y for each descriptor, kernel values recomputed in
// FP64.  y is ncols x nrhs (ldy), u is nrows x nrhs (ldu) with rows starting at row0.
struct KMatvecDesc {
  const int* cols;
  const double* y;
  double* u;
  int row0, nrows, col0, ncols, ldy, ldu;
  double scale;  // -1 / (2 h^2)
};
void kernel_matvec(const double* Xp, int d, int nrhs, const KMatvecDesc* descs_dev, int ndesc,
                   int max_rows, cudaStream_t st);

// Conditioning probe: out[q * KROWSUM_ROWS + r] = sum_j K(x_i, x_j) over the N points of
// problem q, for KROWSUM_ROWS rows i spread evenly over the problem's tree order.  The
// largest of them bounds ||K||_2 from below for a near-constant kernel and estimates it.
constexpr int KROWSUM_ROWS = 64;
struct RowSumDesc {
  int pbase, N;
  double scale;  // -1 / (2 h^2)
};
void kernel_rowsums(const double* Xp, int d, const RowSumDesc* descs_dev, int nprob, double* out,
                    cudaStream_t st);

// Any entry non-finite -> atomicOr(status, DEV_BADINPUT).
void check_finite(const double* x, int64_t n, int* dev_status, cudaStream_t st);

}  // namespace iaskit
