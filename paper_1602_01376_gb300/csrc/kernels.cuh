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

// Median split on the coordinate of largest spread, level by level (Sec. II-A).
// X: N x d row-major (original order, device).  level_off[l] holds the 2^l + 1
// node offsets of level l (host).  Writes perm (device, N): perm[pos] = original index,
// and split_dim (device, 2^L - 1 entries, heap order minus one).
void build_tree(const double* X, int N, int d, int L, const std::vector<std::vector<int>>& level_off,
                int* perm, int* split_dim, TreeScratch& s, cudaStream_t st);

// iperm[perm[p]] = p and Xp[p] = X[perm[p]] (rows of d doubles).
void permute_points(const double* X, const int* perm, int N, int d, int* iperm, double* Xp,
                    cudaStream_t st);

// ------------------------------------------------------------------- kNN (a2)
struct KnnScratch {
  DevBuf x32, cand_d, cand_i, flagged, counter, maxabs;
  void release() {
    for (DevBuf* b : {&x32, &cand_d, &cand_i, &flagged, &counter, &maxabs}) b->release();
  }
};

// kappa nearest neighbours of every point by (squared distance, index), self
// excluded, distance = sum_k (x_k - y_k)^2 in FP64 with every operation rounded
// (no contraction), k in order.  X is N x d row-major FP64 (original order).
// knn: N x kappa int32 (original indices).  Returns the number of queries that
// needed the exact fallback scan.
int knn_bruteforce(const double* X, int N, int d, int kappa, int* knn, KnnScratch& s,
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

// Sampled rows of every node of level l (see the sampling rule in sampling.cu).
// off: device offsets of the level (2^l + 1).  samp_off: device, per node start in
// `samp`; n_samp of node i = min(samp_cap, N - size_i).
void sample_level(const int* knn_pos, int N, int kappa, int level, const int* off_dev,
                  const std::vector<int>& off_host, int samp_cap, const int* samp_off_dev,
                  uint64_t seed, int* samp, int* dev_status, SampleScratch& s, cudaStream_t st);

// ------------------------------------------------------- dense batched kernels
// Kernel block K(x_rows, x_cols) (+ diag where the row and column positions agree),
// column-major into out.  Rows: rows ? rows[i] : row0 + i.  Columns: colsA ?
// (j < nA ? colsA[j] : colsB[j - nA]) : col0 + j.  Points are positions in Xp.
struct KDesc {
  const int* rows;
  const int* colsA;
  const int* colsB;
  double* out;
  int row0, nrows, col0, nA, ncols, ld;
  double diag;
};
void kernel_blocks(const double* Xp, int d, double h, const KDesc* descs_dev, int ndesc,
                   int64_t max_entries_per_desc, cudaStream_t st);

// Column-pivoted Householder QR + interpolative decomposition of each block.
// A (nrows x ncols, ld) is overwritten: its first s rows hold, in pivoted column
// order, R11 and T = R11^{-1} R12 in place of R12.  piv receives the column
// permutation; rank[0] receives s.
struct CpqrDesc {
  double* A;
  int* piv;
  int* rank;
  int ld, nrows, ncols;
};
void cpqr_id(const CpqrDesc* descs_dev, int ndesc, int max_rows, int max_cols, int s_max,
             double tol, cudaStream_t st);

// Builds P (s x ncols, ld = s) from a cpqr_id result and the skeleton list
// skel[k] = cols[piv[k]] with cols as in KDesc (colsA/colsB/col0).
struct PDesc {
  const double* A;  // cpqr output (ld)
  const int* piv;
  const int* colsA;
  const int* colsB;
  double* P;
  int* skel;
  int ld, ncols, s, nA, col0;
};
void assemble_P(const PDesc* descs_dev, int ndesc, int max_cols, cudaStream_t st);

// LU with partial pivoting (ties to the lowest row) of each n x n block in place.
struct LuDesc {
  double* A;
  int* ipiv;
  int n, ld;
};
void getrf_batched(const LuDesc* descs_dev, int ndesc, int max_n, int* dev_status,
                   cudaStream_t st);

// B <- A^{-1} B from getrf output, for each descriptor; B is n x ncols (ldb).
struct LuSolveDesc {
  const double* LU;
  const int* ipiv;
  double* B;
  int n, ldlu, ldb, ncols;
};
void getrs_batched(const LuSolveDesc* descs_dev, int ndesc, int max_n, int max_cols,
                   cudaStream_t st);

// C <- alpha * A * B + beta * C (column-major, no transposes) for each descriptor.
struct GemmDesc {
  const double* A;
  const double* B;
  double* C;
  int M, N, K, lda, ldb, ldc;
  double alpha, beta;
};
// Work items (descriptor index, tile row, tile column) of 64 x 64 tiles.
struct GemmTile {
  int desc, tm, tn;
};
void gemm_grouped(const GemmDesc* descs_dev, const GemmTile* tiles_dev, int ntiles,
                  cudaStream_t st);

// dst (rows x cols, ldd) <- src (rows x cols, lds), batched.
struct CopyDesc {
  const double* src;
  double* dst;
  int rows, cols, lds, ldd;
};
void copy_batched(const CopyDesc* descs_dev, int ndesc, int64_t max_entries, cudaStream_t st);

// Z'' = [[I, C_l], [C_r, I]] of size (s_l + s_r), ld = s_l + s_r.
struct ZDesc {
  const double* Cl;  // s_l x s_r, ld s_l
  const double* Cr;  // s_r x s_l, ld s_r
  double* Z;
  int sl, sr;
};
void form_Z(const ZDesc* descs_dev, int ndesc, int64_t max_entries, cudaStream_t st);

// Row permutation of an N x ncols column-major block: out[p] = in[perm[p]] (gather)
// or out[perm[p]] = in[p] (scatter).
void permute_rows(const double* in, int ldi, double* out, int ldo, const int* perm, int N,
                  int ncols, bool scatter, cudaStream_t st);

// u_rows += K(x_rows, x_cols) * y for each descriptor, kernel values recomputed in
// FP64.  y is ncols x nrhs (ldy), u is nrows x nrhs (ldu) with rows starting at row0.
struct KMatvecDesc {
  const int* cols;
  const double* y;
  double* u;
  int row0, nrows, col0, ncols, ldy, ldu;
};
void kernel_matvec(const double* Xp, int d, double h, int nrhs, const KMatvecDesc* descs_dev,
                   int ndesc, int max_rows, cudaStream_t st);

// Any entry non-finite -> atomicOr(status, DEV_BADINPUT).
void check_finite(const double* x, int64_t n, int* dev_status, cudaStream_t st);

}  // namespace iaskit
