// INV-ASKIT orchestration on one GPU and the C ABI of include/iaskit.h.
//
// Factorization (Sec. II-C, Alg. "Factorize", run bottom-up with loops over levels
// as the paper's implementation does):
//   tree -> kNN -> skeletonize bottom-up (sample, kernel block, CPQR/ID, nested P)
//   -> leaf LU of lambda I + K_aa -> for every node above the leaves, bottom-up:
//   U blocks K_{l r~}, K_{r l~}, W = Solve(child subtree, U) for all children at once
//   (a "forest solve"), reduced systems Z and their LU.
// Solve (Alg. "Solve"): a forest solve rooted at the roots.
//
// Many independent problems (each with its own points, h and lambda) are factored
// together: their points are concatenated, every node has a global id, and every
// step is one launch over the nodes of all problems at the same height above the
// leaves.  A single problem is the batch of one.
//
// The forest solve applies Solve to the blocks of a set of subtrees at once.  At a
// node beta with children a, b it needs V v = [P_{b~ b} v_b; P_{a~ a} v_a] (eq.
// blocksmw).  The full P_{a~ a} of eq. innerid is never formed: t_a = P_{a~ a} v_a is
// carried up the tree.  A leaf computes t = P v from its own ID; after beta's update
// v_a -= W_{a b~} y1 the carried value becomes t_a - (P_{a~ a} W_{a b~}) y1, and the
// product P_{a~ a} W_{a b~} is exactly the off-diagonal block C_a of beta's reduced
// system, kept from the factorization; then t_beta = P_{beta~ [a~ b~]} [t_a; t_b].
// This gives the same vectors as the literal products in O(s^2) per node instead of
// O(s |beta|).
// The reduced system is stored with blocks in the order [a~ part; b~ part]:
// Z'' = [[I, C_a], [C_b, I]] acting on [y2; y1] with right side [t_a; t_b]; it is
// the paper's [[I, C_b], [C_a, I]] with both block rows and block columns swapped.
//
// Two precisions:
//  * plain: everything in FP64;
//  * mixed: the factorization (sampled blocks, CPQR updates, leaf LU, W, C, Z) in
//    FP32 with pivot norms compared in FP64; the operator lambda I + K~ is kept in
//    FP64 (leaf blocks and U blocks evaluated once in FP64 and stored, P in FP64),
//    and the solve refines w += Solve32(u - (lambda I + K~) w) until the relative
//    residual of every column is below the target.  K~ is the one defined by the
//    skeletons and P this factorization chose, so the FP32 factorization is an
//    approximate inverse of exactly the operator the residual uses.
#include <algorithm>
#include <chrono>
#include <climits>
#include <numeric>
#include <random>
#include <cmath>
#include <memory>
#include <type_traits>

#include "kernels.cuh"

namespace iaskit {

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Host staging of descriptor arrays, uploaded with one copy.
struct Arena {
  std::vector<char> host;
  size_t push_raw(const void* p, size_t bytes) {
    size_t off = (host.size() + 15) & ~size_t(15);
    host.resize(off + bytes);
    if (bytes) std::memcpy(host.data() + off, p, bytes);
    return off;
  }
  template <typename T>
  size_t push(const std::vector<T>& v) { return push_raw(v.data(), v.size() * sizeof(T)); }
  void clear() { host.clear(); }
};

enum Precision { PREC_FP64 = 0, PREC_MIXED = 1 };

struct Options {
  int kappa = 16;
  int samp_factor = 2;
  uint64_t seed = 0;
  int refine = 0;
  double refine_tol = 1e-10;
  double mem_cap_gb = 0.0;
  int precision = PREC_FP64;
  int problem = 0;  // problem the introspection calls refer to
  // mixed form: problems whose estimated condition number exceeds this are factored in FP64
  double mixed_cond_max = 1e6;
  int sampling = 0;         // 0: kNN + uniform; 1: learned proposal judged per node
  int cand_factor = 8;      // learned candidates per sampled row
  int keep_candidates = 0;  // keep candidates, features and scores for introspection
  int train_batch = 4096;
  double learned_temp = 0.0;  // Gumbel temperature of the learned selection (0: top scores)
  int gemm_tc = 1;            // FP32 products with more than 16 columns on the tensor cores (3xTF32)
  int cpqr_cluster = 1;       // FP32 IDs of up to 512 x 512 on a cluster of blocks per node
  // FP32 LUs inverted once and applied as products: 1 the leaf blocks, 2 the leaf blocks
  // and the reduced systems up to height lu_inverse_zh; 0 none (LU solves).  Inverses of
  // the reduced systems above height 1 raised the refinement's GMRES iterations on the
  // manifold in d 64 (10 -> 16); those of height 1 did not
  int lu_inverse = 2;
  int lu_inverse_zh = 1;
  // mixed form: problems whose condition estimate exceeds this keep their operator
  // blocks in FP64 from the start; any other problem whose refinement stops at the
  // FP32-pair operator's rounding floor is upgraded to FP64 and refined again.  Measured
  // pair floors: below 4e-13 at condition estimate 1.9e4 (mixture in d 54), 4.6e-9 at
  // 4.5e5 (manifold in d 64), against the default 1e-10 target
  double pair_cond_max = 1e5;
  // operator: 0 = lambda I + K~ (i not in alpha), 1 = lambda I + K~ + S, the kNN-separated
  // operator of eq. (askit); the factorization (of lambda I + K~) then preconditions the
  // refinement's GMRES
  int near_field = 0;
  // failure-path test hook: flags (DEV_* bits) that the host ORs into the device status
  // word just before the next status read, as a kernel's bounded wait or pivot check
  // would; one-shot (cleared once injected)
  int inject_status = 0;
  // kNN: 1 = search in tree order with tile pruning (default), 0 = brute force over
  // every pair; the lists are identical
  int knn_prune = 1;
  // mixed form with FP64 operator blocks: GMRES's inner operator applies on FP32 pairs,
  // every cycle's residual in FP64 (1), or every apply in FP64 (0, the default: the
  // pair products of FP64-stored blocks split every entry on the FP64 pipe and were
  // measured no faster than FP64 products on C4)
  int inner_pair = 0;
  // mixed form with FP64 operator blocks: the operator's FP64 products on the BF16
  // tensor cores by exact 8-bit slicing (1, default), or on the FP64 pipe (0)
  int op_slices = 1;
  // the kernel of the next factorization: 0 Gaussian, 1 (x . y / h^2 + poly_c)^poly_p
  int kernel = 0;
  int poly_p = 2;
  double poly_c = 1.0;
};

struct Prob {
  int N = 0, L = 0, m_max = 0;
  double h = 0, lam = 0, scale = 0;  // scale = -1 / (2 h^2)
  int pbase = 0;                     // first global position (and original index)
  int nbase = 0;                     // global id of heap id 0: gid = nbase + uid
  double cond_est = 0;               // 1 + max sampled kernel row sum / lambda
  bool f64 = true;                   // factorization stored in FP64 (else FP32)
  bool op64 = false;                 // mixed form: operator blocks in FP64 (else FP32 pairs)
};

struct Node {
  int prob = 0, uid = 0, level = 0;
  int off = 0, size = 0;  // global position range
  int s = 0;              // rank (skeleton count); 0 for a root
  int ncols = 0;          // ID columns: size (leaf) or s_l + s_r
  int nsamp = 0;
  int leaf = -1;          // global leaf index (leaves only)
  // offsets into the typed factorization buffers of the node's problem precision (LU, W,
  // Z, C) and into the FP64 operator blocks kept by the mixed form (K: leaf, U)
  int64_t DI_off = 0;  // FP32 nodes: the dinv area of the node's LU (leaf block or Z)
  int64_t samp_off = 0, P_off = 0, W_off = 0, LU_off = 0, Z_off = 0, Zpiv_off = 0, CL_off = 0,
          CR_off = 0, K_off = 0, U_off = 0;
};

// A refined column that stopped at its rounding floor: problem, column, its relative
// residual and the floor estimate 2^-53 ||A|| ||w|| / ||u||, and whether the problem's
// operator blocks were FP64 (else FP32 pairs, whose floor is about 2^9 higher).
struct StagCol {
  int prob, col;
  double resid, floor;
  bool op64;
};

struct Stats {
  double t_tree = 0, t_knn = 0, t_skel = 0, t_leaf_lu = 0, t_factor_levels = 0, t_factor = 0;
  double t_solve = 0, t_apply = 0;
  int knn_fallback = 0;
  KnnPruneStats knn_prune;
  double near_values = 0.0;
  int64_t bytes_W = 0, bytes_LU = 0, bytes_P = 0, bytes_operator = 0, bytes_slices = 0;
  std::vector<double> refine_hist;
  int refine_sweeps = 0;
  int refine_iters = 0;       // GMRES iterations (operator applications) of the last solve
  int refine_stagnated = 0;   // columns stopped at the rounding floor of the FP64 operator
  std::vector<StagCol> stagnated;  // those columns with their residual and floor estimate
  int fp64_problems = 0;      // problems factored in FP64
  int fp64_operator_problems = 0;  // mixed form: problems whose operator blocks stay in FP64
  int operator_upgrades = 0;       // of those, upgraded after their refinement stopped at the floor
  int learned_nodes = 0, fallback_nodes = 0, judged_nodes = 0;
  double judge_err_plain = 0, judge_err_chosen = 0;  // sums over judged nodes
  std::vector<double> train_loss;                    // mean batch loss per epoch
  int64_t train_rows = 0;
};

template <typename T>
struct RootBlock {
  int gid;
  T* V;
  int ld;
  int nc;
  T* t_out;  // P_c v_c destination when the caller needs it (may be null)
  int t_ld;
};

template <typename T>
double gemm_flops(const std::vector<GemmDescT<T>>& g) {
  double f = 0;
  for (const auto& d : g) f += 2.0 * d.M * (double)d.N * d.K;
  return f;
}
template <typename T>
double getrs_flops(const std::vector<LuSolveDescT<T>>& v) {
  double f = 0;
  for (const auto& d : v) f += 2.0 * d.n * (double)d.n * d.ncols;
  return f;
}
// GETRI from the LU: 4/3 n^3 (LAPACK's count)
double getri_flops(const std::vector<LuSolveDescT<float>>& v) {
  double f = 0;
  for (const auto& d : v) f += 4.0 / 3.0 * d.n * (double)d.n * d.n;
  return f;
}
template <typename T>
double getrf_flops(const std::vector<LuDescT<T>>& v) {
  double f = 0;
  for (const auto& d : v) f += 2.0 / 3.0 * d.n * (double)d.n * d.n;
  return f;
}
// Algorithmic work of kernel blocks: 2d + 3 flops per entry (the squared distance or
// dot product, scale and shift) plus one exponential, counted as the entries' flops.
template <typename D>
double kblock_flops(const std::vector<D>& kd, int d) {
  double e = 0;
  for (const auto& k : kd) e += (double)k.nrows * k.ncols;
  return e * (2.0 * d + 3.0);
}
template <typename T>
void add_gemm(std::vector<GemmDescT<T>>& g, const T* A, int lda, const T* B, int ldb, T* C,
              int ldc, int M, int Ncol, int K, double alpha, double beta) {
  if (M <= 0 || Ncol <= 0) return;
  g.push_back(GemmDescT<T>{A, B, C, M, Ncol, K, lda, ldb, ldc, alpha, beta});
}

// Tile list of one grouped launch: 256 x 16 tiles when no problem has more than 16
// columns (right-hand-side blocks of a solve); otherwise 128 x 128 tensor-core tiles
// for FP32 products (when enabled) and 64 x 64 tiles for FP64 ones (on FP64 or on
// FP32 pairs).
// A CUDA-core launch (tunable: not on the tensor cores, not on FP32 pairs) takes the
// autotuned shape of its (type, largest N, largest M) bucket when the table has one.
template <typename T>
GemmShape make_tiles(const std::vector<GemmDescT<T>>& g, std::vector<GemmTile>& t, bool tc, bool tunable) {
  int maxn = 0, maxm = 0;
  for (const auto& d : g) {
    maxn = std::max(maxn, d.N);
    maxm = std::max(maxm, d.M);
  }
  GemmShape shape = maxn <= 16                                      ? GEMM_SKINNY
                    : (tc && std::is_same<T, float>::value) ? GEMM_TC
                                                                  : GEMM_SQUARE;
  constexpr bool fp64 = std::is_same<T, double>::value;
  if (tunable && shape != GEMM_TC) {
    const int e = gemm_tuned(fp64, gemm_n_bucket(maxn), gemm_m_bucket(maxm));
    if (e >= 0 && e < GEMM_NSHAPES && gemm_shape_valid((GemmShape)e, fp64)) shape = (GemmShape)e;
  }
  const int tm_ = gemm_tile_m(shape), tn_ = gemm_tile_n(shape);
  t.clear();
  for (int idx = 0; idx < (int)g.size(); ++idx)
    for (int tn = 0; tn < (g[idx].N + tn_ - 1) / tn_; ++tn)
      for (int tm = 0; tm < (g[idx].M + tm_ - 1) / tm_; ++tm) t.push_back(GemmTile{idx, tm, tn});
  return shape;
}

// Per problem block of an N_p x nrhs right-hand side inside the concatenated layout.
struct BlockDesc {
  int64_t base;  // element offset of the block (pbase * nrhs)
  int n;         // N_p
  double a;      // per-problem scalar
};

__global__ void gather_rows_kernel(const double* in, double* out, const int* perm, const int* pid,
                                   const BlockDesc* blocks, int Ntot, int nrhs, bool scatter) {
  const int64_t total = (int64_t)Ntot * nrhs;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e % Ntot), c = (int)(e / Ntot);
    const BlockDesc b = blocks[pid[p]];
    const int pb = (int)(b.base / nrhs);
    const int64_t dst = b.base + (int64_t)(p - pb) + (int64_t)c * b.n;
    const int64_t src = b.base + (int64_t)(perm[p] - pb) + (int64_t)c * b.n;
    if (scatter) out[src] = in[dst];
    else out[dst] = in[src];
  }
}
__global__ void scale_blocks_kernel(const double* x, double* y, const BlockDesc* blocks, int nrhs) {
  const BlockDesc b = blocks[blockIdx.y];
  const int64_t n = (int64_t)b.n * nrhs;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[b.base + i] = b.a * x[b.base + i];
}
__global__ void axpby_kernel(const double* u, double* r, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    r[i] = u[i] - r[i];
}
// One block per (column, problem): the 2-norm of that column of that problem's block.
// Reductions over long vectors in two fixed-order stages: blocks of RED_CHUNK elements
// write partial sums, then one thread per result adds its chunks in order (the result
// does not depend on scheduling, and a vector of 2^20 elements spreads over 64 blocks).
constexpr int RED_CHUNK = 16384;
__device__ __forceinline__ double block_sum(double s) {
  __shared__ double red[32];
  s = warp_sum(s);
  __syncthreads();  // red is free (a previous call of this block has read it)
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
  }
  return s;  // valid in thread 0
}
// part[(q nrhs + c) nch + chunk] = sum of squares of column c of problem q over the chunk
__global__ void colnorm_part_kernel(const double* x, const BlockDesc* blocks, int nrhs, int nch, double* part) {
  const int ch = blockIdx.x, c = blockIdx.y, q = blockIdx.z;
  const BlockDesc b = blocks[q];
  const int64_t i0 = (int64_t)ch * RED_CHUNK;
  if (i0 >= b.n) {
    if (threadIdx.x == 0) part[((size_t)q * nrhs + c) * nch + ch] = 0.0;
    return;
  }
  const double* col = x + b.base + (int64_t)c * b.n;
  const int64_t i1 = min((int64_t)b.n, i0 + RED_CHUNK);
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s = fma(col[i], col[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) part[((size_t)q * nrhs + c) * nch + ch] = s;
}
__global__ void colnorm_reduce_kernel(const double* part, int total, int nch, double* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  double s = 0.0;
  for (int ch = 0; ch < nch; ++ch) s += part[(size_t)e * nch + ch];
  out[e] = sqrt(s);
}

// One GMRES segment: a column of one problem's block, [base, base + len).
struct GSeg {
  int64_t base;
  int len;
};

// part[((i S) + q) nch + chunk] = <V_i, x> over one chunk of segment q
__global__ void seg_dots_part_kernel(const double* V, size_t vstride, const double* x, const GSeg* segs, int S,
                                     int nch, double* part) {
  const int ch = blockIdx.x, i = blockIdx.y, q = blockIdx.z;
  const GSeg sg = segs[q];
  const int64_t e0 = (int64_t)ch * RED_CHUNK;
  double* dst = part + ((size_t)i * S + q) * nch + ch;
  if (e0 >= sg.len) {
    if (threadIdx.x == 0) *dst = 0.0;
    return;
  }
  const int64_t e1 = min((int64_t)sg.len, e0 + RED_CHUNK);
  const double* v = V + (size_t)i * vstride + sg.base;
  const double* y = x + sg.base;
  double acc = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) acc = fma(v[e], y[e], acc);
  acc = block_sum(acc);
  if (threadIdx.x == 0) *dst = acc;
}
__global__ void chunk_sum_kernel(const double* part, int total, int nch, double* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  double s = 0.0;
  for (int ch = 0; ch < nch; ++ch) s += part[(size_t)e * nch + ch];
  out[e] = s;
}
__global__ void seg_axpy_kernel(double* x, const double* V, size_t vstride, int k, const double* coef,
                                double sign, const GSeg* segs, int S) {
  const int q = blockIdx.y;
  const GSeg sg = segs[q];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < sg.len; e += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc = fma(coef[(size_t)i * S + q], V[(size_t)i * vstride + sg.base + e], acc);
    x[sg.base + e] += sign * acc;
  }
}
__global__ void seg_scale_kernel(double* out, const double* x, const double* coef, const GSeg* segs) {
  const int q = blockIdx.y;
  const GSeg sg = segs[q];
  const double a = coef[q];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < sg.len; e += gridDim.x * blockDim.x)
    out[sg.base + e] = a * x[sg.base + e];
}

// Copy with type conversion of element ranges: dst[dst + e] = src[src + e], e < len.
struct ConvSeg {
  int64_t src, dst, len;
};
template <typename D, typename S>
__device__ __forceinline__ D conv_val(S v) {
  return (D)v;
}
// FP32 pairs: the FP32 value is hi (hi = fl32(hi + lo)); the FP64 value is hi + lo
template <>
__device__ __forceinline__ float conv_val<float, float2>(float2 v) {
  return v.x;
}
template <>
__device__ __forceinline__ double conv_val<double, float2>(float2 v) {
  return (double)v.x + (double)v.y;
}
template <typename S, typename D>
__global__ void conv_segs_kernel(const S* __restrict__ src, D* __restrict__ dst, const ConvSeg* segs) {
  const ConvSeg sg = segs[blockIdx.y];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < sg.len;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[sg.dst + e] = conv_val<D, S>(src[sg.src + e]);
}
// The same block descriptor writing FP32 pairs into the bytes of an FP64 array.
KDescT<float2> pair_desc(const KDesc& k) {
  return KDescT<float2>{k.rows, k.colsA, k.colsB, reinterpret_cast<float2*>(k.out), k.row0, k.nrows,
                        k.col0, k.nA, k.ncols, k.ld, k.diag, k.scale};
}

unsigned grid_cap(int64_t work, unsigned cap) {
  int64_t b = (work + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

class Solver {
 public:
  cudaStream_t st = nullptr;
  Options opt;
  Stats stats;
  bool factored = false;
  bool skeletonized = false;  // ranks of the current tree are known (set before factor_levels)
  KernelSpec kspec;           // the kernel of the current factorization
  // Every translation unit that evaluates kernel values gets the spec (stream-ordered).
  void use_kernel(const KernelSpec& k) {
    kspec_set_dense(k, st);
    kspec_set_near(k, st);
    kspec_set_predict(k, st);
  }
  int prec = PREC_FP64;  // precision of the current factorization
  int Ntot = 0, d = 0, s_max = 0, kappa = 0, m_max = 0, Hmax = 0, nleaves = 0;
  double tol = 0;
  std::vector<Prob> pr;
  std::vector<Node> nd;                       // global ids; unused slot at each nbase
  std::vector<std::vector<int>> by_height;    // gids of each height (0 = leaves), roots included
  DevBuf X, Xp, perm, iperm, pid, knn, knn_pos, samp, ranks, skel, piv_ws, A_ws, status,
      arena_dev, step_dev, tbuf, vbuf, vbuf32, ubuf, rbuf, wt, io, normbuf, redpart, blocks_dev, gseg_dev,
      kryl, kzb, coefbuf, cseg_dev, rowsum, xnrm;
  // learned sampling: per-step scratch, MLP parameters and training data
  DevBuf l_cand, l_hits, l_feat, l_score, l_linfo, l_samp, l_rk, l_Ptmp, l_sktmp, l_hold, l_err,
      l_cols, l_gram, l_dense, mlp_master, mlp_m, mlp_v, mlp_grad, mlp_b16, mlp_loss, tr_feat, tr_tgt,
      tr_lev, tr_bx, tr_bt, tr_y, tr_H1, tr_H2, tr_idx;
  int mlp_step = 0;
  bool mlp_ready = false;
  // factorization storage: FP64 (plain) and FP32 (mixed)
  DevBuf LU, LUpiv, Wb, Zb, Zpiv, Cb, LU32, Wb32, Zb32, Cb32, tbuf32;
  // operator blocks kept by the mixed form, evaluated in FP64 and stored as FP32 pairs:
  // leaf blocks lambda I + K_aa and U blocks
  DevBuf Kleaf, Ustore;
  DevBuf Pd, Pf;  // nested P of every node: FP64, and its FP32 copy (mixed)
  DevBuf Ppair;   // mixed form: P as FP32 pairs for the operator (Kleaf, Ustore hold pairs too)
  DevBuf Xpair;   // mixed form: permuted coordinates as FP32 pairs
  DevBuf DInv32;  // FP32 LUs: inverses of their 32 x 32 diagonal blocks and pivot permutations
  DevBuf LUi32, Zi32;  // explicit inverses of the FP32 leaf LUs and reduced systems (lu_inverse)
  DevBuf fsS;          // forest solves with inverses: the right-hand sides' copy
  bool inv_leaf = false, inv_z = false;  // this factorization's FP32 leaf LUs / Zs have inverses
  int inv_zh = 0;                         // the Zs up to this height (inv_z)
  DevBuf rhs_keep;  // mixed form: the right-hand side, for a refinement after an operator upgrade
  DevBuf pred_part, pred_io;  // kernel sums at test points: chunk partials; host-call staging
  DevBuf kperm, kiperm, Xk;   // kNN search order (tree of 128-point leaves) and its points
  std::vector<char> stag_prob;  // per problem: a column of the last refinement stopped at its floor
  TreeScratch tree_s;
  KnnScratch knn_s;
  SampleScratch samp_s;
  Arena arena;

  // ------------------------------------------------------------ tree helpers
  int left(int g) const { return pr[nd[g].prob].nbase + 2 * nd[g].uid; }
  int right(int g) const { return left(g) + 1; }
  int parent(int g) const { return pr[nd[g].prob].nbase + (nd[g].uid >> 1); }
  int sibling(int g) const { return pr[nd[g].prob].nbase + (nd[g].uid ^ 1); }
  bool is_root(int g) const { return nd[g].uid == 1; }
  bool is_leaf(int g) const { return nd[g].level == pr[nd[g].prob].L; }
  int height(int g) const { return pr[nd[g].prob].L - nd[g].level; }
  int n2(int g) const { return nd[left(g)].s + nd[right(g)].s; }  // reduced-system size
  // row offset of child c's skeletons inside the parent's [t_a; t_b]
  int rowoff(int c) const { return (nd[c].uid & 1) ? nd[sibling(c)].s : 0; }
  double scale_of(int g) const { return pr[nd[g].prob].scale; }

  // typed views of the factorization storage
  template <typename T>
  T* luP() { return std::is_same<T, float>::value ? (T*)LU32.p : (T*)LU.p; }
  // the dinv area of node g's LU (FP32 only; null for FP64)
  template <typename T>
  T* dinvP(int g) { return std::is_same<T, float>::value ? (T*)(DInv32.as<float>() + nd[g].DI_off) : nullptr; }
  template <typename T>
  T* wP() { return std::is_same<T, float>::value ? (T*)Wb32.p : (T*)Wb.p; }
  template <typename T>
  T* zP() { return std::is_same<T, float>::value ? (T*)Zb32.p : (T*)Zb.p; }
  template <typename T>
  T* cP() { return std::is_same<T, float>::value ? (T*)Cb32.p : (T*)Cb.p; }
  template <typename T>
  T* pP() { return std::is_same<T, float>::value ? (T*)Pf.p : (T*)Pd.p; }
  template <typename T>
  DevBuf& tB() { return std::is_same<T, float>::value ? tbuf32 : tbuf; }

  // ---------------------------------------------------------------- helpers
  char* upload_arena() {
    size_t bytes = std::max<size_t>(arena.host.size(), 16);
    if (bytes > arena_dev.bytes) {
      IA_CUDA(cudaStreamSynchronize(st));
      arena_dev.ensure(bytes * 2);
    }
    h2d(arena_dev.as<char>(), arena.host.data(), arena.host.size(), st);
    return arena_dev.as<char>();
  }
  int read_status_and_clear() {
    int v = 0;
    if (opt.inject_status) {  // the hook writes the device word itself, from the host
      d2h(&v, status.as<int>(), 1, st);
      IA_CUDA(cudaStreamSynchronize(st));
      v |= opt.inject_status;
      opt.inject_status = 0;
      h2d(status.as<int>(), &v, 1, st);
      v = 0;
    }
    d2h(&v, status.as<int>(), 1, st);
    IA_CUDA(cudaStreamSynchronize(st));
    IA_CUDA(cudaMemsetAsync(status.as<int>(), 0, sizeof(int), st));
    return v;
  }
  void raise_status(int v) {
    if (v & DEV_BADINPUT) throw Error(IASKIT_ERR_INPUT, "non-finite input value");
    if (v & DEV_SINGULAR) throw Error(IASKIT_ERR_SINGULAR, "exact zero pivot in an LU");
    if (v & DEV_TIMEOUT) throw Error(IASKIT_ERR_TIMEOUT, "bounded device wait expired");
    if (v & DEV_OVERFLOW) throw Error(IASKIT_ERR_UNSUPPORTED, "internal bound exceeded");
  }
  // FP64 products of the mixed form's factorization and preconditioner (problems
  // factored in FP64), and the updates of their LU solves outside the diagonal blocks,
  // run on FP32 pairs (about 2^-44 relative, on the FP32 pipes); the operator apply
  // keeps FP64 products for the problems whose operator is in FP64.
  bool in_apply = false;
  bool apply_low = false;  // an operator apply inside GMRES: FP64 products on pairs too
  template <typename T>
  bool pair_products() const {
    return std::is_same<T, double>::value && prec == PREC_MIXED && (!in_apply || apply_low);
  }
  template <typename T>
  void launch_gemms(const GemmDescT<T>* descs_dev, const GemmTile* tiles_dev, int ntiles, GemmShape shape) {
    if (pair_products<T>())
      gemm_pair64_grouped(reinterpret_cast<const GemmDesc*>(descs_dev), tiles_dev, ntiles, shape, st);
    else
      gemm_grouped(descs_dev, tiles_dev, ntiles, shape, st, status.as<int>());
  }
  template <typename T>
  void run_gemms(const std::vector<GemmDescT<T>>& g) {
    if (g.empty()) return;
    std::vector<GemmTile> t;
    const GemmShape shape = make_tiles(g, t, opt.gemm_tc != 0, !pair_products<T>());
    arena.clear();
    size_t og = arena.push(g), ot = arena.push(t);
    char* base = upload_arena();
    prof().flops[pair_products<T>() ? PK_GEMM_PAIR : pk_of<T>(PK_GEMM)] += gemm_flops(g);
    launch_gemms((const GemmDescT<T>*)(base + og), (const GemmTile*)(base + ot), (int)t.size(), shape);
  }
  // C (+)= A B with A stored as FP32 pairs (the operator blocks of the mixed form)
  static void add_pair_gemm(std::vector<GemmDescPair>& g, const float2* A, int lda, const double* B, int ldb,
                            double* C, int ldc, int M, int Ncol, int K, double beta) {
    if (M <= 0 || Ncol <= 0) return;
    g.push_back(GemmDescPair{A, B, C, M, Ncol, K, lda, ldb, ldc, 1.0, beta});
  }
  void run_pair_gemms(const std::vector<GemmDescPair>& g) {
    if (g.empty()) return;
    std::vector<GemmTile> t;
    double fl = 0;
    for (int idx = 0; idx < (int)g.size(); ++idx) {
      for (int tn = 0; tn < (g[idx].N + GEMM_PAIR_TN - 1) / GEMM_PAIR_TN; ++tn)
        for (int tm = 0; tm < (g[idx].M + GEMM_PAIR_TM - 1) / GEMM_PAIR_TM; ++tm) t.push_back(GemmTile{idx, tm, tn});
      fl += 2.0 * g[idx].M * g[idx].N * g[idx].K;
    }
    arena.clear();
    size_t og = arena.push(g), ot = arena.push(t);
    char* base = upload_arena();
    prof().flops[PK_GEMM_PAIR] += fl;
    gemm_pair_grouped((const GemmDescPair*)(base + og), (const GemmTile*)(base + ot), (int)t.size(), st);
  }
  // per-problem blocks of an nrhs-column right-hand side (uploaded to blocks_dev)
  const BlockDesc* upload_blocks(int nrhs, bool lam_scalar) {
    std::vector<BlockDesc> b(pr.size());
    for (size_t q = 0; q < pr.size(); ++q)
      b[q] = BlockDesc{(int64_t)pr[q].pbase * nrhs, pr[q].N, lam_scalar ? pr[q].lam : 0.0};
    BlockDesc* dv = blocks_dev.ensure_n<BlockDesc>(b.size());
    h2d(dv, b.data(), b.size(), st);
    return dv;
  }
  template <typename Src, typename Dst>
  void conv_segs(const Src* src, Dst* dst, const std::vector<ConvSeg>& segs) {
    int64_t mx = 0;
    for (const ConvSeg& c : segs) mx = std::max(mx, c.len);
    if (mx == 0) return;
    ConvSeg* dv = cseg_dev.ensure_n<ConvSeg>(segs.size());
    h2d(dv, segs.data(), segs.size(), st);
    ProfScope _ps(PK_MISC, st);
    conv_segs_kernel<Src, Dst><<<dim3(grid_cap(mx, 1024), (unsigned)segs.size()), 256, 0, st>>>(src, dst, dv);
    IA_LAUNCH_CHECK();
  }
  bool f64(int g) const { return pr[nd[g].prob].f64; }
  bool any_prec(bool want_f64) const {
    for (const Prob& P : pr)
      if (P.f64 == want_f64) return true;
    return false;
  }
  void gather(const double* in, double* out, int nrhs, const BlockDesc* blocks, bool scatter) {
    ProfScope _ps(PK_MISC, st);
    gather_rows_kernel<<<grid_cap((int64_t)Ntot * nrhs, 8192), 256, 0, st>>>(
        in, out, perm.as<int>(), pid.as<int>(), blocks, Ntot, nrhs, scatter);
    IA_LAUNCH_CHECK();
  }

  // ------------------------------------------------------------- forest solve
  // Applies (lambda I + K~_cc)^{-1} to the block of every root c, in place, with the
  // factorization stored in precision T.  Writes P_c v_c to roots[].t_out when given.
  template <typename T>
  void forest_solve(const std::vector<RootBlock<T>>& roots) {
    const bool need_t = !roots.empty() && roots[0].t_out != nullptr;
    std::vector<int> root_of(nd.size(), -1);
    std::vector<T*> Vp(nd.size(), nullptr);
    int max_nc = 0, top = 0;
    for (size_t q = 0; q < roots.size(); ++q) {
      max_nc = std::max(max_nc, roots[q].nc);
      const int c = roots[q].gid;
      top = std::max(top, height(c));
      std::vector<int> stack{c};
      while (!stack.empty()) {
        int u = stack.back();
        stack.pop_back();
        root_of[u] = (int)q;
        Vp[u] = roots[q].V + (nd[u].off - nd[c].off);
        if (!is_leaf(u)) {
          stack.push_back(left(u));
          stack.push_back(right(u));
        }
      }
    }
    // T and Y scratch for internal forest nodes
    std::vector<int64_t> Toff(nd.size(), -1);
    int64_t tsz = 0;
    for (int hh = 1; hh <= top; ++hh)
      for (int u : by_height[hh]) {
        if (root_of[u] < 0) continue;
        Toff[u] = tsz;
        tsz += 2 * (int64_t)n2(u) * roots[root_of[u]].nc;
      }
    T* Tb = tB<T>().template ensure_n<T>(std::max<int64_t>(tsz, 1));
    auto Tp = [&](int u) { return Tb + Toff[u]; };
    auto Yp = [&](int u) { return Tb + Toff[u] + (int64_t)n2(u) * roots[root_of[u]].nc; };
    auto ldV = [&](int u) { return roots[root_of[u]].ld; };
    auto ncV = [&](int u) { return roots[root_of[u]].nc; };
    // where node u's carried t goes: its parent's T, or the root's output
    auto tdst = [&](int u, T*& dst, int& ldd) {
      if (roots[root_of[u]].gid == u) {
        dst = roots[root_of[u]].t_out;
        ldd = roots[root_of[u]].t_ld;
      } else {
        const int par = parent(u);
        dst = Tp(par) + rowoff(u);
        ldd = n2(par);
      }
    };

    // FP32 LUs with inverses: the leaf solves and the reduced systems are products
    const bool fp32 = std::is_same<T, float>::value;
    const bool inv = fp32 && inv_leaf, invz = fp32 && inv_z;
    // 1. leaf LU solves; leaf t = P v
    {
      std::vector<LuSolveDescT<T>> ds;
      std::vector<GemmDescT<T>> g, gl;
      std::vector<CopyDescT<T>> cps;
      std::vector<int64_t> soff(roots.size(), 0);
      int64_t max_cp = 0;
      T* S = nullptr;
      if (inv) {  // every root's right-hand sides to the scratch, read there by the products
        int64_t so = 0;
        for (size_t q = 0; q < roots.size(); ++q) {
          soff[q] = so;
          so += (int64_t)nd[roots[q].gid].size * roots[q].nc;
        }
        S = fsS.ensure_n<T>(std::max<int64_t>(so, 1));
        for (size_t q = 0; q < roots.size(); ++q) {
          const int rows = nd[roots[q].gid].size;
          cps.push_back(CopyDescT<T>{roots[q].V, S + soff[q], rows, roots[q].nc, roots[q].ld, rows});
          max_cp = std::max<int64_t>(max_cp, (int64_t)rows * roots[q].nc);
        }
      }
      for (int u : by_height[0]) {
        if (root_of[u] < 0) continue;
        if (inv) {
          const RootBlock<T>& R = roots[root_of[u]];
          const int rows = nd[R.gid].size;
          add_gemm<T>(gl, (const T*)LUi32.as<float>() + nd[u].LU_off, nd[u].size,
                      S + soff[root_of[u]] + (nd[u].off - nd[R.gid].off), rows, Vp[u], ldV(u), nd[u].size, ncV(u),
                      nd[u].size, 1.0, 0.0);
        } else {
          ds.push_back(LuSolveDescT<T>{luP<T>() + nd[u].LU_off,
                                       LUpiv.as<int>() + (int64_t)nd[u].leaf * m_max, Vp[u],
                                       nd[u].size, nd[u].size, ldV(u), ncV(u), dinvP<T>(u)});
        }
        const bool top_root = roots[root_of[u]].gid == u;
        if (!top_root || need_t) {
          T* dst;
          int ldd;
          tdst(u, dst, ldd);
          add_gemm<T>(g, pP<T>() + nd[u].P_off, nd[u].s, Vp[u], ldV(u), dst, ldd, nd[u].s, ncV(u),
                      nd[u].size, 1.0, 0.0);
        }
      }
      arena.clear();
      if (inv) {
        size_t o = arena.push(cps);
        char* base = upload_arena();
        copy_batched((const CopyDescT<T>*)(base + o), (int)cps.size(), max_cp, st);
        run_gemms(gl);
      } else {
        size_t o = arena.push(ds);
        char* base = upload_arena();
        prof().flops[pk_of<T>(PK_GETRS)] += getrs_flops(ds);
        getrs_batched((const LuSolveDescT<T>*)(base + o), (int)ds.size(), m_max, max_nc, st,
                      std::is_same<T, float>::value, pair_products<T>());
      }
      run_gemms(g);
    }
    // 2. heights 1 .. top
    for (int hh = 1; hh <= top; ++hh) {
      const bool invzh = invz && hh <= inv_zh;
      std::vector<CopyDescT<T>> cp;
      std::vector<LuSolveDescT<T>> zs;
      std::vector<GemmDescT<T>> g1, g2, gz;
      int64_t max_cp = 0;
      int max_n2 = 0, nodes_here = 0;
      for (int b : by_height[hh]) {
        if (root_of[b] < 0) continue;
        ++nodes_here;
        const int a = left(b), c = right(b);  // children: a left, c right
        const int sa = nd[a].s, sc = nd[c].s, nb2 = sa + sc, nc = ncV(b);
        max_n2 = std::max(max_n2, nb2);
        max_cp = std::max<int64_t>(max_cp, (int64_t)nb2 * nc);
        if (invzh) {  // y = Z^-1 t
          add_gemm<T>(gz, (const T*)Zi32.as<float>() + nd[b].Z_off, nb2, Tp(b), nb2, Yp(b), nb2, nb2, nc, nb2,
                      1.0, 0.0);
        } else {
          cp.push_back(CopyDescT<T>{Tp(b), Yp(b), nb2, nc, nb2, nb2});
          zs.push_back(LuSolveDescT<T>{zP<T>() + nd[b].Z_off, Zpiv.as<int>() + nd[b].Zpiv_off, Yp(b),
                                       nb2, nb2, nb2, nc, dinvP<T>(b)});
        }
        const T* W = wP<T>();
        // v_a -= W_{a c~} y1 (y1 = Y[sa : nb2]);  v_c -= W_{c a~} y2 (y2 = Y[0 : sa])
        add_gemm<T>(g1, W + nd[a].W_off, nd[a].size, Yp(b) + sa, nb2, Vp[a], ldV(b), nd[a].size, nc,
                    sc, -1.0, 1.0);
        add_gemm<T>(g1, W + nd[c].W_off, nd[c].size, Yp(b), nb2, Vp[c], ldV(b), nd[c].size, nc, sa,
                    -1.0, 1.0);
        const bool top_root = roots[root_of[b]].gid == b;
        if (!top_root || need_t) {
          const T* C = cP<T>();
          add_gemm<T>(g1, C + nd[b].CL_off, sa, Yp(b) + sa, nb2, Tp(b), nb2, sa, nc, sc, -1.0, 1.0);
          add_gemm<T>(g1, C + nd[b].CR_off, sc, Yp(b), nb2, Tp(b) + sa, nb2, sc, nc, sa, -1.0, 1.0);
          T* dst;
          int ldd;
          tdst(b, dst, ldd);
          add_gemm<T>(g2, pP<T>() + nd[b].P_off, nd[b].s, Tp(b), nb2, dst, ldd, nd[b].s, nc, nb2, 1.0,
                      0.0);
        }
      }
      if (nodes_here == 0) continue;
      std::vector<GemmTile> t1, t2, tz;
      const GemmShape sh1 = make_tiles(g1, t1, opt.gemm_tc != 0, !pair_products<T>()),
                      sh2 = make_tiles(g2, t2, opt.gemm_tc != 0, !pair_products<T>()),
                      shz = make_tiles(gz, tz, opt.gemm_tc != 0, !pair_products<T>());
      arena.clear();
      size_t ocp = arena.push(cp), ozs = arena.push(zs), og1 = arena.push(g1), ot1 = arena.push(t1),
             og2 = arena.push(g2), ot2 = arena.push(t2), ogz = arena.push(gz), otz = arena.push(tz);
      char* base = upload_arena();
      prof().flops[pk_of<T>(PK_GETRS)] += getrs_flops(zs);
      prof().flops[pair_products<T>() ? PK_GEMM_PAIR : pk_of<T>(PK_GEMM)] +=
          gemm_flops(g1) + gemm_flops(g2) + gemm_flops(gz);
      if (invzh) {
        launch_gemms((const GemmDescT<T>*)(base + ogz), (const GemmTile*)(base + otz), (int)tz.size(), shz);
      } else {
        copy_batched((const CopyDescT<T>*)(base + ocp), (int)cp.size(), max_cp, st);
        getrs_batched((const LuSolveDescT<T>*)(base + ozs), (int)zs.size(), max_n2, max_nc, st,
                      std::is_same<T, float>::value, pair_products<T>());
      }
      launch_gemms((const GemmDescT<T>*)(base + og1), (const GemmTile*)(base + ot1), (int)t1.size(), sh1);
      launch_gemms((const GemmDescT<T>*)(base + og2), (const GemmTile*)(base + ot2), (int)t2.size(), sh2);
    }
  }

  // ------------------------------------------------------------- factorization
  struct ProbIn {
    const double* X;
    int64_t N;
    double h, lam;
  };

  void factor(const std::vector<ProbIn>& in, bool on_device, bool concatenated, int d_, int leaf_m,
              int s_max_, double tol_) {
    factored = false;
    skeletonized = false;
    near_ready = false;
    slices_ready = false;
    xdig_ready = false;
    if (in.empty()) throw Error(IASKIT_ERR_ARG, "no problem");
    if (d_ < 1) throw Error(IASKIT_ERR_ARG, "d must be >= 1");
    if (leaf_m < 2) throw Error(IASKIT_ERR_ARG, "leaf_m must be >= 2");
    if (s_max_ < 1) throw Error(IASKIT_ERR_ARG, "s_max must be >= 1");
    int64_t total = 0;
    for (size_t q = 0; q < in.size(); ++q) {
      const ProbIn& p = in[q];
      if (p.N < 2) throw Error(IASKIT_ERR_ARG, "N must be >= 2");
      if (!(p.h > 0.0) || !std::isfinite(p.h)) throw Error(IASKIT_ERR_ARG, "h must be > 0");
      if (!(p.lam >= 0.0) || !std::isfinite(p.lam)) throw Error(IASKIT_ERR_ARG, "lambda must be >= 0");
      if (!p.X && (!concatenated || q == 0)) throw Error(IASKIT_ERR_ARG, "points is null");
      total += p.N;
    }
    if (total > ((int64_t)1 << 30)) throw Error(IASKIT_ERR_ARG, "more than 2^30 points");
    stats = Stats{};
    Ntot = (int)total;
    d = d_;
    s_max = s_max_;
    tol = tol_;
    prec = opt.precision;
    kspec = KernelSpec{opt.kernel, opt.poly_p, opt.poly_c};
    if (kspec.poly && opt.sampling == 1)
      throw Error(IASKIT_ERR_UNSUPPORTED, "learned sampling is built for the Gaussian kernel");
    use_kernel(kspec);
    const double t0 = now_ms();
    // problems and tree shapes (data independent)
    pr.assign(in.size(), Prob{});
    int pbase = 0, nbase = 0, min_n = Ntot;
    Hmax = 0;
    for (size_t q = 0; q < in.size(); ++q) {
      Prob& P = pr[q];
      P.N = (int)in[q].N;
      P.h = in[q].h;
      P.lam = in[q].lam;
      P.scale = kspec.poly ? 1.0 / (P.h * P.h) : -1.0 / (2.0 * P.h * P.h);
      P.pbase = pbase;
      P.nbase = nbase;
      P.L = 0;
      while ((P.N + (1 << P.L) - 1) / (1 << P.L) > leaf_m) ++P.L;
      if (P.L > 24) throw Error(IASKIT_ERR_UNSUPPORTED, "tree deeper than 24 levels");
      pbase += P.N;
      nbase += 2 << P.L;
      min_n = std::min(min_n, P.N);
      Hmax = std::max(Hmax, P.L);
    }
    kappa = std::min(opt.kappa, min_n - 1);
    nd.assign((size_t)nbase, Node{});
    by_height.assign(Hmax + 1, {});
    m_max = 0;
    nleaves = 0;
    for (size_t q = 0; q < pr.size(); ++q) {
      Prob& P = pr[q];
      Node& root = nd[P.nbase + 1];
      root.prob = (int)q;
      root.uid = 1;
      root.level = 0;
      root.off = P.pbase;
      root.size = P.N;
      for (int l = 0; l < P.L; ++l)
        for (int i = 0; i < (1 << l); ++i) {
          const int u = (1 << l) + i;
          const Node& p = nd[P.nbase + u];
          Node& a = nd[P.nbase + 2 * u];
          Node& b = nd[P.nbase + 2 * u + 1];
          a.prob = b.prob = (int)q;
          a.uid = 2 * u;
          b.uid = 2 * u + 1;
          a.level = b.level = l + 1;
          a.off = p.off;
          a.size = p.size / 2;
          b.off = p.off + a.size;
          b.size = p.size - a.size;
        }
      P.m_max = 0;
      for (int i = 0; i < (1 << P.L); ++i) P.m_max = std::max(P.m_max, nd[P.nbase + (1 << P.L) + i].size);
      m_max = std::max(m_max, P.m_max);
    }
    for (int hh = 0; hh <= Hmax; ++hh)
      for (size_t q = 0; q < pr.size(); ++q) {
        const int l = pr[q].L - hh;
        if (l < 0) continue;
        for (int i = 0; i < (1 << l); ++i) by_height[hh].push_back(pr[q].nbase + (1 << l) + i);
      }
    for (int g : by_height[0]) nd[g].leaf = nleaves++;
    if (m_max > 1536) throw Error(IASKIT_ERR_UNSUPPORTED, "leaf size above 1536");
    if (2 * s_max > 1536 && Hmax > 0) throw Error(IASKIT_ERR_UNSUPPORTED, "s_max above 768");

    status.ensure_n<int>(1);
    IA_CUDA(cudaMemsetAsync(status.as<int>(), 0, sizeof(int), st));
    double* Xd = X.ensure_n<double>((size_t)Ntot * d);
    if (concatenated) {
      IA_CUDA(cudaMemcpyAsync(Xd, in[0].X, (size_t)Ntot * d * sizeof(double),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else {
      for (size_t q = 0; q < pr.size(); ++q)
        IA_CUDA(cudaMemcpyAsync(Xd + (size_t)pr[q].pbase * d, in[q].X, (size_t)pr[q].N * d * sizeof(double),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    }
    check_finite(Xd, (int64_t)Ntot * d, status.as<int>(), st);
    raise_status(read_status_and_clear());
    {
      std::vector<int> hp(Ntot);
      for (size_t q = 0; q < pr.size(); ++q)
        std::fill(hp.begin() + pr[q].pbase, hp.begin() + pr[q].pbase + pr[q].N, (int)q);
      int* dp = pid.ensure_n<int>(Ntot);
      h2d(dp, hp.data(), hp.size(), st);
      IA_CUDA(cudaStreamSynchronize(st));
    }

    // a1: tree, one step per level from the root; finished problems pass through
    std::vector<TreeLevel> levels(Hmax);
    for (int l = 0; l < Hmax; ++l) {
      TreeLevel& lv = levels[l];
      for (size_t q = 0; q < pr.size(); ++q) {
        const Prob& P = pr[q];
        if (l < P.L) {
          for (int i = 0; i < (1 << l); ++i) {
            const Node& n = nd[P.nbase + (1 << l) + i];
            lv.off.push_back(n.off);
            lv.kleft.push_back(n.size / 2);
            lv.split.push_back(1);
          }
        } else {
          lv.off.push_back(P.pbase);
          lv.kleft.push_back(P.N);
          lv.split.push_back(0);
        }
      }
      lv.off.push_back(Ntot);
    }
    int* pm = perm.ensure_n<int>(Ntot);
    build_tree(Xd, Ntot, d, levels, pm, tree_s, st);
    permute_points(Xd, pm, Ntot, d, iperm.ensure_n<int>(Ntot), Xp.ensure_n<double>((size_t)Ntot * d), st);
    point_norms(Xp.as<double>(), Ntot, d, xnrm.ensure_n<double>(Ntot), st);
    if (prec == PREC_MIXED)  // coordinates as FP32 pairs for the operator blocks
      split_pairs(Xp.as<double>(), Xpair.ensure_n<float2>((size_t)Ntot * d), (int64_t)Ntot * d, st);
    choose_precisions();
    const double t1 = now_ms();
    stats.t_tree = t1 - t0;

    if (Hmax > 0) {
      // a2: kNN inside every problem
      std::vector<std::pair<int, int>> probs;
      for (const Prob& P : pr) probs.emplace_back(P.pbase, P.N);
      stats.knn_prune = KnnPruneStats{};
      if (opt.knn_prune) {
        // the search runs in the order of a finer tree of the same splitting rule, with
        // leaves of at most 128 points (one prefilter tile), so that every tile is a
        // compact box; its first levels are the levels of the method's tree
        std::vector<TreeLevel> kl;
        std::vector<std::vector<std::pair<int, int>>> cur(pr.size());
        int depth = 0;
        for (size_t q = 0; q < pr.size(); ++q) {
          cur[q] = {{pr[q].pbase, pr[q].N}};
          int Lq = 0;
          while ((pr[q].N + (1 << Lq) - 1) / (1 << Lq) > KNN_TILE) ++Lq;
          depth = std::max(depth, Lq);
        }
        for (int l = 0; l < depth; ++l) {
          TreeLevel lv;
          for (size_t q = 0; q < pr.size(); ++q) {
            std::vector<std::pair<int, int>> nxt;
            const bool splits = std::any_of(cur[q].begin(), cur[q].end(),
                                            [](const std::pair<int, int>& n) { return n.second > KNN_TILE; });
            if (!splits) {  // finished: one pass-through node for the whole problem
              lv.off.push_back(pr[q].pbase);
              lv.kleft.push_back(pr[q].N);
              lv.split.push_back(0);
              continue;
            }
            for (const auto& n : cur[q]) {
              lv.off.push_back(n.first);
              lv.kleft.push_back(n.second / 2);
              lv.split.push_back(1);
              nxt.push_back({n.first, n.second / 2});
              nxt.push_back({n.first + n.second / 2, n.second - n.second / 2});
            }
            cur[q] = nxt;
          }
          lv.off.push_back(Ntot);
          kl.push_back(lv);
        }
        int* kp = kperm.ensure_n<int>(Ntot);
        build_tree(Xd, Ntot, d, kl, kp, tree_s, st);
        permute_points(Xd, kp, Ntot, d, kiperm.ensure_n<int>(Ntot), Xk.ensure_n<double>((size_t)Ntot * d), st);
        stats.knn_fallback = knn_tree(Xk.as<double>(), kp, Ntot, d, kappa, knn.ensure_n<int>((size_t)Ntot * kappa),
                                      probs, knn_s, st, &stats.knn_prune);
      } else {
        stats.knn_fallback =
            knn_bruteforce(Xd, Ntot, d, kappa, knn.ensure_n<int>((size_t)Ntot * kappa), probs, knn_s, st);
      }
      IA_CUDA(cudaStreamSynchronize(st));
      const double t2 = now_ms();
      stats.t_knn = t2 - t1;
      if (prec == PREC_MIXED) skeletonize<float>();
      else skeletonize<double>();
      IA_CUDA(cudaStreamSynchronize(st));
      stats.t_skel = now_ms() - t2;
    }
    skeletonized = true;
    const double t3 = now_ms();
    leaf_lu();
    raise_status(read_status_and_clear());
    const double t4 = now_ms();
    stats.t_leaf_lu = t4 - t3;
    factor_levels();
    raise_status(read_status_and_clear());
    stats.t_factor_levels = now_ms() - t4;
    stats.t_factor = now_ms() - t0;
    prof().resolve();
    factored = true;
  }

  // Factorization of lambda' I + K~ for new regularizations lambda' (Sec. II-C: the
  // skeletons and the P matrices do not depend on lambda, so a new lambda recomputes
  // only the leaf LUs, W and the reduced systems Z).  The tree, the kNN lists, the
  // samples, the skeletons and P are kept; the leaf blocks lambda' I + K_aa, the U
  // blocks, W and Z are formed again, in the form (plain or mixed) of the kept
  // factorization.  The mixed form re-chooses each problem's precisions, since the
  // condition estimate 1 + r / lambda' changes with lambda'.
  void refactor(const double* lam, int nprob) {
    if (!lam) throw Error(IASKIT_ERR_ARG, "lambda is null");
    if (nprob != (int)pr.size()) throw Error(IASKIT_ERR_ARG, "one lambda per factored problem");
    for (int q = 0; q < nprob; ++q)
      if (!(lam[q] >= 0.0) || !std::isfinite(lam[q])) throw Error(IASKIT_ERR_ARG, "lambda must be >= 0");
    factored = false;
    slices_ready = false;
    use_kernel(kspec);
    const double t0 = now_ms();
    for (int q = 0; q < nprob; ++q) pr[q].lam = lam[q];
    stats.t_tree = stats.t_knn = stats.t_skel = 0.0;
    stats.t_solve = stats.t_apply = 0.0;
    stats.bytes_operator = 0;
    stats.bytes_slices = 0;
    stats.refine_hist.clear();
    stats.refine_sweeps = stats.refine_iters = stats.refine_stagnated = 0;
    choose_precisions();
    const double t1 = now_ms();
    leaf_lu();
    raise_status(read_status_and_clear());
    const double t2 = now_ms();
    stats.t_leaf_lu = t2 - t1;
    factor_levels();
    raise_status(read_status_and_clear());
    stats.t_factor_levels = now_ms() - t2;
    stats.t_factor = now_ms() - t0;
    prof().resolve();
    factored = true;
  }

  // Per problem: cond_est = 1 + r / lambda with r the largest of KROWSUM_ROWS sampled kernel
  // row sums (an estimate of ||K||_2 and of the largest eigenvalue of lambda I + K, whose
  // smallest is about lambda).  The plain form factors every problem in FP64; the mixed
  // form factors a problem in FP32 only while cond_est <= mixed_cond_max, so that the
  // FP32 factorization keeps a few correct digits and refinement converges quickly.
  void choose_precisions() {
    std::vector<RowSumDesc> rd(pr.size());
    for (size_t q = 0; q < pr.size(); ++q) rd[q] = RowSumDesc{pr[q].pbase, pr[q].N, pr[q].scale};
    arena.clear();
    size_t o = arena.push(rd);
    char* base = upload_arena();
    double* rs = rowsum.ensure_n<double>(pr.size() * KROWSUM_ROWS);
    int max_n = 0;
    for (const Prob& P : pr) max_n = std::max(max_n, P.N);
    kernel_rowsums(Xp.as<double>(), d, (const RowSumDesc*)(base + o), (int)pr.size(), max_n, rs, st);
    std::vector<double> hrs(pr.size() * KROWSUM_ROWS);
    d2h(hrs.data(), rs, hrs.size(), st);
    IA_CUDA(cudaStreamSynchronize(st));
    stats.fp64_problems = 0;
    stats.fp64_operator_problems = 0;
    stats.operator_upgrades = 0;
    for (size_t q = 0; q < pr.size(); ++q) {
      double mx = 0.0;
      for (int r = 0; r < KROWSUM_ROWS; ++r) mx = std::max(mx, hrs[q * KROWSUM_ROWS + r]);
      Prob& P = pr[q];
      P.cond_est = P.lam > 0.0 ? 1.0 + mx / P.lam : HUGE_VAL;
      P.f64 = prec != PREC_MIXED || !(P.cond_est <= opt.mixed_cond_max);
      P.op64 = prec == PREC_MIXED && !(P.cond_est <= opt.pair_cond_max);
      stats.fp64_problems += P.f64 ? 1 : 0;
      stats.fp64_operator_problems += P.op64 ? 1 : 0;
    }
  }

  // ------------------------------------------------------------ sampling steps
  // One sampling step (height hh): the node list covering all points (problems with no
  // node at this height pass through), uploaded, and the plain samples of its nodes.
  struct StepLists {
    std::vector<int> nodes;            // gids of the height's non-root nodes
    std::vector<int> off;              // nn + 1 offsets
    std::vector<SampleNodeInfo> info;  // nn entries
    std::vector<int> gid;              // nn entries: the node's gid, -1 for a pass-through
    int* od = nullptr;
    SampleNodeInfo* id = nullptr;
  };
  void sample_step(int hh, int samp_cap, int* sp, StepLists& L) {
    L = StepLists{};
    for (int g : by_height[hh])
      if (!is_root(g)) L.nodes.push_back(g);
    if (L.nodes.empty()) return;
    size_t k = 0;
    for (size_t q = 0; q < pr.size(); ++q) {
      const Prob& P = pr[q];
      const int l = P.L - hh;
      if (l >= 1) {
        for (int i = 0; i < (1 << l); ++i) {
          const int g = L.nodes[k++];
          const Node& n = nd[g];
          L.off.push_back(n.off);
          L.info.push_back(SampleNodeInfo{P.pbase, P.N, n.uid, (int)n.samp_off, 1});
          L.gid.push_back(g);
        }
      } else {
        L.off.push_back(P.pbase);
        L.info.push_back(SampleNodeInfo{P.pbase, P.N, 0, 0, 0});
        L.gid.push_back(-1);
      }
    }
    L.off.push_back(Ntot);
    const int nn = (int)L.info.size();
    L.od = step_dev.ensure_n<int>(nn + 1 + (int64_t)nn * (sizeof(SampleNodeInfo) / sizeof(int)));
    h2d(L.od, L.off.data(), nn + 1, st);
    L.id = reinterpret_cast<SampleNodeInfo*>(L.od + nn + 1);
    h2d(L.id, L.info.data(), L.info.size(), st);
    sample_level(knn_pos.as<int>(), Ntot, kappa, L.od, L.id, L.off, L.info, samp_cap, opt.seed, sp,
                 status.as<int>(), samp_s, st);
  }

  // ID columns of node g as a KDesc/feature column spec
  void cols_of(int g, const int*& colsA, const int*& colsB, int& col0, int& nA, int& ncols) const {
    const Node& n = nd[g];
    if (is_leaf(g)) {
      colsA = colsB = nullptr;
      col0 = n.off;
      nA = 0;
      ncols = n.size;
    } else {
      const int* sk = skel.as<int>();
      colsA = sk + (size_t)left(g) * s_max;
      colsB = sk + (size_t)right(g) * s_max;
      col0 = 0;
      nA = nd[left(g)].s;
      ncols = nA + nd[right(g)].s;
    }
  }

  // Candidates and features of the learned proposal for the nodes of a step right after
  // its sample_level (which left the kNN candidate ranking in samp_s).  Fills li (nn
  // entries, uploaded to l_linfo) and l_cand / l_hits / l_feat; returns the nodes
  // with candidates and their total count in tot.
  std::vector<int> learned_candidates_step(const StepLists& L, std::vector<LearnNodeInfo>& li,
                                           int64_t& tot, int& max_cand) {
    const int nn = (int)L.info.size();
    li.assign(nn, LearnNodeInfo{0, 0, 0});
    std::vector<int> out;
    tot = 0;
    max_cand = 0;
    for (int e = 0; e < nn; ++e) {
      const int g = L.gid[e];
      if (g < 0) continue;
      const Node& n = nd[g];
      const int comp = pr[n.prob].N - n.size;
      if (n.nsamp <= 0 || n.nsamp >= comp) continue;
      const int nc = (int)std::min<int64_t>((int64_t)opt.cand_factor * n.nsamp, comp);
      li[e] = LearnNodeInfo{(int)tot, nc, n.nsamp};
      tot += nc;
      max_cand = std::max(max_cand, nc);
      out.push_back(g);
    }
    if (out.empty()) return out;
    if (tot > (int64_t)INT_MAX / 8) throw Error(IASKIT_ERR_UNSUPPORTED, "too many learned candidates");
    int* cand = l_cand.ensure_n<int>(tot);
    float* hits = l_hits.ensure_n<float>(tot);
    uint16_t* feat = l_feat.ensure_n<uint16_t>(tot * 8);
    LearnNodeInfo* lid = l_linfo.ensure_n<LearnNodeInfo>(nn);
    h2d(lid, li.data(), nn, st);
    int pos_bits = 0;
    while (((uint64_t)1 << pos_bits) <= (uint64_t)Ntot) ++pos_bits;
    learned_candidates(samp_s.vals2.as<uint32_t>(), samp_s.keys2.as<uint64_t>(), samp_s.node_start.as<int>(),
                       samp_s.node_cnt.as<int>(), pos_bits, L.od, L.id, lid, nn, opt.seed, max_cand, cand,
                       hits, status.as<int>(), st);
    std::vector<LearnFeatDesc> fd;
    for (int e = 0; e < nn; ++e) {
      if (li[e].n_cand <= 0) continue;
      const int g = L.gid[e];
      const Node& n = nd[g];
      const Prob& P = pr[n.prob];
      LearnFeatDesc f{};
      cols_of(g, f.colsA, f.colsB, f.col0, f.nA, f.ncols);
      f.cand = cand + li[e].cand_off;
      f.hits = hits + li[e].cand_off;
      f.n_cand = li[e].n_cand;
      f.cand_off = li[e].cand_off;
      f.f4 = (float)(n.level / (double)std::max(P.L, 1));
      f.f5 = (float)(std::log2((double)n.size) / std::log2((double)P.N));
      f.inv_h = (float)(1.0 / P.h);
      f.inv_log1p_kappa = (float)(1.0 / std::log1p((double)kappa));
      f.scale = P.scale;
      fd.push_back(f);
    }
    arena.clear();
    size_t of = arena.push(fd);
    char* base = upload_arena();
    learned_features(Xp.as<double>(), d, (const LearnFeatDesc*)(base + of), (int)fd.size(), max_cand, feat, st);
    return out;
  }

  // stratified row draw of node g (sibling half, outside-the-parent half)
  StreamDesc strat_desc(int g, int out_off) const {
    const Node& n = nd[g];
    const Prob& P = pr[n.prob];
    const Node& sb = nd[sibling(g)];
    const Node& pa = nd[parent(g)];
    return StreamDesc{P.pbase, P.N, n.uid, out_off, sb.off - P.pbase, sb.size, pa.off - P.pbase, pa.size};
  }
  void strat_weights(int g, int count, int& cs, double& ws, double& wr) const {
    const Node& sb = nd[sibling(g)];
    const int far = pr[nd[g].prob].N - nd[parent(g)].size;
    cs = far == 0 ? count : count / 2;
    ws = (double)sb.size / cs;
    wr = far == 0 ? 0.0 : (double)far / (count - cs);
  }

  MlpDev mlp_dev() {
    uint16_t* b = mlp_b16.as<uint16_t>();
    return MlpDev{mlp_master.as<float>(), b, b + 1024, b + 1024 + 16384, b + 1024 + 2 * 16384};
  }
  void mlp_alloc() {
    mlp_master.ensure_n<float>(MLP_NPARAM);
    mlp_m.ensure_n<float>(MLP_NPARAM);
    mlp_v.ensure_n<float>(MLP_NPARAM);
    mlp_grad.ensure_n<float>(MLP_NPARAM);
    mlp_b16.ensure_n<uint16_t>(1024 + 2 * 16384 + 128);
    mlp_loss.ensure_n<float>(1);
  }
  // new master weights: Adam state cleared, BF16 copies refreshed
  void mlp_load(const float* host) {
    mlp_alloc();
    h2d(mlp_master.as<float>(), host, MLP_NPARAM, st);
    IA_CUDA(cudaMemsetAsync(mlp_m.p, 0, MLP_NPARAM * sizeof(float), st));
    IA_CUDA(cudaMemsetAsync(mlp_v.p, 0, MLP_NPARAM * sizeof(float), st));
    IA_CUDA(cudaMemsetAsync(mlp_grad.p, 0, MLP_NPARAM * sizeof(float), st));
    mlp_refresh_copies(mlp_dev(), st);
    IA_CUDA(cudaStreamSynchronize(st));
    mlp_step = 0;
    mlp_ready = true;
  }

  // Kept candidates for introspection (option keep_candidates): per node gid.
  struct Kept {
    int64_t off = -1;
    int n = 0, n_samp = 0, chosen = -1;
    double err_plain = 0, err_learned = 0;
  };
  std::vector<Kept> kept;
  std::vector<int> kept_cand;
  std::vector<uint16_t> kept_feat;
  std::vector<float> kept_val;
  void keep_step(const StepLists& L, const std::vector<LearnNodeInfo>& li, int64_t tot, const float* val) {
    if (!opt.keep_candidates || tot == 0) return;
    const int64_t base = (int64_t)kept_cand.size();
    kept_cand.resize(base + tot);
    kept_feat.resize((base + tot) * 8);
    kept_val.resize(base + tot);
    d2h(kept_cand.data() + base, l_cand.as<int>(), tot, st);
    d2h(kept_feat.data() + base * 8, l_feat.as<uint16_t>(), tot * 8, st);
    d2h(kept_val.data() + base, val, tot, st);
    IA_CUDA(cudaStreamSynchronize(st));
    for (size_t e = 0; e < li.size(); ++e)
      if (li[e].n_cand > 0) {
        Kept& k = kept[L.gid[e]];
        k.off = base + li[e].cand_off;
        k.n = li[e].n_cand;
        k.n_samp = li[e].n_samp;
      }
  }

  // a3 + a4 + a5: skeletons, heights 0 .. Hmax-1 (roots excluded); TS is the
  // precision of the sampled blocks and of the Householder updates.  With learned
  // sampling every eligible node also takes the ID of its learned sample, and the
  // held-out error of the two IDs picks the one it keeps.
  template <typename TS>
  void skeletonize() {
    int* kp = knn_pos.ensure_n<int>((size_t)Ntot * kappa);
    knn_to_positions(knn.as<int>(), perm.as<int>(), iperm.as<int>(), Ntot, kappa, kp, st);
    const int samp_cap = opt.samp_factor * s_max;
    int64_t tot = 0;
    for (int hh = 0; hh <= Hmax; ++hh)
      for (int g : by_height[hh]) {
        if (is_root(g)) continue;
        Node& n = nd[g];
        n.nsamp = std::min(samp_cap, pr[n.prob].N - n.size);
        n.samp_off = tot;
        tot += n.nsamp;
      }
    const bool learn = opt.sampling == 1;
    if (learn && !mlp_ready) throw Error(IASKIT_ERR_ARG, "learned sampling needs trained or set weights");
    int* sp = samp.ensure_n<int>(std::max<int64_t>(tot, 1));
    int* lsp = learn ? l_samp.ensure_n<int>(std::max<int64_t>(tot, 1)) : nullptr;
    int* rk = ranks.ensure_n<int>(nd.size());
    int* rkl = learn ? l_rk.ensure_n<int>(nd.size()) : nullptr;
    IA_CUDA(cudaMemsetAsync(rk, 0, nd.size() * sizeof(int), st));
    int* sk = skel.ensure_n<int>(nd.size() * (size_t)s_max);
    kept.assign(opt.keep_candidates ? nd.size() : 0, Kept{});
    kept_cand.clear();
    kept_feat.clear();
    kept_val.clear();
    int64_t p_total = 0;
    std::vector<int> rall(nd.size(), 0), rlrn(learn ? nd.size() : 0, 0);
    for (int hh = 0; hh < Hmax; ++hh) {
      StepLists S;
      sample_step(hh, samp_cap, sp, S);
      const std::vector<int>& nodes = S.nodes;
      if (nodes.empty()) continue;
      // learned proposal: candidates, features, scores, the best n_samp of each node
      std::vector<int> lnodes;
      std::vector<LearnNodeInfo> li;
      int64_t ctot = 0;
      if (learn) {
        int max_cand = 0;
        lnodes = learned_candidates_step(S, li, ctot, max_cand);
        if (!lnodes.empty()) {
          float* score = l_score.ensure_n<float>(ctot);
          mlp_forward(l_feat.as<uint16_t>(), ctot, mlp_dev(), score, nullptr, nullptr, st);
          perturb_scores(score, l_linfo.as<LearnNodeInfo>(), S.id, (int)S.info.size(), max_cand, opt.seed,
                         opt.learned_temp, st);
          learned_select(score, l_cand.as<int>(), l_linfo.as<LearnNodeInfo>(), S.id, (int)S.info.size(),
                         max_cand, lsp, st);
          keep_step(S, li, ctot, score);
        }
      }
      // sampled blocks and IDs: plain [0, nk), learned [nk, nk + nl)
      const int nk = (int)nodes.size(), nl = (int)lnodes.size(), nt = nk + nl;
      auto node_of = [&](int i) { return i < nk ? nodes[i] : lnodes[i - nk]; };
      int64_t asz = 0, pvsz = 0, max_e = 0;
      int max_r = 0, max_c = 0;
      std::vector<int64_t> aoff(nt), poff(nt);
      for (int i = 0; i < nt; ++i) {
        Node& n = nd[node_of(i)];
        n.ncols = is_leaf(node_of(i)) ? n.size : n2(node_of(i));
        aoff[i] = asz;
        poff[i] = pvsz;
        asz += (int64_t)n.nsamp * n.ncols;
        pvsz += n.ncols;
        max_e = std::max<int64_t>(max_e, (int64_t)n.nsamp * n.ncols);
        max_r = std::max(max_r, n.nsamp);
        max_c = std::max(max_c, n.ncols);
      }
      TS* A = A_ws.ensure_n<TS>(asz);
      int* pv = piv_ws.ensure_n<int>(pvsz);
      std::vector<KDescT<TS>> kd(nt);
      std::vector<CpqrDescT<TS>> qd(nt);
      for (int i = 0; i < nt; ++i) {
        const int g = node_of(i);
        Node& n = nd[g];
        KDescT<TS> k{};
        k.rows = (i < nk ? sp : lsp) + n.samp_off;
        k.nrows = n.nsamp;
        k.out = A + aoff[i];
        k.ld = n.nsamp;
        k.ncols = n.ncols;
        k.diag = 0.0;
        k.scale = scale_of(g);
        cols_of(g, k.colsA, k.colsB, k.col0, k.nA, k.ncols);
        kd[i] = k;
        qd[i] = CpqrDescT<TS>{A + aoff[i], pv + poff[i], (i < nk ? rk : rkl) + g, n.nsamp, n.nsamp, n.ncols};
      }
      arena.clear();
      size_t ok = arena.push(kd), oq = arena.push(qd);
      char* base = upload_arena();
      prof().flops[pk_of<TS>(PK_KBLOCK)] += kblock_flops(kd, d);
      kernel_blocks<TS>(Xp.as<double>(), xnrm.as<double>(), d, (const KDescT<TS>*)(base + ok), nt, max_e, st);
      cpqr_id<TS>((const CpqrDescT<TS>*)(base + oq), nt, max_r, max_c, s_max, tol, st, opt.cpqr_cluster != 0);
      d2h(rall.data(), rk, nd.size(), st);
      if (nl) d2h(rlrn.data(), rkl, nd.size(), st);
      IA_CUDA(cudaStreamSynchronize(st));
      raise_status(read_status_and_clear());
      std::vector<int> rank_of(nt);
      double qr_flops = 0;
      for (int i = 0; i < nt; ++i) {
        const Node& n = nd[node_of(i)];
        rank_of[i] = i < nk ? rall[node_of(i)] : rlrn[node_of(i)];
        // Householder update (dot + axpy) and norm recomputation per step
        for (int k = 0; k < rank_of[i]; ++k) qr_flops += 6.0 * (n.nsamp - k) * (double)(n.ncols - k);
      }
      prof().flops[pk_of<TS>(PK_CPQR)] += qr_flops;
      {  // T = R11^{-1} R12 in place (the ID), many blocks per node
        std::vector<LuSolveDescT<TS>> td;
        int max_s = 0, max_t = 0;
        for (int i = 0; i < nt; ++i) {
          const Node& n = nd[node_of(i)];
          const int si = rank_of[i], ti = n.ncols - si;
          if (si <= 0 || ti <= 0) continue;
          td.push_back(LuSolveDescT<TS>{A + aoff[i], nullptr, A + aoff[i] + (size_t)si * n.nsamp, si, n.nsamp,
                                        n.nsamp, ti});
          max_s = std::max(max_s, si);
          max_t = std::max(max_t, ti);
        }
        if (!td.empty()) {
          arena.clear();
          size_t otd = arena.push(td);
          base = upload_arena();
          prof().flops[pk_of<TS>(PK_GETRS)] += getrs_flops(td) / 2;  // one triangle
          trsm_upper_batched<TS>((const LuSolveDescT<TS>*)(base + otd), (int)td.size(), max_s, max_t, st);
        }
      }
      // P and skeletons of every ID: straight into the final storage without learning,
      // else into temporaries from which the chosen ID is copied
      std::vector<int> chosen(nk);  // descriptor index kept by plain node i
      for (int i = 0; i < nk; ++i) chosen[i] = i;
      std::vector<int64_t> ptoff(nt);
      int64_t ptsz = 0;
      for (int i = 0; i < nt; ++i) {
        ptoff[i] = ptsz;
        ptsz += (int64_t)rank_of[i] * nd[node_of(i)].ncols;
      }
      double* Pt = nl ? l_Ptmp.ensure_n<double>(std::max<int64_t>(ptsz, 1)) : nullptr;
      int* skt = nl ? l_sktmp.ensure_n<int>((size_t)nt * s_max) : nullptr;
      if (nl) {
        std::vector<PDescT<TS>> pd(nt);
        for (int i = 0; i < nt; ++i) {
          const int g = node_of(i);
          const Node& n = nd[g];
          PDescT<TS> pp{};
          pp.A = A + aoff[i];
          pp.piv = pv + poff[i];
          pp.P = Pt + ptoff[i];
          pp.skel = skt + (size_t)i * s_max;
          pp.ld = n.nsamp;
          pp.s = rank_of[i];
          int ncols_unused;
          cols_of(g, pp.colsA, pp.colsB, pp.col0, pp.nA, ncols_unused);
          pp.ncols = n.ncols;
          pd[i] = pp;
        }
        arena.clear();
        size_t op = arena.push(pd);
        base = upload_arena();
        assemble_P<TS>((const PDescT<TS>*)(base + op), nt, max_c, st);
        // judge: held-out rows, then both IDs' errors
        std::vector<StreamDesc> sd(nl);
        std::vector<int> plain_idx(nl);
        std::vector<int> pos_of(nd.size(), -1);
        for (int i = 0; i < nk; ++i) pos_of[nodes[i]] = i;
        for (int j = 0; j < nl; ++j) {
          const int g = lnodes[j];
          const Node& n = nd[g];
          const Prob& P = pr[n.prob];
          sd[j] = strat_desc(g, j * NHOLD);
          plain_idx[j] = pos_of[g];
        }
        int* hold = l_hold.ensure_n<int>((size_t)nl * NHOLD);
        std::vector<JudgeDesc> jd(2 * nl);
        int max_s = 1;
        for (int j = 0; j < nl; ++j)
          for (int v = 0; v < 2; ++v) {
            const int i = v == 0 ? plain_idx[j] : nk + j;
            const int g = lnodes[j];
            JudgeDesc J{};
            J.H = hold + (size_t)j * NHOLD;
            strat_weights(g, NHOLD, J.nh_s, J.w_s, J.w_r);
            cols_of(g, J.colsA, J.colsB, J.col0, J.nA, J.ncols);
            J.skel = skt + (size_t)i * s_max;
            J.s = rank_of[i];
            J.P = Pt + ptoff[i];
            J.scale = scale_of(g);
            jd[2 * j + v] = J;
            max_s = std::max(max_s, J.s);
          }
        arena.clear();
        size_t os = arena.push(sd), oj = arena.push(jd);
        base = upload_arena();
        stream_rows((const StreamDesc*)(base + os), nl, NHOLD, opt.seed, HOLD_SALT, hold, st);
        double* errd = l_err.ensure_n<double>((size_t)4 * nl);
        id_judge(Xp.as<double>(), d, (const JudgeDesc*)(base + oj), 2 * nl, NHOLD, max_s, errd, st);
        std::vector<double> err(4 * (size_t)nl);
        d2h(err.data(), errd, err.size(), st);
        IA_CUDA(cudaStreamSynchronize(st));
        std::vector<ConvSeg> sseg;
        for (int j = 0; j < nl; ++j) {
          const double ep = err[4 * j + 1] > 0 ? err[4 * j] / err[4 * j + 1] : 0.0;
          const double el = err[4 * j + 3] > 0 ? err[4 * j + 2] / err[4 * j + 3] : 0.0;
          const bool take = el <= ep;
          const Node& n = nd[lnodes[j]];
          if (take) {
            chosen[plain_idx[j]] = nk + j;
            sseg.push_back(ConvSeg{n.samp_off, n.samp_off, n.nsamp});
            ++stats.learned_nodes;
          } else {
            ++stats.fallback_nodes;
          }
          stats.judge_err_plain += ep;
          stats.judge_err_chosen += take ? el : ep;
          ++stats.judged_nodes;
          if (opt.keep_candidates) {
            Kept& kk = kept[lnodes[j]];
            kk.chosen = take ? 1 : 0;
            kk.err_plain = ep;
            kk.err_learned = el;
          }
        }
        conv_segs<int, int>(lsp, sp, sseg);  // the kept sample of every node that took the learned one
      }
      int64_t psz = 0;
      for (int i = 0; i < nk; ++i) {
        Node& n = nd[nodes[i]];
        n.s = rank_of[chosen[i]];
        rall[nodes[i]] = n.s;
        n.P_off = p_total + psz;
        psz += (int64_t)n.s * n.ncols;
      }
      // P storage grows by height; earlier heights are copied along when it grows
      if ((p_total + psz) * (int64_t)sizeof(double) > (int64_t)Pd.bytes) {
        DevBuf tmp;
        double* t = tmp.ensure_n<double>(std::max<int64_t>(p_total, 1));
        if (p_total)
          IA_CUDA(cudaMemcpyAsync(t, Pd.as<double>(), p_total * sizeof(double), cudaMemcpyDeviceToDevice, st));
        IA_CUDA(cudaStreamSynchronize(st));
        Pd.ensure_n<double>(2 * (p_total + psz));
        if (p_total)
          IA_CUDA(cudaMemcpyAsync(Pd.as<double>(), t, p_total * sizeof(double), cudaMemcpyDeviceToDevice, st));
        IA_CUDA(cudaStreamSynchronize(st));
      }
      double* P = Pd.as<double>();
      if (nl) {
        std::vector<ConvSeg> pseg, kseg;
        for (int i = 0; i < nk; ++i) {
          const Node& n = nd[nodes[i]];
          pseg.push_back(ConvSeg{ptoff[chosen[i]], n.P_off, (int64_t)n.s * n.ncols});
          kseg.push_back(ConvSeg{(int64_t)chosen[i] * s_max, (int64_t)nodes[i] * s_max, n.s});
        }
        conv_segs<double, double>(Pt, P, pseg);
        conv_segs<int, int>(skt, sk, kseg);
        h2d(rk, rall.data(), nd.size(), st);
      } else {
        std::vector<PDescT<TS>> pd(nk);
        for (int i = 0; i < nk; ++i) {
          const int g = nodes[i];
          Node& n = nd[g];
          PDescT<TS> pp{};
          pp.A = A + aoff[i];
          pp.piv = pv + poff[i];
          pp.P = P + n.P_off;
          pp.skel = sk + (size_t)g * s_max;
          pp.ld = n.nsamp;
          pp.s = n.s;
          int ncols_unused;
          cols_of(g, pp.colsA, pp.colsB, pp.col0, pp.nA, ncols_unused);
          pp.ncols = n.ncols;
          pd[i] = pp;
        }
        arena.clear();
        size_t op = arena.push(pd);
        base = upload_arena();
        assemble_P<TS>((const PDescT<TS>*)(base + op), nk, max_c, st);
      }
      p_total += psz;
      stats.bytes_P += psz * 8;
    }
    if (prec == PREC_MIXED && p_total > 0) {
      convert_d2f(Pd.as<double>(), Pf.ensure_n<float>(p_total), p_total, st);
      split_pairs(Pd.as<double>(), Ppair.ensure_n<float2>(p_total), p_total, st);
    }
  }

  // ------------------------------------------------------- sampler training
  // Labels for every node of a training problem, then Adam epochs on the MLP.  The
  // problem is factored in FP64 with plain sampling (lambda = 1); that factorization
  // stays current.  Per height, for each node with a learned candidate set: B = K(gram
  // rows, cols) over NGRAM stratified rows and its transpose, G = B^T diag(w) B + mu I,
  // the LU of G, and the candidates' ridge leverage b_c^T G^{-1} b_c as standardized
  // log targets.
  void train_sampler(const double* Xh, int64_t N, int d_, double h, int leaf_m, int s_max_, double tol_,
                     int epochs, double lr) {
    if (epochs < 0 || epochs > 100000) throw Error(IASKIT_ERR_ARG, "invalid epochs");
    if (!(lr > 0.0) || !std::isfinite(lr)) throw Error(IASKIT_ERR_ARG, "invalid learning rate");
    if (opt.kernel != 0) throw Error(IASKIT_ERR_UNSUPPORTED, "learned sampling is built for the Gaussian kernel");
    const Options saved = opt;
    opt.sampling = 0;
    opt.precision = PREC_FP64;
    try {
      factor({ProbIn{Xh, N, h, 1.0}}, false, false, d_, leaf_m, s_max_, tol_);
    } catch (...) {
      opt = saved;
      throw;
    }
    opt = saved;
    const int samp_cap = opt.samp_factor * s_max;
    kept.assign(opt.keep_candidates ? nd.size() : 0, Kept{});
    kept_cand.clear();
    kept_feat.clear();
    kept_val.clear();
    const double tol2 = tol > 0 ? tol * tol : 1e-12;
    int64_t rows = 0;
    // first pass: candidate counts per height for the training arrays
    std::vector<int64_t> per_h(Hmax, 0);
    for (int hh = 0; hh < Hmax; ++hh)
      for (int g : by_height[hh]) {
        if (is_root(g)) continue;
        const Node& n = nd[g];
        const int comp = pr[n.prob].N - n.size;
        if (n.nsamp > 0 && n.nsamp < comp) per_h[hh] += std::min<int64_t>((int64_t)opt.cand_factor * n.nsamp, comp);
      }
    const int64_t total = std::accumulate(per_h.begin(), per_h.end(), (int64_t)0);
    if (total == 0) throw Error(IASKIT_ERR_ARG, "training problem has no node with a candidate set");
    if (total > (int64_t)INT_MAX / 8) throw Error(IASKIT_ERR_UNSUPPORTED, "training set too large");
    uint16_t* TF = tr_feat.ensure_n<uint16_t>(total * 8);
    float* TT = tr_tgt.ensure_n<float>(total);
    double* TL = tr_lev.ensure_n<double>(total);
    for (int hh = 0; hh < Hmax; ++hh) {
      if (per_h[hh] == 0) continue;
      StepLists S;
      sample_step(hh, samp_cap, samp.as<int>(), S);
      std::vector<LearnNodeInfo> li;
      int64_t ctot = 0;
      int max_cand = 0;
      const std::vector<int> lnodes = learned_candidates_step(S, li, ctot, max_cand);
      IA_CUDA(cudaMemcpyAsync(TF + rows * 8, l_feat.p, ctot * 8 * sizeof(uint16_t), cudaMemcpyDeviceToDevice, st));
      // node -> its candidate range inside this step
      std::vector<int> cand_off(nd.size(), -1), ncand(nd.size(), 0);
      for (size_t e = 0; e < li.size(); ++e)
        if (li[e].n_cand > 0) {
          cand_off[S.gid[e]] = li[e].cand_off;
          ncand[S.gid[e]] = li[e].n_cand;
        }
      // nodes in chunks of at most ~4e8 doubles of dense blocks
      size_t j0 = 0;
      while (j0 < lnodes.size()) {
        size_t j1 = j0;
        int64_t dsz = 0;
        while (j1 < lnodes.size()) {
          const Node& n = nd[lnodes[j1]];
          const int64_t need = 2 * (int64_t)n.ncols * NGRAM + (int64_t)n.ncols * n.ncols +
                               2 * (int64_t)n.ncols * ncand[lnodes[j1]];
          if (j1 > j0 && dsz + need > (int64_t)400000000) break;
          dsz += need;
          ++j1;
        }
        const int nl = (int)(j1 - j0);
        std::vector<ColsDesc> cd(nl);
        std::vector<StreamDesc> sd(nl);
        int64_t csz = 0;
        std::vector<int64_t> coff(nl), boff(nl), toff(nl), goff(nl), c1off(nl), c2off(nl);
        int64_t o = 0;
        int max_nc = 0, max_ncand = 0;
        int64_t max_bt = 0, max_b = 0, max_c = 0;
        for (int j = 0; j < nl; ++j) {
          const int g = lnodes[j0 + j];
          const Node& n = nd[g];
          const Prob& P = pr[n.prob];
          ColsDesc c{};
          int nc;
          cols_of(g, c.colsA, c.colsB, c.col0, c.nA, nc);
          c.ncols = nc;
          c.out_off = (int)csz;
          cd[j] = c;
          coff[j] = csz;
          csz += nc;
          sd[j] = strat_desc(g, j * NGRAM);
          toff[j] = o;  o += (int64_t)nc * NGRAM;   // K(cols, gram), nc x NGRAM
          boff[j] = o;  o += (int64_t)nc * NGRAM;   // K(gram, cols), NGRAM x nc
          goff[j] = o;  o += (int64_t)nc * nc;      // G
          c1off[j] = o; o += (int64_t)nc * ncand[g];
          c2off[j] = o; o += (int64_t)nc * ncand[g];
          max_nc = std::max(max_nc, nc);
          max_ncand = std::max(max_ncand, ncand[g]);
          max_bt = std::max<int64_t>(max_bt, (int64_t)nc * NGRAM);
          max_c = std::max<int64_t>(max_c, (int64_t)nc * ncand[g]);
        }
        max_b = max_bt;
        int* cols = l_cols.ensure_n<int>(std::max<int64_t>(csz, 1));
        int* gram = l_gram.ensure_n<int>((size_t)nl * NGRAM);
        double* D = l_dense.ensure_n<double>(std::max<int64_t>(o, 1));
        int* gpiv = piv_ws.ensure_n<int>((size_t)nl * max_nc);
        std::vector<KDesc> kt, kb, kc;
        std::vector<GemmDesc> gg;
        std::vector<RidgeDesc> rd;
        std::vector<LuDesc> ld;
        std::vector<LuSolveDesc> ls;
        std::vector<LevDesc> lv;
        std::vector<RowScaleDesc> rs;
        for (int j = 0; j < nl; ++j) {
          const int g = lnodes[j0 + j];
          const Node& n = nd[g];
          const int nc = cd[j].ncols, nca = ncand[g];
          const double sc = scale_of(g);
          KDesc a{};
          a.rows = cols + coff[j]; a.nrows = nc; a.colsA = gram + (size_t)j * NGRAM; a.nA = NGRAM;
          a.ncols = NGRAM; a.out = D + toff[j]; a.ld = nc; a.scale = sc;
          kt.push_back(a);
          KDesc b{};
          b.rows = gram + (size_t)j * NGRAM; b.nrows = NGRAM; b.colsA = cols + coff[j]; b.nA = nc;
          b.ncols = nc; b.out = D + boff[j]; b.ld = NGRAM; b.scale = sc;
          kb.push_back(b);
          for (int rep = 0; rep < 2; ++rep) {
            KDesc c{};
            c.rows = cols + coff[j]; c.nrows = nc; c.colsA = l_cand.as<int>() + cand_off[g]; c.nA = nca;
            c.ncols = nca; c.out = D + (rep ? c2off[j] : c1off[j]); c.ld = nc; c.scale = sc;
            kc.push_back(c);
          }
          int cs;
          double ws, wr;
          strat_weights(g, NGRAM, cs, ws, wr);
          rs.push_back(RowScaleDesc{D + boff[j], NGRAM, nc, NGRAM, cs, ws, wr});
          gg.push_back(GemmDesc{D + toff[j], D + boff[j], D + goff[j], nc, nc, NGRAM, nc, NGRAM, nc, 1.0, 0.0});
          rd.push_back(RidgeDesc{D + goff[j], nc});
          ld.push_back(LuDesc{D + goff[j], gpiv + (size_t)j * max_nc, nc, nc});
          ls.push_back(LuSolveDesc{D + goff[j], gpiv + (size_t)j * max_nc, D + c1off[j], nc, nc, nc, nca});
          lv.push_back(LevDesc{D + c2off[j], D + c1off[j], nc, nca, (int)(rows + cand_off[g])});
        }
        arena.clear();
        const size_t ocd = arena.push(cd), osd = arena.push(sd), okt = arena.push(kt), okb = arena.push(kb),
                     okc = arena.push(kc), ors = arena.push(rs);
        char* base = upload_arena();
        gather_cols((const ColsDesc*)(base + ocd), nl, cols, st);
        stream_rows((const StreamDesc*)(base + osd), nl, NGRAM, opt.seed, GRAM_SALT, gram, st);
        kernel_blocks<double>(Xp.as<double>(), xnrm.as<double>(), d, (const KDesc*)(base + okt), nl, max_bt, st);
        kernel_blocks<double>(Xp.as<double>(), xnrm.as<double>(), d, (const KDesc*)(base + okb), nl, max_b, st);
        kernel_blocks<double>(Xp.as<double>(), xnrm.as<double>(), d, (const KDesc*)(base + okc), 2 * nl, max_c, st);
        scale_rows((const RowScaleDesc*)(base + ors), nl, st);  // B <- diag(w) B
        run_gemms(gg);  // its own upload is stream-ordered after the launches above
        arena.clear();
        const size_t ord2 = arena.push(rd), old2 = arena.push(ld), ols2 = arena.push(ls), olv2 = arena.push(lv);
        base = upload_arena();
        add_ridge((const RidgeDesc*)(base + ord2), nl, tol2, st);
        prof().flops[PK_GETRF] += getrf_flops(ld);
        getrf_batched<double>((const LuDesc*)(base + old2), nl, max_nc, status.as<int>(), st);
        prof().flops[PK_GETRS] += getrs_flops(ls);
        getrs_batched<double>((const LuSolveDesc*)(base + ols2), nl, max_nc, max_ncand, st);
        leverage_targets((const LevDesc*)(base + olv2), nl, TL, TT, st);
        IA_CUDA(cudaStreamSynchronize(st));
        raise_status(read_status_and_clear());
        j0 = j1;
      }
      keep_step(S, li, ctot, TT + rows);
      rows += ctot;
    }
    stats.train_rows = rows;
    // training
    if (!mlp_ready) {
      std::vector<float> w0(MLP_NPARAM, 0.0f);
      std::mt19937_64 gen(opt.seed ^ 0x5EEDull);
      std::uniform_real_distribution<double> u1(-std::sqrt(6.0 / MLP_F), std::sqrt(6.0 / MLP_F));
      std::uniform_real_distribution<double> u2(-std::sqrt(6.0 / MLP_W), std::sqrt(6.0 / MLP_W));
      for (int e = MLP_OFF_W1; e < MLP_OFF_B1; ++e) w0[e] = (float)u1(gen);
      for (int e = MLP_OFF_W2; e < MLP_OFF_B2; ++e) w0[e] = (float)u2(gen);
      for (int e = MLP_OFF_W3; e < MLP_OFF_B3; ++e) w0[e] = (float)u2(gen);
      mlp_load(w0.data());
    }
    const int B = std::max(1, std::min<int>(opt.train_batch, (int)std::min<int64_t>(rows, INT_MAX)));
    uint16_t* bx = tr_bx.ensure_n<uint16_t>((size_t)B * 8);
    float* bt = tr_bt.ensure_n<float>(B);
    float* by = tr_y.ensure_n<float>(B);
    uint16_t* H1 = tr_H1.ensure_n<uint16_t>((size_t)B * MLP_W);
    uint16_t* H2 = tr_H2.ensure_n<uint16_t>((size_t)B * MLP_W);
    int* idx = tr_idx.ensure_n<int>(rows);
    std::vector<int> perm_h(rows);
    std::iota(perm_h.begin(), perm_h.end(), 0);
    std::mt19937_64 gen(opt.seed ^ 0x5A4D1Eull);
    stats.train_loss.clear();
    const MlpDev w = mlp_dev();
    for (int ep = 0; ep < epochs; ++ep) {
      std::shuffle(perm_h.begin(), perm_h.end(), gen);
      h2d(idx, perm_h.data(), rows, st);
      IA_CUDA(cudaMemsetAsync(mlp_loss.p, 0, sizeof(float), st));
      int nb = 0;
      for (int64_t r0 = 0; r0 < rows; r0 += B) {
        const int nbt = (int)std::min<int64_t>(B, rows - r0);
        gather_train(TF, TT, idx + r0, nbt, bx, bt, st);
        mlp_forward(bx, nbt, w, by, H1, H2, st);
        mlp_backward(bx, H1, H2, by, bt, nbt, 1.0 / nbt, w, mlp_grad.as<float>(), mlp_loss.as<float>(), st);
        mlp_adam(w, mlp_grad.as<float>(), mlp_m.as<float>(), mlp_v.as<float>(), ++mlp_step, lr, 0.9, 0.999,
                 1e-8, st);
        ++nb;
      }
      float loss = 0.0f;
      d2h(&loss, mlp_loss.as<float>(), 1, st);
      IA_CUDA(cudaStreamSynchronize(st));
      stats.train_loss.push_back(loss / std::max(nb, 1));
    }
    IA_CUDA(cudaStreamSynchronize(st));
  }

  // The operator blocks of the given problems re-evaluated in FP64 (same offsets, same
  // bytes per entry); the apply then uses FP64 products for them.
  void upgrade_operator(const std::vector<int>& probs) {
    slices_ready = false;
    std::vector<KDesc> kl, ku;
    int64_t max_l = 0, max_u = 0;
    const int* sk = skel.as<int>();
    for (int q : probs) {
      pr[q].op64 = true;
      ++stats.fp64_operator_problems;
      ++stats.operator_upgrades;
    }
    for (size_t g = 0; g < nd.size(); ++g) {
      const Node& n = nd[g];
      if (!pr[n.prob].op64 || std::find(probs.begin(), probs.end(), n.prob) == probs.end()) continue;
      if (is_leaf((int)g)) {
        KDesc k{};
        k.row0 = n.off;
        k.nrows = n.size;
        k.col0 = n.off;
        k.ncols = n.size;
        k.out = Kleaf.as<double>() + n.K_off;
        k.ld = n.size;
        k.diag = pr[n.prob].lam;
        k.scale = scale_of((int)g);
        kl.push_back(k);
        max_l = std::max<int64_t>(max_l, (int64_t)n.size * n.size);
      }
      if (!is_root((int)g)) {
        const int sib = sibling((int)g);
        KDesc k{};
        k.row0 = n.off;
        k.nrows = n.size;
        k.colsA = sk + (size_t)sib * s_max;
        k.nA = nd[sib].s;
        k.ncols = nd[sib].s;
        k.out = Ustore.as<double>() + n.U_off;
        k.ld = n.size;
        k.diag = 0.0;
        k.scale = scale_of((int)g);
        if (k.ncols > 0) {
          ku.push_back(k);
          max_u = std::max<int64_t>(max_u, (int64_t)n.size * k.ncols);
        }
      }
    }
    for (std::vector<KDesc>* kv : {&kl, &ku}) {
      for (size_t b = 0; b < kv->size(); b += 65535) {
        const size_t e = std::min(kv->size(), b + 65535);
        std::vector<KDesc> part(kv->begin() + b, kv->begin() + e);
        kblocks64(part, kv == &kl ? max_l : max_u);
      }
    }
  }

  // Operator blocks of the mixed form: FP32 pairs for the problems whose operator is
  // kept in pairs (the descriptors' out pointers address the pair array's bytes), FP64
  // (Gram form) for the others.
  void run_operator_blocks(const std::vector<KDesc>& kd, const std::vector<int>& gids, int64_t max_e) {
    std::vector<KDescT<float2>> kp;
    std::vector<KDesc> k64;
    for (size_t i = 0; i < kd.size(); ++i) {
      if (pr[nd[gids[i]].prob].op64) k64.push_back(kd[i]);
      else kp.push_back(pair_desc(kd[i]));
    }
    arena.clear();
    size_t op = arena.push(kp);
    char* base = upload_arena();
    prof().flops[PK_KBLOCK_PAIR] += kblock_flops(kp, d);
    if (!kp.empty())
      kernel_blocks_pair(Xpair.as<float2>(), d, (const KDescT<float2>*)(base + op), (int)kp.size(), max_e, st);
    kblocks64(k64, max_e);
  }
  // FP64 operator blocks (leaf and U blocks: consecutive rows): with op_slices and the
  // Gaussian, dot products on the tensor cores from the points' digits (built once per
  // factorization), else the FP64 Gram form.
  bool xdig_ready = false;
  DevBuf ozXD, ozXE;
  void kblocks64(const std::vector<KDesc>& kd, int64_t max_e) {
    if (kd.empty()) return;
    bool sliced_ok = prec == PREC_MIXED && opt.op_slices && kspec.poly == 0 && oz_dpad(d) > 0;
    for (const KDesc& k : kd) sliced_ok = sliced_ok && k.rows == nullptr;
    arena.clear();
    if (!sliced_ok) {
      const size_t ok = arena.push(kd);
      char* base = upload_arena();
      prof().flops[PK_KBLOCK] += kblock_flops(kd, d);
      kernel_blocks<double>(Xp.as<double>(), xnrm.as<double>(), d, (const KDesc*)(base + ok), (int)kd.size(), max_e,
                            st);
      return;
    }
    if (!xdig_ready) {
      uint16_t* XD = ozXD.ensure_n<uint16_t>((size_t)Ntot * OZ_S * oz_dpad(d));
      int* XE = ozXE.ensure_n<int>((size_t)Ntot);
      oz_points(Xp.as<double>(), Ntot, d, XD, XE, st);
      xdig_ready = true;
    }
    std::vector<OzKDesc> od;
    int tiles = 0;
    for (const KDesc& k : kd) {
      if (k.nrows <= 0 || k.ncols <= 0) continue;
      od.push_back(OzKDesc{k.colsA, k.colsB, k.out, k.row0, k.nrows, k.col0, k.nA, k.ncols, k.ld, k.diag, k.scale,
                           tiles, nullptr});
      tiles += (int)ceil_div((size_t)k.nrows, OZ_TM);
    }
    const size_t oo = arena.push(od);
    char* base = upload_arena();
    prof().flops[PK_KBLOCK_OZ] += kblock_flops(kd, d);
    oz_kblocks(ozXD.as<uint16_t>(), ozXE.as<int>(), xnrm.as<double>(), d, (const OzKDesc*)(base + oo), (int)od.size(),
               tiles, status.as<int>(), st);
  }
  // FP32 and FP64 solve copies of operator blocks; list [t] holds the ranges whose
  // operator is in FP64 (t = 1) or in FP32 pairs (t = 0).
  void conv_operator(const double* src, float* d32, double* d64, std::vector<ConvSeg> (&s32)[2],
                     std::vector<ConvSeg> (&s64)[2]) {
    const float2* sp = reinterpret_cast<const float2*>(src);
    conv_segs<float2, float>(sp, d32, s32[0]);
    conv_segs<double, float>(src, d32, s32[1]);
    conv_segs<float2, double>(sp, d64, s64[0]);
    conv_segs<double, double>(src, d64, s64[1]);
  }

  // a4 + a6: leaf LU of lambda I + K_aa, in each problem's precision.  The mixed form
  // keeps the FP64 blocks for the operator (Kleaf) and factors a copy: rounded to FP32,
  // or in FP64 for the problems it factors in FP64.
  void leaf_lu() {
    const bool mixed = prec == PREC_MIXED;
    // dinv areas of every FP32 LU: the leaf blocks and the reduced systems (ranks known)
    int64_t di = 0;
    for (size_t g = 0; g < nd.size(); ++g) {
      if (f64((int)g)) continue;
      const bool leaf = is_leaf((int)g);
      nd[g].DI_off = di;
      di += lu_dinv_size(leaf ? nd[g].size : n2((int)g));
    }
    if (di > 0) DInv32.ensure_n<float>(di);
    int64_t tot = 0, tot_t[2] = {0, 0};
    for (int g : by_height[0]) {
      Node& n = nd[g];
      const int64_t e = (int64_t)n.size * n.size;
      n.K_off = tot;
      tot += e;
      n.LU_off = tot_t[f64(g)];
      tot_t[f64(g)] += e;
    }
    double* blocks = mixed ? Kleaf.ensure_n<double>(tot) : LU.ensure_n<double>(tot);
    int* lp = LUpiv.ensure_n<int>((size_t)nleaves * m_max);
    std::vector<KDesc> kd;
    for (int g : by_height[0]) {
      const Node& n = nd[g];
      KDesc k{};
      k.row0 = n.off;
      k.nrows = n.size;
      k.col0 = n.off;
      k.ncols = n.size;
      k.out = blocks + n.K_off;
      k.ld = n.size;
      k.diag = pr[n.prob].lam;
      k.scale = scale_of(g);
      kd.push_back(k);
    }
    const int nl = (int)kd.size();
    arena.clear();
    if (mixed) {  // the operator keeps the blocks as FP32 pairs (in the bytes of Kleaf), or in FP64
      run_operator_blocks(kd, by_height[0], (int64_t)m_max * m_max);
    } else {
      size_t ok = arena.push(kd);
      char* base = upload_arena();
      prof().flops[PK_KBLOCK] += kblock_flops(kd, d);
      kernel_blocks<double>(Xp.as<double>(), xnrm.as<double>(), d, (const KDesc*)(base + ok), nl,
                            (int64_t)m_max * m_max, st);
    }
    float* lu32 = tot_t[0] ? LU32.ensure_n<float>(tot_t[0]) : nullptr;
    double* lu64 = blocks;
    if (mixed) {
      // one range per problem: its leaves are consecutive in both layouts
      std::vector<ConvSeg> s32[2], s64[2];  // [operator in FP64]
      for (const Prob& P : pr) {
        const int first = P.nbase + (1 << P.L), nlv = 1 << P.L;
        const Node& a = nd[first];
        const Node& b = nd[first + nlv - 1];
        const int64_t len = b.K_off + (int64_t)b.size * b.size - a.K_off;
        (P.f64 ? s64 : s32)[P.op64].push_back(ConvSeg{a.K_off, a.LU_off, len});
      }
      if (tot_t[1]) lu64 = LU.ensure_n<double>(tot_t[1]);
      conv_operator(blocks, lu32, lu64, s32, s64);
      stats.bytes_operator += tot * 8;
    }
    stats.bytes_LU = tot_t[0] * 4 + tot_t[1] * 8;
    std::vector<LuDescT<float>> l32;
    std::vector<LuDesc> l64;
    for (int g : by_height[0]) {
      const Node& n = nd[g];
      int* piv = lp + (int64_t)n.leaf * m_max;
      if (f64(g)) l64.push_back(LuDesc{lu64 + n.LU_off, piv, n.size, n.size});
      else l32.push_back(LuDescT<float>{lu32 + n.LU_off, piv, n.size, n.size, dinvP<float>(g)});
    }
    arena.clear();
    size_t o32 = arena.push(l32), o64 = arena.push(l64);
    char* base = upload_arena();
    if (!l32.empty()) {
      prof().flops[PK_GETRF32] += getrf_flops(l32);
      getrf_batched<float>((const LuDescT<float>*)(base + o32), (int)l32.size(), m_max, status.as<int>(), st,
                           true);
    }
    if (!l64.empty()) {
      prof().flops[PK_GETRF] += getrf_flops(l64);
      getrf_batched<double>((const LuDesc*)(base + o64), (int)l64.size(), m_max, status.as<int>(), st);
    }
    // the FP32 LUs' inverses (lu_inverse), after the launches above that read the
    // previous descriptor upload
    inv_leaf = mixed && opt.lu_inverse >= 1;
    inv_z = mixed && opt.lu_inverse == 2;
    inv_zh = opt.lu_inverse_zh;
    if (inv_leaf && !l32.empty()) {
      float* li = LUi32.ensure_n<float>(tot_t[0]);
      std::vector<LuSolveDescT<float>> ri;
      for (int g : by_height[0]) {
        if (f64(g)) continue;
        const Node& n = nd[g];
        ri.push_back(LuSolveDescT<float>{lu32 + n.LU_off, lp + (int64_t)n.leaf * m_max, li + n.LU_off, n.size,
                                         n.size, n.size, n.size, dinvP<float>(g)});
      }
      arena.clear();
      size_t oi = arena.push(ri);
      char* bi = upload_arena();
      prof().flops[PK_GETRI32] += getri_flops(ri);
      getri_batched((const LuSolveDescT<float>*)(bi + oi), (int)ri.size(), m_max, st);
      stats.bytes_LU += tot_t[0] * 4;
    }
  }

  // a7 + a8: W and Z, heights 1 .. Hmax, each problem's factorization in its own
  // precision.  The U blocks K_{c s~} are evaluated in FP64 for every child c of the
  // height; the mixed form keeps them (Ustore) for the operator and solves a copy.
  void factor_levels() {
    if (Hmax == 0) return;
    const bool mixed = prec == PREC_MIXED;
    int64_t wsz[2] = {0, 0}, zsz[2] = {0, 0}, csz[2] = {0, 0}, usz = 0, zp = 0;
    for (int hh = 0; hh < Hmax; ++hh)
      for (int g : by_height[hh]) {
        if (is_root(g)) continue;
        Node& n = nd[g];
        const int64_t e = (int64_t)n.size * nd[sibling(g)].s;
        n.U_off = usz;
        usz += e;
        n.W_off = wsz[f64(g)];
        wsz[f64(g)] += e;
      }
    int64_t zinv = 0;  // FP32 Zs of heights <= inv_zh, inverted: a prefix of the FP32 Z pool
    for (int hh = 1; hh <= Hmax; ++hh) {
      for (int g : by_height[hh]) {
        Node& n = nd[g];
        const int t = f64(g);
        const int sa = nd[left(g)].s, sb = nd[right(g)].s;
        n.Z_off = zsz[t];
        zsz[t] += (int64_t)(sa + sb) * (sa + sb);
        n.Zpiv_off = zp;
        zp += sa + sb;
        n.CL_off = csz[t];
        csz[t] += (int64_t)sa * sb;
        n.CR_off = csz[t];
        csz[t] += (int64_t)sb * sa;
      }
      if (inv_z && hh <= inv_zh) zinv = zsz[0];
    }
    const double bytes = (double)(wsz[0] + zsz[0] + zinv + csz[0]) * 4 +
                         (double)(wsz[1] + zsz[1] + csz[1]) * 8 + (mixed ? (double)usz * 8 : 0.0);
    if (opt.mem_cap_gb > 0 && bytes > opt.mem_cap_gb * 1e9)
      throw Error(IASKIT_ERR_NOMEM, "factorization exceeds mem_cap_gb");
    if (wsz[0]) Wb32.ensure_n<float>(wsz[0]);
    if (zsz[0]) Zb32.ensure_n<float>(zsz[0]);
    if (zinv) Zi32.ensure_n<float>(zinv);
    if (csz[0]) Cb32.ensure_n<float>(csz[0]);
    if (wsz[1]) Wb.ensure_n<double>(wsz[1]);
    if (zsz[1]) Zb.ensure_n<double>(zsz[1]);
    if (csz[1]) Cb.ensure_n<double>(csz[1]);
    Zpiv.ensure_n<int>(std::max<int64_t>(zp, 1));
    // the plain form evaluates U straight into W (same layout: every problem is FP64)
    double* U64 = mixed ? Ustore.ensure_n<double>(std::max<int64_t>(usz, 1))
                        : Wb.ensure_n<double>(std::max<int64_t>(wsz[1], 1));
    stats.bytes_W = wsz[0] * 4 + wsz[1] * 8;
    stats.bytes_LU += zinv * 4;
    if (mixed) stats.bytes_operator += usz * 8;
    int* sk = skel.as<int>();
    for (int hh = 1; hh <= Hmax; ++hh) {
      const std::vector<int>& nodes = by_height[hh];
      std::vector<KDesc> kd;
      int64_t max_e = 0;
      std::vector<ConvSeg> s32[2], s64[2];  // [operator in FP64]
      std::vector<int> kg;                  // child of each descriptor
      for (int g : nodes)
        for (int c : {left(g), right(g)}) {
          const Node& n = nd[c];
          const int sib = sibling(c);
          kg.push_back(c);
          KDesc k{};
          k.row0 = n.off;
          k.nrows = n.size;
          k.colsA = sk + (size_t)sib * s_max;
          k.nA = nd[sib].s;
          k.ncols = nd[sib].s;
          k.out = U64 + n.U_off;
          k.ld = n.size;
          k.diag = 0.0;
          k.scale = scale_of(c);
          kd.push_back(k);
          const int64_t e = (int64_t)n.size * k.ncols;
          max_e = std::max<int64_t>(max_e, e);
          // consecutive children of one precision extend the previous range
          std::vector<ConvSeg>& sv = (f64(c) ? s64 : s32)[pr[n.prob].op64];
          if (!sv.empty() && sv.back().src + sv.back().len == n.U_off &&
              sv.back().dst + sv.back().len == n.W_off)
            sv.back().len += e;
          else
            sv.push_back(ConvSeg{n.U_off, n.W_off, e});
        }
      arena.clear();
      if (mixed) {  // the operator keeps the U blocks as FP32 pairs (in the bytes of Ustore), or in FP64
        run_operator_blocks(kd, kg, max_e);
        conv_operator(U64, Wb32.as<float>(), Wb.as<double>(), s32, s64);
      } else {
        size_t ok = arena.push(kd);
        char* base = upload_arena();
        prof().flops[PK_KBLOCK] += kblock_flops(kd, d);
        kernel_blocks<double>(Xp.as<double>(), xnrm.as<double>(), d, (const KDesc*)(base + ok), (int)kd.size(),
                              max_e, st);
      }
      level_step<float>(nodes);
      level_step<double>(nodes);
    }
  }

  // W = Solve(child, U) for the children of the nodes of one height whose problems are
  // stored in precision T (C blocks come back as P_c W_c), then the reduced systems
  // Z'' = [[I, C_l], [C_r, I]] and their LU.
  template <typename T>
  void level_step(const std::vector<int>& all_nodes) {
    std::vector<int> nodes;
    for (int g : all_nodes)
      if (f64(g) == std::is_same<T, double>::value) nodes.push_back(g);
    if (nodes.empty()) return;
    T* W = wP<T>();
    T* C = cP<T>();
    std::vector<RootBlock<T>> rb;
    for (int g : nodes)
      for (int c : {left(g), right(g)}) {
        const Node& n = nd[c];
        const int sib = sibling(c);
        // left child: C_l = P_l W_{l r~} (s_l x s_r); right child: C_r = P_r W_{r l~}
        T* tout = C + ((n.uid & 1) == 0 ? nd[g].CL_off : nd[g].CR_off);
        rb.push_back(RootBlock<T>{c, W + n.W_off, n.size, nd[sib].s, tout, n.s});
      }
    forest_solve<T>(rb);
    std::vector<ZDescT<T>> zd;
    std::vector<LuDescT<T>> ld;
    int64_t max_z = 0;
    int max_n = 0;
    for (int g : nodes) {
      const int sa = nd[left(g)].s, sb = nd[right(g)].s;
      zd.push_back(ZDescT<T>{C + nd[g].CL_off, C + nd[g].CR_off, zP<T>() + nd[g].Z_off, sa, sb});
      ld.push_back(LuDescT<T>{zP<T>() + nd[g].Z_off, Zpiv.as<int>() + nd[g].Zpiv_off, sa + sb, sa + sb,
                              dinvP<T>(g)});
      max_z = std::max<int64_t>(max_z, (int64_t)(sa + sb) * (sa + sb));
      max_n = std::max(max_n, sa + sb);
    }
    arena.clear();
    size_t oz = arena.push(zd), ol = arena.push(ld);
    char* base = upload_arena();
    form_Z<T>((const ZDescT<T>*)(base + oz), (int)zd.size(), max_z, st);
    prof().flops[pk_of<T>(PK_GETRF)] += getrf_flops(ld);
    getrf_batched<T>((const LuDescT<T>*)(base + ol), (int)ld.size(), max_n, status.as<int>(), st,
                     std::is_same<T, float>::value);
    if (std::is_same<T, float>::value && inv_z && height(nodes[0]) <= inv_zh) {
      std::vector<LuSolveDescT<float>> ri;
      for (int g : nodes) {
        const int n2g = n2(g);
        ri.push_back(LuSolveDescT<float>{Zb32.as<float>() + nd[g].Z_off, Zpiv.as<int>() + nd[g].Zpiv_off,
                                         Zi32.as<float>() + nd[g].Z_off, n2g, n2g, n2g, n2g, dinvP<float>(g)});
      }
      arena.clear();
      size_t oi = arena.push(ri);
      char* bi = upload_arena();
      prof().flops[PK_GETRI32] += getri_flops(ri);
      getri_batched((const LuSolveDescT<float>*)(bi + oi), (int)ri.size(), max_n, st);
    }
  }

  // ------------------------------------------------------------------ solve
  // rhs: all problems' N_p x nrhs blocks, one after the other (ORIGINAL order), device
  void solve_device(double* rhs, int nrhs) {
    if (!factored) throw Error(IASKIT_ERR_NOT_FACTORED, "no factorization");
    if (nrhs < 1 || (int64_t)Ntot * nrhs > ((int64_t)1 << 31)) throw Error(IASKIT_ERR_ARG, "bad nrhs");
    const double t0 = now_ms();
    check_finite(rhs, (int64_t)Ntot * nrhs, status.as<int>(), st);
    raise_status(read_status_and_clear());
    stats.refine_hist.clear();
    stats.refine_sweeps = 0;
    stats.refine_stagnated = 0;
    stats.stagnated.clear();
    const int sweeps = opt.refine > 0 ? opt.refine : (prec == PREC_MIXED ? 200 : 0);
    if (sweeps <= 0) {
      plain_solve(rhs, nrhs, rhs);
    } else {
      const size_t n = (size_t)Ntot * nrhs;
      double* rhs0 = nullptr;
      if (prec == PREC_MIXED) {  // kept for a second refinement after an operator upgrade
        rhs0 = rhs_keep.ensure_n<double>(n);
        IA_CUDA(cudaMemcpyAsync(rhs0, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      }
      stag_prob.clear();
      refine_solve(rhs, nrhs, sweeps);
      // problems whose columns stopped at the rounding floor of the FP32-pair operator
      // get their operator blocks in FP64, and the solve is refined again
      std::vector<int> up;
      for (size_t q = 0; q < stag_prob.size(); ++q)
        if (stag_prob[q] && !pr[q].op64) up.push_back((int)q);
      if (rhs0 && !up.empty()) {  // continue from the current solution
        upgrade_operator(up);
        const int it0 = stats.refine_iters;
        refine_solve(rhs, nrhs, sweeps, rhs0);
        stats.refine_iters += it0;
      }
    }
    IA_CUDA(cudaStreamSynchronize(st));
    prof().resolve();
    stats.t_solve = now_ms() - t0;
  }

  // Exact kernel sums K(T, X_q) w at M test points for the selected problem q (Sec. III,
  // kernel regression): T M x d row-major, w N_q x nrhs column-major in q's original
  // order, out M x nrhs column-major; all device pointers.
  void predict_device(const double* T, int64_t M, const double* w, int nrhs, double* out, int q) {
    if (!skeletonized && !factored) throw Error(IASKIT_ERR_NOT_FACTORED, "no factorization");
    if (M < 0 || M > INT_MAX / 2) throw Error(IASKIT_ERR_ARG, "bad number of test points");
    if (nrhs < 1 || nrhs > 4096) throw Error(IASKIT_ERR_ARG, "bad nrhs");
    if (M == 0) return;
    const Prob& P = pr[q];
    check_finite(T, M * d, status.as<int>(), st);
    check_finite(w, (int64_t)P.N * nrhs, status.as<int>(), st);
    raise_status(read_status_and_clear());
    double* part = pred_part.ensure_n<double>(predict_scratch_doubles((int)M, P.N, nrhs));
    use_kernel(kspec);
    kernel_predict(T, (int)M, Xp.as<double>(), xnrm.as<double>(), perm.as<int>(), P.pbase, P.N, d, P.scale, w, P.N,
                   nrhs, part, out, (int)M, st);
    IA_CUDA(cudaStreamSynchronize(st));
    prof().resolve();
  }

  // out <- (lambda I + K~)^{-1} in with the stored factorization; in and out may alias.
  // Problems factored in FP32 are solved on an FP32 copy of their blocks.
  void plain_solve(const double* in, int nrhs, double* out) {
    const size_t n = (size_t)Ntot * nrhs;
    const BlockDesc* blocks = upload_blocks(nrhs, false);
    double* V = vbuf.ensure_n<double>(n);
    gather(in, V, nrhs, blocks, false);
    std::vector<RootBlock<float>> r32;
    std::vector<RootBlock<double>> r64;
    std::vector<ConvSeg> back;
    float* V32 = any_prec(false) ? vbuf32.ensure_n<float>(n) : nullptr;
    for (const Prob& P : pr) {
      const int64_t o = (int64_t)P.pbase * nrhs;
      if (P.f64) {
        r64.push_back(RootBlock<double>{P.nbase + 1, V + o, P.N, nrhs, nullptr, 0});
      } else {
        r32.push_back(RootBlock<float>{P.nbase + 1, V32 + o, P.N, nrhs, nullptr, 0});
        const int64_t len = (int64_t)P.N * nrhs;
        if (!back.empty() && back.back().src + back.back().len == o) back.back().len += len;
        else back.push_back(ConvSeg{o, o, len});
      }
    }
    if (!r32.empty()) {
      conv_segs<double, float>(V, V32, back);
      forest_solve<float>(r32);
      conv_segs<float, double>(V32, V, back);
    }
    if (!r64.empty()) forest_solve<double>(r64);
    gather(V, out, nrhs, blocks, true);
  }

  // Iterative refinement with flexible GMRES (FGMRES-IR; Carson & Higham's GMRES-IR with
  // the preconditioned basis kept, Saad's flexible variant): residuals r = u - A w with the
  // FP64 operator; each correction solves A z = r by restarted GMRES in FP64, right-
  // preconditioned by the stored factorization M^-1.  The vectors Z_j = M^-1 v_j are kept
  // and the update is w += Z y, so it matches the Arnoldi relation even though M^-1 runs
  // partly in FP32 (no second, differently rounded application of M^-1).
  // Every (problem, column) pair is its own segment; all open segments advance together,
  // so one preconditioner and one operator application serve all of them per iteration.
  // In the mixed form with FP64 operator blocks (option inner_pair), the operator
  // applies inside a GMRES cycle form their FP64 products on FP32 pairs (about 2^-44
  // relative, on the FP32 pipes) and each cycle aims at a reduction of 1e-7 of its
  // starting residual; every cycle's residual is recomputed with FP64 products, so the
  // outer iteration converges to the FP64 operator's solution (GMRES-IR with an inner
  // operator of lower precision than the residual, after Carson & Higham).
  // A segment closes when its relative residual is <= refine_tol, or when a cycle whose
  // own GMRES estimate reached its target lowered the recomputed residual by less than
  // half, or (FP64 inner products) left it a hundred times above that estimate: then the
  // rounding floor of the FP64 residual itself, about eps ||A|| ||w|| / ||u||, lies above
  // the target and further cycles cannot help.
  // max_iters bounds the total number of GMRES iterations.
  // u_in: null - w holds the right-hand side and receives the solution, starting from
  // the plain solve; else u_in is the right-hand side and w an initial iterate.
  void refine_solve(double* w, int nrhs, int max_iters, const double* u_in = nullptr) {
    const size_t n = (size_t)Ntot * nrhs;
    const int S = (int)pr.size() * nrhs;
    // restart length: at most 30, and (2m + 1) n doubles of bases within about 16 GB
    const int m = (int)std::max<int64_t>(1, std::min<int64_t>(30, (int64_t)(1e9 / (double)n) - 1));
    std::vector<GSeg> hseg(S);
    for (size_t q = 0; q < pr.size(); ++q)
      for (int c = 0; c < nrhs; ++c)
        hseg[q * nrhs + c] = GSeg{(int64_t)pr[q].pbase * nrhs + (int64_t)c * pr[q].N, pr[q].N};
    GSeg* segs = gseg_dev.ensure_n<GSeg>(S);
    h2d(segs, hseg.data(), S, st);
    max_seg_len = 1;
    for (const GSeg& g : hseg) max_seg_len = std::max(max_seg_len, g.len);
    double* u = rbuf.ensure_n<double>(2 * n);  // copy of the right-hand side, residual
    double* r = u + n;
    double* V = kryl.ensure_n<double>((size_t)(m + 1) * n);
    double* Zb_ = kzb.ensure_n<double>((size_t)m * n);
    double* coef = coefbuf.ensure_n<double>((size_t)(m + 1) * S);
    IA_CUDA(cudaMemcpyAsync(u, u_in ? u_in : w, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    std::vector<double> un, rn, hn, prev(S, 0.0), est_end(S, HUGE_VAL);
    std::vector<int> state(S, 0);  // 0 open, 1 converged, 2 at the rounding floor
    column_norms(u, nrhs, un);
    if (!u_in) plain_solve(u, nrhs, w);  // x0 = M^-1 u
    int& iters = stats.refine_iters;
    iters = 0;
    bool first = true;
    bool low = false;  // inner applies on pairs: some problem keeps FP64 operator blocks
    if (prec == PREC_MIXED && opt.inner_pair)
      for (const Prob& P : pr) low = low || P.op64;
    std::vector<double> cyc_tgt(S, 0.0);  // the last cycle's target per segment
    struct LowScope {
      bool& f;
      explicit LowScope(bool& flag) : f(flag) {}
      ~LowScope() { f = false; }
    } low_scope(apply_low);
    while (true) {
      apply_device(w, r, nrhs);  // r = u - A w
      axpby(u, r, n);
      column_norms(r, nrhs, rn);
      double worst = 0;
      bool open = false;
      for (int q = 0; q < S; ++q) {
        const double rel = un[q] > 0 ? rn[q] / un[q] : rn[q];
        if (!std::isfinite(rel)) throw Error(IASKIT_ERR_NOT_CONVERGED, "refinement produced a non-finite residual");
        worst = std::max(worst, rel);
        if (state[q] == 0) {
          // at the floor: the cycle's own GMRES estimate met 0.1 refine_tol, and the
          // recomputed residual either fell by less than half or lies a hundred times
          // above that estimate (FGMRES's estimate is the true residual up to rounding)
          if (rel <= opt.refine_tol) state[q] = 1;
          else if (!first && est_end[q] <= cyc_tgt[q] &&
                   (rn[q] > 0.5 * prev[q] || (!low && rn[q] > 100.0 * est_end[q])))
            state[q] = 2;
        }
        prev[q] = rn[q];
        open = open || state[q] == 0;
      }
      stats.refine_hist.push_back(worst);
      if (!open) {
        stats.refine_stagnated = (int)std::count(state.begin(), state.end(), 2);
        stag_prob.assign(pr.size(), 0);
        for (int q = 0; q < S; ++q)
          if (state[q] == 2) stag_prob[q / nrhs] = 1;
        // every stopped column beside the rounding floor of its residual: 2^-53 ||A|| ||w|| / ||u||
        // with ||A|| ~ lambda + the largest sampled kernel row sum = lambda cond_est
        stats.stagnated.clear();
        if (stats.refine_stagnated > 0) {
          std::vector<double> wn;
          column_norms(w, nrhs, wn);
          for (int q = 0; q < S; ++q)
            if (state[q] == 2) {
              const Prob& P = pr[q / nrhs];
              const double anorm = P.lam > 0 ? P.lam * P.cond_est : HUGE_VAL;
              const double rel = un[q] > 0 ? rn[q] / un[q] : rn[q];
              stats.stagnated.push_back(
                  StagCol{q / nrhs, q % nrhs, rel, 0x1p-53 * anorm * wn[q] / std::max(un[q], 1e-300), P.op64});
            }
        }
        return;
      }
      if (iters >= max_iters) throw Error(IASKIT_ERR_NOT_CONVERGED, "refinement did not converge");
      // inner GMRES(m) on A z = r, right-preconditioned, open segments only
      std::vector<double> H((size_t)S * (m + 1) * m, 0.0), cs((size_t)S * m), sn((size_t)S * m),
          g((size_t)S * (m + 1), 0.0);
      auto Hs = [&](int q, int i, int j) -> double& { return H[((size_t)q * (m + 1) + i) * m + j]; };
      std::vector<double> inv(S);
      for (int q = 0; q < S; ++q) {
        const bool live = state[q] == 0 && rn[q] > 0;
        g[(size_t)q * (m + 1)] = live ? rn[q] : 0.0;
        inv[q] = live ? 1.0 / rn[q] : 0.0;  // closed segments get a zero basis and no update
        cyc_tgt[q] = std::max(0.1 * opt.refine_tol * std::max(un[q], 1e-300), low ? 1e-7 * rn[q] : 0.0);
      }
      h2d(coef, inv.data(), S, st);
      seg_scale(V, r, coef, segs, S);  // V_0 = r / beta
      int k = 0;
      for (int j = 0; j < m && iters < max_iters; ++j) {
        double* vj = V + (size_t)j * n;
        double* vn = V + (size_t)(j + 1) * n;
        double* zj = Zb_ + (size_t)j * n;
        plain_solve(vj, nrhs, zj);      // Z_j = M^-1 v_j
        apply_low = low;
        apply_device(zj, vn, nrhs);     // v_{j+1} = A Z_j
        apply_low = false;
        std::vector<double> h1, h2;
        seg_dots(V, n, j + 1, vn, segs, S, coef, h1);     // classical Gram-Schmidt,
        seg_axpy(vn, V, n, j + 1, coef, -1.0, segs, S);    // twice
        seg_dots(V, n, j + 1, vn, segs, S, coef, h2);
        seg_axpy(vn, V, n, j + 1, coef, -1.0, segs, S);
        column_norms(vn, nrhs, hn);
        for (int q = 0; q < S; ++q) inv[q] = hn[q] > 0 ? 1.0 / hn[q] : 0.0;
        h2d(coef, inv.data(), S, st);
        seg_scale(vn, vn, coef, segs, S);
        ++iters;
        k = j + 1;
        bool met = true;
        for (int q = 0; q < S; ++q) {
          for (int i = 0; i <= j; ++i) Hs(q, i, j) = h1[(size_t)i * S + q] + h2[(size_t)i * S + q];
          Hs(q, j + 1, j) = hn[q];
          for (int i = 0; i < j; ++i) {  // earlier Givens rotations
            const double a = Hs(q, i, j), b = Hs(q, i + 1, j);
            Hs(q, i, j) = cs[(size_t)q * m + i] * a + sn[(size_t)q * m + i] * b;
            Hs(q, i + 1, j) = -sn[(size_t)q * m + i] * a + cs[(size_t)q * m + i] * b;
          }
          const double a = Hs(q, j, j), b = Hs(q, j + 1, j);
          const double rr = std::hypot(a, b);
          const double c = rr > 0 ? a / rr : 1.0, sgn = rr > 0 ? b / rr : 0.0;
          cs[(size_t)q * m + j] = c;
          sn[(size_t)q * m + j] = sgn;
          Hs(q, j, j) = rr;
          Hs(q, j + 1, j) = 0.0;
          double& gj = g[(size_t)q * (m + 1) + j];
          g[(size_t)q * (m + 1) + j + 1] = -sgn * gj;
          gj = c * gj;
          const double est = std::fabs(g[(size_t)q * (m + 1) + j + 1]);
          est_end[q] = est;
          met = met && (state[q] != 0 || est <= cyc_tgt[q]);
        }
        if (met) break;
      }
      // y = R^-1 g per segment, w += Z y
      std::vector<double> y((size_t)k * S, 0.0);
      for (int q = 0; q < S; ++q)
        for (int i = k - 1; i >= 0; --i) {
          double acc = g[(size_t)q * (m + 1) + i];
          for (int l = i + 1; l < k; ++l) acc -= Hs(q, i, l) * y[(size_t)l * S + q];
          const double dd = Hs(q, i, i);
          y[(size_t)i * S + q] = dd != 0.0 ? acc / dd : 0.0;
        }
      h2d(coef, y.data(), y.size(), st);
      seg_axpy(w, Zb_, n, k, coef, 1.0, segs, S);
      stats.refine_sweeps += 1;
      first = false;
    }
  }

  // out[i*S + q] = <V_i, x> over segment q, i < k (segments of at most max_seg_len)
  int max_seg_len = 1;
  void seg_dots(const double* V, size_t vstride, int k, const double* x, const GSeg* segs, int S,
                double* dev_out, std::vector<double>& out) {
    {
      ProfScope _ps(PK_MISC, st);
      const int nch = std::max(1, (int)ceil_div((size_t)max_seg_len, RED_CHUNK));
      double* part = redpart.ensure_n<double>((size_t)k * S * nch);
      seg_dots_part_kernel<<<dim3(nch, k, S), 256, 0, st>>>(V, vstride, x, segs, S, nch, part);
      IA_LAUNCH_CHECK();
      chunk_sum_kernel<<<ceil_div((size_t)k * S, 256), 256, 0, st>>>(part, k * S, nch, dev_out);
      IA_LAUNCH_CHECK();
    }
    out.resize((size_t)k * S);
    d2h(out.data(), dev_out, out.size(), st);  // dev_out keeps them for the following update
    IA_CUDA(cudaStreamSynchronize(st));
  }
  // x_seg += sign * sum_{i<k} coef[i*S + q] V_i,seg
  void seg_axpy(double* x, const double* V, size_t vstride, int k, const double* coef, double sign,
                const GSeg* segs, int S) {
    ProfScope _ps(PK_MISC, st);
    seg_axpy_kernel<<<dim3(256, S), 256, 0, st>>>(x, V, vstride, k, coef, sign, segs, S);
    IA_LAUNCH_CHECK();
  }
  // out_seg = coef[q] * x_seg
  void seg_scale(double* out, const double* x, const double* coef, const GSeg* segs, int S) {
    ProfScope _ps(PK_MISC, st);
    seg_scale_kernel<<<dim3(256, S), 256, 0, st>>>(out, x, coef, segs);
    IA_LAUNCH_CHECK();
  }

  void column_norms(const double* x, int nrhs, std::vector<double>& out) {
    const BlockDesc* blocks = upload_blocks(nrhs, false);
    double* dn = normbuf.ensure_n<double>((size_t)nrhs * pr.size());
    {
      ProfScope _ps(PK_MISC, st);
      int max_n = 1;
      for (const Prob& P : pr) max_n = std::max(max_n, P.N);
      const int nch = (int)ceil_div((size_t)max_n, RED_CHUNK);
      double* part = redpart.ensure_n<double>((size_t)nrhs * pr.size() * nch);
      colnorm_part_kernel<<<dim3(nch, nrhs, (unsigned)pr.size()), 256, 0, st>>>(x, blocks, nrhs, nch, part);
      IA_LAUNCH_CHECK();
      const int tot = nrhs * (int)pr.size();
      colnorm_reduce_kernel<<<ceil_div((size_t)tot, 256), 256, 0, st>>>(part, tot, nch, dn);
      IA_LAUNCH_CHECK();
    }
    out.resize((size_t)nrhs * pr.size());
    d2h(out.data(), dn, out.size(), st);
    IA_CUDA(cudaStreamSynchronize(st));
  }
  void axpby(const double* u, double* r, size_t n) {
    ProfScope _ps(PK_MISC, st);
    axpby_kernel<<<grid_cap((int64_t)n, 8192), 256, 0, st>>>(u, r, n);
    IA_LAUNCH_CHECK();
  }

  // ------------------------------------------------------- hierarchical apply
  // u = (lambda I + K~) w (all problems' blocks, ORIGINAL order, device).  Skeletonize
  // (w~ = P w up the tree) then Evaluate (u_c += K_{c s~} w~_s for the sibling s of
  // every non-root node c, and the leaf blocks).  The plain form recomputes the
  // kernel entries in FP64; the mixed form multiplies the FP64 blocks it stored.
  // ---------------------------------------------------------- near field
  // Per node: the targets whose Evaluate list holds the node and whose kNN lists hold
  // one of its points (global positions), built once per tree and kNN lists.
  struct NearList {
    int g, level, first, n;
  };
  bool near_ready = false;
  std::vector<NearList> near_lists;
  DevBuf near_mask, near_tgt, near_part, near_io;
  void near_build() {
    std::vector<NearProb> np(pr.size());
    for (size_t q = 0; q < pr.size(); ++q) np[q] = NearProb{pr[q].pbase, pr[q].N, pr[q].L, pr[q].nbase, pr[q].scale};
    arena.clear();
    const size_t op = arena.push(np);
    char* base = upload_arena();
    unsigned* dm = near_mask.ensure_n<unsigned>(Ntot);
    near_masks(knn_pos.as<int>(), kappa, pid.as<int>(), (const NearProb*)(base + op), Ntot, dm, st);
    std::vector<unsigned> hm(Ntot);
    d2h(hm.data(), dm, Ntot, st);
    IA_CUDA(cudaStreamSynchronize(st));
    near_lists.clear();
    std::vector<int> tgt;
    for (int hh = 0; hh < Hmax; ++hh)
      for (int g : by_height[hh]) {
        if (is_root(g)) continue;
        const Node& sb = nd[sibling(g)];
        const int l = nd[g].level;
        NearList L{g, l, (int)tgt.size(), 0};
        for (int p = sb.off; p < sb.off + sb.size; ++p)
          if (hm[p] >> l & 1u) tgt.push_back(p);
        L.n = (int)tgt.size() - L.first;
        if (L.n > 0) near_lists.push_back(L);
      }
    stats.near_values = 0.0;  // kernel values of one near-field apply per right-hand side
    for (const NearList& L : near_lists) stats.near_values += (double)L.n * (nd[L.g].size + nd[L.g].s);
    int* dt = near_tgt.ensure_n<int>(std::max<size_t>(tgt.size(), 1));
    h2d(dt, tgt.data(), tgt.size(), st);
    IA_CUDA(cudaStreamSynchronize(st));
    near_ready = true;
  }
  void near_field_apply(const double* Wp, const double* WT, const std::vector<int64_t>& woff, double* Up,
                        int nrhs) {
    if (!near_ready) near_build();
    const int TR = near_tile_rows(), RMAX = near_max_rhs();
    constexpr int CHUNK = 4096;  // columns per item of a node's points
    for (int c0 = 0; c0 < nrhs; c0 += RMAX) {
      const int nr = std::min(RMAX, nrhs - c0);
      for (int level = 1; level <= Hmax; ++level) {
        std::vector<NearItem> items;
        std::vector<NearReduce> red;
        int64_t psz = 0;
        int max_list = 0;
        // sizes first: the partial blocks of every item of this level
        for (const NearList& L : near_lists) {
          if (L.level != level) continue;
          const Node& A = nd[L.g];
          const int nchunks = (A.size + CHUNK - 1) / CHUNK + (A.s > 0 ? 1 : 0);
          psz += (int64_t)((L.n + TR - 1) / TR) * nchunks * TR * nr;
        }
        if (psz == 0) continue;
        double* part = near_part.ensure_n<double>(psz);
        int64_t po = 0;
        for (const NearList& L : near_lists) {
          if (L.level != level) continue;
          const Node& A = nd[L.g];
          const Prob& P = pr[A.prob];
          const int par = parent(L.g);
          const int nchunks = (A.size + CHUNK - 1) / CHUNK + (A.s > 0 ? 1 : 0);
          const int* tg = near_tgt.as<int>() + L.first;
          red.push_back(NearReduce{tg, L.n, nchunks, part + po, (size_t)P.pbase * nrhs + (size_t)c0 * P.N, P.pbase,
                                   P.N});
          max_list = std::max(max_list, L.n);
          for (int r0 = 0; r0 < L.n; r0 += TR) {
            for (int j = 0; j < A.size; j += CHUNK) {  // exact: the node's points
              NearItem it{};
              it.tgt = tg;
              it.n = L.n;
              it.r0 = r0;
              it.cols = nullptr;
              it.col0 = A.off + j;
              it.ncols = std::min(CHUNK, A.size - j);
              it.y = Wp + (size_t)P.pbase * nrhs + (size_t)(A.off + j - P.pbase) + (size_t)c0 * P.N;
              it.ldy = P.N;
              it.sign = 1.0;
              it.scale = P.scale;
              it.part = part + po;
              po += (int64_t)TR * nr;
              items.push_back(it);
            }
            if (A.s > 0) {  // minus the skeleton evaluation: K(x, X_skel) w~
              NearItem it{};
              it.tgt = tg;
              it.n = L.n;
              it.r0 = r0;
              it.cols = skel.as<int>() + (size_t)L.g * s_max;
              it.col0 = 0;
              it.ncols = A.s;
              it.y = WT + woff[par] + rowoff(L.g) + (size_t)c0 * n2(par);
              it.ldy = n2(par);
              it.sign = -1.0;
              it.scale = P.scale;
              it.part = part + po;
              po += (int64_t)TR * nr;
              items.push_back(it);
            }
          }
        }
        arena.clear();
        const size_t oi = arena.push(items), orr = arena.push(red);
        char* base = upload_arena();
        near_tiles(Xp.as<double>(), xnrm.as<double>(), d, nr, (const NearItem*)(base + oi), (int)items.size(),
                   (const NearReduce*)(base + orr), (int)red.size(), max_list, Up, st);
        IA_CUDA(cudaStreamSynchronize(st));  // the arena is reused by the next level
      }
    }
  }

  // ------------------------------------------------- sliced FP64 operator blocks
  // The mixed form's FP64 operator blocks (problems with op64) as BF16 digit records for
  // the tensor-core products of ozaki.cu, split from Kleaf / Ustore at the first apply
  // after a factorization, a refactorization or an operator upgrade.
  bool slices_ready = false;
  DevBuf ozrec, ozexp, ozb;
  std::vector<int64_t> oz_lrec, oz_lexp, oz_urec, oz_uexp, oz_prec, oz_pexp;  // per node (-1: none)
  size_t ozb_bytes = 0;  // B records of the largest Evaluate launch (OZ_NR columns each)
  bool sliced(int g) const { return prec == PREC_MIXED && opt.op_slices && pr[nd[g].prob].op64; }
  void build_slices() {
    const size_t nn = nd.size();
    oz_lrec.assign(nn, -1);
    oz_lexp.assign(nn, -1);
    oz_urec.assign(nn, -1);
    oz_uexp.assign(nn, -1);
    oz_prec.assign(nn, -1);
    oz_pexp.assign(nn, -1);
    size_t rb = 0;
    int64_t eb = 0;
    for (size_t g = 0; g < nn; ++g) {
      if (!sliced((int)g)) continue;
      const Node& n = nd[g];
      if (is_leaf((int)g)) {
        oz_lrec[g] = (int64_t)rb;
        rb += oz_arec_bytes(n.size, n.size);
        oz_lexp[g] = eb;
        eb += n.size;
      }
      if (!is_root((int)g) && nd[sibling((int)g)].s > 0) {
        oz_urec[g] = (int64_t)rb;
        rb += oz_arec_bytes(n.size, nd[sibling((int)g)].s);
        oz_uexp[g] = eb;
        eb += n.size;
      }
      if (!is_root((int)g) && n.s > 0 && n.ncols > 0) {  // P of the skeletonize step
        oz_prec[g] = (int64_t)rb;
        rb += oz_arec_bytes(n.s, n.ncols);
        oz_pexp[g] = eb;
        eb += n.s;
      }
    }
    // B records of one Evaluate launch: one height's U blocks, or the leaf blocks
    ozb_bytes = 0;
    for (int hh = 0; hh <= Hmax; ++hh) {
      size_t bu = 0, bl = 0, bp = 0;
      for (int c : by_height[hh]) {
        if (oz_urec[c] >= 0) bu += oz_brec_bytes(nd[sibling(c)].s) + 256;
        if (oz_lrec[c] >= 0) bl += oz_brec_bytes(nd[c].size) + 256;
        if (oz_prec[c] >= 0) bp += oz_brec_bytes(nd[c].ncols) + 256;
      }
      ozb_bytes = std::max(ozb_bytes, std::max(bp, std::max(bu, bl)));
    }
    if (rb == 0) {
      slices_ready = true;
      return;
    }
    if (opt.mem_cap_gb > 0 && (double)rb > opt.mem_cap_gb * 1e9)
      throw Error(IASKIT_ERR_NOMEM, "sliced operator exceeds mem_cap_gb");
    unsigned char* rec = ozrec.ensure_n<unsigned char>(rb);
    int* ex = ozexp.ensure_n<int>((size_t)eb);
    ozb.ensure_n<unsigned char>(std::max<size_t>(ozb_bytes, 256));
    stats.bytes_slices = (int64_t)rb + eb * 4;
    std::vector<OzSplitDesc> sd;
    int tiles = 0;
    for (size_t g = 0; g < nn; ++g) {
      const Node& n = nd[g];
      if (oz_lrec[g] >= 0) {
        sd.push_back(OzSplitDesc{Kleaf.as<double>() + n.K_off, n.size, n.size, n.size, rec + oz_lrec[g],
                                 ex + oz_lexp[g], tiles});
        tiles += (int)ceil_div((size_t)n.size, OZ_TM);
      }
      if (oz_urec[g] >= 0) {
        sd.push_back(OzSplitDesc{Ustore.as<double>() + n.U_off, n.size, n.size, nd[sibling((int)g)].s,
                                 rec + oz_urec[g], ex + oz_uexp[g], tiles});
        tiles += (int)ceil_div((size_t)n.size, OZ_TM);
      }
      if (oz_prec[g] >= 0) {
        sd.push_back(OzSplitDesc{Pd.as<double>() + n.P_off, n.s, n.s, n.ncols, rec + oz_prec[g], ex + oz_pexp[g],
                                 tiles});
        tiles += (int)ceil_div((size_t)n.s, OZ_TM);
      }
    }
    arena.clear();
    const size_t od = arena.push(sd);
    char* base = upload_arena();
    prof().bytes[PK_OZ_SPLIT] += (double)rb + (double)rb / (OZ_S * 2) * 8;  // digits written, FP64 read
    oz_split_blocks((const OzSplitDesc*)(base + od), (int)sd.size(), tiles, st);
    slices_ready = true;
  }
  // One launch of sliced blocks: out (+)= A w per job (add = 0: out = A w), OZ_NR columns
  // per pass.
  struct OzJob {
    const unsigned char* arec;
    const int* rexp;
    int rows, K;
    const double* w;
    int ldw;
    double* out;
    int ldo;
    int add;
  };
  void run_slices(const std::vector<OzJob>& jobs, int nrhs) {
    if (jobs.empty()) return;
    for (int g0 = 0; g0 < nrhs; g0 += OZ_NR) {
      const int nr = std::min(OZ_NR, nrhs - g0);
      std::vector<OzVecDesc> vd;
      std::vector<OzApplyDesc> ad;
      unsigned char* brec = ozb.as<unsigned char>();
      size_t bo = 0;
      int tiles = 0;
      double flops = 0, bytes = 0;
      for (const OzJob& J : jobs) {
        int* cexp = reinterpret_cast<int*>(brec + bo);  // 16 exponents, then the records
        unsigned char* rec = brec + bo + 256;
        bo += oz_brec_bytes(J.K) + 256;
        vd.push_back(OzVecDesc{J.w + (size_t)g0 * J.ldw, J.ldw, J.K, nr, rec, cexp});
        ad.push_back(OzApplyDesc{J.arec, J.rexp, rec, cexp, J.out + (size_t)g0 * J.ldo, J.ldo, J.rows,
                                 (int)ceil_div((size_t)J.K, OZ_KC), nr, tiles, J.add});
        tiles += (int)ceil_div((size_t)J.rows, OZ_TM);
        flops += 2.0 * J.rows * J.K * nr;
        bytes += (double)oz_arec_bytes(J.rows, J.K) + 2.0 * 8.0 * J.rows * nr;
      }
      if (bo > ozb.bytes) throw Error(IASKIT_ERR_UNSUPPORTED, "sliced operator: right-hand-side records");
      arena.clear();
      const size_t ov = arena.push(vd), oa = arena.push(ad);
      char* base = upload_arena();
      prof().flops[PK_OZ] += flops;
      prof().bytes[PK_OZ] += bytes;
      oz_split_vecs((const OzVecDesc*)(base + ov), (int)vd.size(), st);
      oz_apply((const OzApplyDesc*)(base + oa), (int)ad.size(), tiles, status.as<int>(), st);
    }
  }

  void apply_device(const double* w, double* u, int nrhs) {
    if (!factored) throw Error(IASKIT_ERR_NOT_FACTORED, "no factorization");
    if (nrhs < 1) throw Error(IASKIT_ERR_ARG, "bad nrhs");
    use_kernel(kspec);
    struct ApplyScope {
      bool& f;
      explicit ApplyScope(bool& flag) : f(flag) { f = true; }
      ~ApplyScope() { f = false; }
    } scope(in_apply);
    const double t0 = now_ms();
    const bool stored = prec == PREC_MIXED;
    const size_t n = (size_t)Ntot * nrhs;
    double* Wp = ubuf.ensure_n<double>(2 * n);
    double* Up = Wp + n;
    const BlockDesc* blocks = upload_blocks(nrhs, true);
    gather(w, Wp, nrhs, blocks, false);
    if (stored) {
      IA_CUDA(cudaMemsetAsync(Up, 0, n * sizeof(double), st));
    } else {
      ProfScope _ps(PK_MISC, st);
      scale_blocks_kernel<<<dim3(1024, (unsigned)pr.size()), 256, 0, st>>>(Wp, Up, blocks, nrhs);
      IA_LAUNCH_CHECK();
    }
    // node g's rows inside its problem's block: base + pbase*nrhs + (off - pbase), ld N_p
    auto rows = [&](double* base, int g) {
      const Prob& P = pr[nd[g].prob];
      return base + (size_t)P.pbase * nrhs + (nd[g].off - P.pbase);
    };
    auto ldp = [&](int g) { return pr[nd[g].prob].N; };
    std::vector<int64_t> woff(nd.size(), 0);
    int64_t tot = 0;
    for (int hh = 1; hh <= Hmax; ++hh)
      for (int g : by_height[hh]) {
        woff[g] = tot;
        tot += (int64_t)n2(g) * nrhs;
      }
    double* WT = wt.ensure_n<double>(std::max<int64_t>(tot, 1));
    auto wsib = [&](int c) {  // w~ of the sibling of c, inside the parent's [w~_a; w~_b]
      const int par = parent(c), sib = sibling(c);
      return WT + woff[par] + rowoff(sib);
    };
    // Skeletonize: w~ = P w, leaves first, up to the children of the roots
    const float2* Pp = Ppair.as<float2>();
    const bool use_oz = stored && opt.op_slices && !apply_low;
    if (use_oz && !slices_ready) build_slices();
    bool oz_ran = false;
    for (int hh = 0; hh < Hmax; ++hh) {
      std::vector<GemmDesc> g;
      std::vector<GemmDescPair> gp;
      std::vector<OzJob> oz;
      for (int c : by_height[hh]) {
        if (is_root(c)) continue;
        const int par = parent(c);
        const double* src = hh == 0 ? rows(Wp, c) : WT + woff[c];
        const int lds = hh == 0 ? ldp(c) : n2(c);
        if (use_oz && sliced(c)) {  // FP64 P on the tensor cores
          if (oz_prec[c] >= 0)
            oz.push_back(OzJob{ozrec.as<unsigned char>() + oz_prec[c], ozexp.as<int>() + oz_pexp[c], nd[c].s,
                               nd[c].ncols, src, lds, WT + woff[par] + rowoff(c), n2(par), 0});
          continue;
        }
        if (stored && !pr[nd[c].prob].op64)
          add_pair_gemm(gp, Pp + nd[c].P_off, nd[c].s, src, lds, WT + woff[par] + rowoff(c), n2(par), nd[c].s,
                        nrhs, nd[c].ncols, 0.0);
        else
          add_gemm<double>(g, Pd.as<double>() + nd[c].P_off, nd[c].s, src, lds,
                           WT + woff[par] + rowoff(c), n2(par), nd[c].s, nrhs, nd[c].ncols, 1.0, 0.0);
      }
      run_gemms(g);
      run_pair_gemms(gp);
      run_slices(oz, nrhs);
      oz_ran = oz_ran || !oz.empty();
    }
    // Evaluate: one launch per height keeps the rows written by a launch disjoint
    int* sk = skel.as<int>();
    for (int hh = 0; hh <= Hmax; ++hh) {
      for (int pass = 0; pass < 2; ++pass) {  // pass 0: sibling skeletons, pass 1: leaf blocks
        if (pass == 1 && hh != 0) continue;
        std::vector<GemmDescPair> g;
        std::vector<GemmDesc> g64;
        std::vector<KMatvecDesc> md;
        std::vector<OzJob> oz;
        int max_rows = 0;
        for (int c : by_height[hh]) {
          if (pass == 0 && is_root(c)) continue;
          if (use_oz && sliced(c)) {  // FP64 blocks on the tensor cores
            const Prob& P = pr[nd[c].prob];
            if (pass == 0 && oz_urec[c] >= 0)
              oz.push_back(OzJob{ozrec.as<unsigned char>() + oz_urec[c], ozexp.as<int>() + oz_uexp[c], nd[c].size,
                                 nd[sibling(c)].s, wsib(c), n2(parent(c)), rows(Up, c), P.N, 1});
            else if (pass == 1 && oz_lrec[c] >= 0)
              oz.push_back(OzJob{ozrec.as<unsigned char>() + oz_lrec[c], ozexp.as<int>() + oz_lexp[c], nd[c].size,
                                 nd[c].size, rows(Wp, c), ldp(c), rows(Up, c), P.N, 1});
            continue;
          }
          if (pass == 0) {
            const int sib = sibling(c);
            if (stored && pr[nd[c].prob].op64)
              add_gemm<double>(g64, Ustore.as<double>() + nd[c].U_off, nd[c].size, wsib(c), n2(parent(c)),
                               rows(Up, c), ldp(c), nd[c].size, nrhs, nd[sib].s, 1.0, 1.0);
            else if (stored)
              add_pair_gemm(g, Ustore.as<float2>() + nd[c].U_off, nd[c].size, wsib(c), n2(parent(c)),
                            rows(Up, c), ldp(c), nd[c].size, nrhs, nd[sib].s, 1.0);
            else
              md.push_back(KMatvecDesc{sk + (size_t)sib * s_max, wsib(c), rows(Up, c), nd[c].off,
                                       nd[c].size, 0, nd[sib].s, n2(parent(c)), ldp(c), scale_of(c)});
          } else {
            if (stored && pr[nd[c].prob].op64)
              add_gemm<double>(g64, Kleaf.as<double>() + nd[c].K_off, nd[c].size, rows(Wp, c), ldp(c),
                               rows(Up, c), ldp(c), nd[c].size, nrhs, nd[c].size, 1.0, 1.0);
            else if (stored)
              add_pair_gemm(g, Kleaf.as<float2>() + nd[c].K_off, nd[c].size, rows(Wp, c), ldp(c),
                            rows(Up, c), ldp(c), nd[c].size, nrhs, nd[c].size, 1.0);
            else
              md.push_back(KMatvecDesc{nullptr, rows(Wp, c), rows(Up, c), nd[c].off, nd[c].size,
                                       nd[c].off, nd[c].size, ldp(c), ldp(c), scale_of(c)});
          }
          max_rows = std::max(max_rows, nd[c].size);
        }
        if (stored) {
          run_pair_gemms(g);
          run_gemms(g64);
          run_slices(oz, nrhs);
          oz_ran = oz_ran || !oz.empty();
        } else if (!md.empty()) {
          arena.clear();
          size_t om = arena.push(md);
          char* base = upload_arena();
          kernel_matvec(Xp.as<double>(), xnrm.as<double>(), d, nrhs, (const KMatvecDesc*)(base + om), (int)md.size(),
                        max_rows, st);
        }
      }
    }
    // kNN-separated operator: nodes of a target's list that hold one of its nearest
    // neighbours are evaluated exactly instead of through their skeletons (eq. askit)
    if (opt.near_field && Hmax > 0 && kappa > 0) near_field_apply(Wp, WT, woff, Up, nrhs);
    gather(Up, u, nrhs, blocks, true);
    IA_CUDA(cudaStreamSynchronize(st));
    if (oz_ran) raise_status(read_status_and_clear());
    prof().resolve();
    stats.t_apply = now_ms() - t0;
  }

  void release() {
    factored = false;
    skeletonized = false;
    near_ready = false;
    slices_ready = false;
    xdig_ready = false;
    DevBuf* all[] = {&X, &Xp, &perm, &iperm, &pid, &knn, &knn_pos, &samp, &ranks, &skel,
                     &piv_ws, &A_ws, &status, &arena_dev, &step_dev, &tbuf, &vbuf, &vbuf32,
                     &ubuf, &rbuf, &wt, &io, &normbuf, &redpart, &blocks_dev, &LU, &LUpiv, &Wb, &Zb, &Zpiv,
                     &Cb, &LU32, &Wb32, &Zb32, &Cb32, &tbuf32, &Kleaf, &Ustore, &Pd, &Pf, &Ppair, &Xpair, &DInv32, &LUi32, &Zi32, &fsS, &rhs_keep,
                     &gseg_dev, &kryl, &kzb, &coefbuf, &cseg_dev, &rowsum, &l_cand, &l_hits,
                     &l_feat, &l_score, &l_linfo, &l_samp, &l_rk, &l_Ptmp, &l_sktmp, &l_hold, &l_err,
                     &l_cols, &l_gram, &l_dense, &mlp_master, &mlp_m, &mlp_v, &mlp_grad, &mlp_b16,
                     &mlp_loss, &tr_feat, &tr_tgt, &tr_lev, &tr_bx, &tr_bt, &tr_y, &tr_H1, &tr_H2, &tr_idx,
                     &xnrm, &pred_part, &pred_io, &kperm, &kiperm, &Xk, &near_mask, &near_tgt, &near_part, &near_io,
                     &ozrec, &ozexp, &ozb, &ozXD, &ozXE};
    mlp_ready = false;
    for (DevBuf* b : all) b->release();
    tree_s.release();
    knn_s.release();
    samp_s.release();
  }
};

Solver& S() {
  static Solver s;
  return s;
}

thread_local std::string g_err = "no error";

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

template <typename F>
int guarded(F&& f) {
  try {
    f();
    return IASKIT_OK;
  } catch (const Error& e) {
    return fail(e.code, e.what());
  } catch (const std::exception& e) {
    return fail(IASKIT_ERR_CUDA, e.what());
  }
}

void require_factored() {
  if (!S().factored) throw Error(IASKIT_ERR_NOT_FACTORED, "no factorization");
}

const Prob& selected_problem() {
  Solver& s = S();
  if (s.opt.problem < 0 || s.opt.problem >= (int)s.pr.size())
    throw Error(IASKIT_ERR_ARG, "selected problem out of range");
  return s.pr[s.opt.problem];
}

// gid of node (level, index) of the selected problem
int check_node(int level, int index) {
  const Prob& P = selected_problem();
  if (level < 1 || level > P.L || index < 0 || index >= (1 << level))
    throw Error(IASKIT_ERR_ARG, "node out of range");
  return P.nbase + (1 << level) + index;
}

int factor_batched_impl(int nprob, const double* const* points, const double* concat,
                        const int64_t* N, int d, const double* h, const double* lambda, int leaf_m,
                        int s_max, double tol, bool dev) {
  int rc = guarded([&] {
    if (nprob < 1 || !N || !h || !lambda) throw Error(IASKIT_ERR_ARG, "bad batch description");
    std::vector<Solver::ProbIn> in;
    for (int q = 0; q < nprob; ++q)
      in.push_back(Solver::ProbIn{concat ? (q == 0 ? concat : nullptr) : points[q], N[q], h[q], lambda[q]});
    S().factor(in, dev, concat != nullptr, d, leaf_m, s_max, tol);
  });
  if (rc != IASKIT_OK) S().factored = false;
  return rc;
}

}  // namespace

// Records a failure for iaskit_last_error() and returns its code.
int report_error(int code, const std::string& msg) { return fail(code, msg); }

int& gemm_tuned(int fp64, int nb, int mb) {
  static int table[2][GT_NB][GT_MB] = {};
  static bool init = false;
  if (!init) {
    for (auto& a : table)
      for (auto& b : a)
        for (int& e : b) e = -1;
    init = true;
  }
  return table[fp64 ? 1 : 0][nb][mb];
}

// One timed grouped CUDA-core GEMM of `count` independent M x N x K problems with the
// given tile shape: average milliseconds over `reps` launches after one warm-up.
double tune_gemm_ms(Solver& s, int fp64, int M, int N, int K, int count, GemmShape shape, int reps) {
  auto run = [&](auto tag) -> double {
    using T = decltype(tag);
    const size_t a = (size_t)M * K, b = (size_t)K * N, c = (size_t)M * N;
    T* base = s.io.ensure_n<T>((a + b + c) * count);
    IA_CUDA(cudaMemsetAsync(base, 0, (a + b + c) * count * sizeof(T), s.st));
    std::vector<GemmDescT<T>> g;
    for (int i = 0; i < count; ++i) {
      T* A = base + (a + b + c) * i;
      add_gemm<T>(g, A, M, A + a, K, A + a + b, M, M, N, K, 1.0, 1.0);
    }
    std::vector<GemmTile> t;
    const int tm = gemm_tile_m(shape), tn = gemm_tile_n(shape);
    for (int idx = 0; idx < count; ++idx)
      for (int j = 0; j < (N + tn - 1) / tn; ++j)
        for (int i = 0; i < (M + tm - 1) / tm; ++i) t.push_back(GemmTile{idx, i, j});
    s.arena.clear();
    const size_t og = s.arena.push(g), ot = s.arena.push(t);
    char* dev = s.upload_arena();
    cudaEvent_t e0, e1;
    IA_CUDA(cudaEventCreate(&e0));
    IA_CUDA(cudaEventCreate(&e1));
    gemm_grouped((const GemmDescT<T>*)(dev + og), (const GemmTile*)(dev + ot), (int)t.size(), shape, s.st,
                 s.status.ensure_n<int>(1));
    IA_CUDA(cudaEventRecord(e0, s.st));
    for (int r = 0; r < reps; ++r)
      gemm_grouped((const GemmDescT<T>*)(dev + og), (const GemmTile*)(dev + ot), (int)t.size(), shape, s.st,
                   s.status.as<int>());
    IA_CUDA(cudaEventRecord(e1, s.st));
    IA_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    IA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / reps;
  };
  return fp64 ? run(double{}) : run(float{});
}
}  // namespace iaskit

using namespace iaskit;

extern "C" {

int iaskit_factor(const double* points, int64_t N, int d, double h, double lambda, int leaf_m,
                  int s_max, double tol) {
  if (!points) return fail(IASKIT_ERR_ARG, "points is null");
  const double* pts[1] = {points};
  return factor_batched_impl(1, pts, nullptr, &N, d, &h, &lambda, leaf_m, s_max, tol, false);
}

int iaskit_factor_device(const double* d_points, int64_t N, int d, double h, double lambda,
                         int leaf_m, int s_max, double tol) {
  if (!d_points) return fail(IASKIT_ERR_ARG, "points is null");
  return factor_batched_impl(1, nullptr, d_points, &N, d, &h, &lambda, leaf_m, s_max, tol, true);
}

int iaskit_factor_batched(int nprob, const double* const* points, const int64_t* N, int d,
                          const double* h, const double* lambda, int leaf_m, int s_max, double tol) {
  if (!points) return fail(IASKIT_ERR_ARG, "points is null");
  return factor_batched_impl(nprob, points, nullptr, N, d, h, lambda, leaf_m, s_max, tol, false);
}

int iaskit_factor_batched_device(int nprob, const double* d_points, const int64_t* N, int d,
                                 const double* h, const double* lambda, int leaf_m, int s_max,
                                 double tol) {
  if (!d_points) return fail(IASKIT_ERR_ARG, "points is null");
  return factor_batched_impl(nprob, nullptr, d_points, N, d, h, lambda, leaf_m, s_max, tol, true);
}

int iaskit_num_problems(void) {
  if (!S().factored) return fail(IASKIT_ERR_NOT_FACTORED, "no factorization");
  return (int)S().pr.size();
}

int iaskit_refactor(const double* lambda, int nprob) {
  int rc = guarded([&] {
    require_factored();
    S().refactor(lambda, nprob);
  });
  // a failure past the argument checks leaves no usable factorization
  if (rc != IASKIT_OK && rc != IASKIT_ERR_ARG && rc != IASKIT_ERR_NOT_FACTORED) S().factored = false;
  return rc;
}

int iaskit_solve_device(double* d_rhs, int nrhs) {
  return guarded([&] {
    if (!d_rhs) throw Error(IASKIT_ERR_ARG, "rhs is null");
    S().solve_device(d_rhs, nrhs);
  });
}

int iaskit_solve_batched_device(double* d_rhs, int nrhs) { return iaskit_solve_device(d_rhs, nrhs); }

int iaskit_solve(double* rhs, int nrhs) {
  return guarded([&] {
    Solver& s = S();
    require_factored();
    if (!rhs) throw Error(IASKIT_ERR_ARG, "rhs is null");
    if (nrhs < 1) throw Error(IASKIT_ERR_ARG, "bad nrhs");
    const size_t n = (size_t)s.Ntot * nrhs;
    double* d = s.io.ensure_n<double>(n);
    h2d(d, rhs, n, s.st);
    s.solve_device(d, nrhs);
    d2h(rhs, d, n, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
}

int iaskit_solve_batched(double* const* rhs, int nrhs) {
  return guarded([&] {
    Solver& s = S();
    require_factored();
    if (!rhs) throw Error(IASKIT_ERR_ARG, "rhs is null");
    if (nrhs < 1) throw Error(IASKIT_ERR_ARG, "bad nrhs");
    const size_t n = (size_t)s.Ntot * nrhs;
    double* d = s.io.ensure_n<double>(n);
    for (size_t q = 0; q < s.pr.size(); ++q) {
      if (!rhs[q]) throw Error(IASKIT_ERR_ARG, "rhs is null");
      h2d(d + (size_t)s.pr[q].pbase * nrhs, rhs[q], (size_t)s.pr[q].N * nrhs, s.st);
    }
    s.solve_device(d, nrhs);
    for (size_t q = 0; q < s.pr.size(); ++q)
      d2h(rhs[q], d + (size_t)s.pr[q].pbase * nrhs, (size_t)s.pr[q].N * nrhs, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
}

int iaskit_apply_device(const double* d_w, double* d_u, int nrhs) {
  return guarded([&] {
    if (!d_w || !d_u) throw Error(IASKIT_ERR_ARG, "null pointer");
    S().apply_device(d_w, d_u, nrhs);
  });
}

int iaskit_gemm_tile(int fp64, int n_bucket, int m_bucket, int shape) {
  return guarded([&] {
    if (fp64 < 0 || fp64 > 1 || n_bucket < 0 || n_bucket >= GT_NB || m_bucket < 0 || m_bucket >= GT_MB)
      throw Error(IASKIT_ERR_ARG, "bad tile table key");
    if (shape != -1 && (shape < 0 || shape >= GEMM_NSHAPES || !gemm_shape_valid((GemmShape)shape, fp64 != 0)))
      throw Error(IASKIT_ERR_ARG, "not a CUDA-core tile shape of this type");
    gemm_tuned(fp64, n_bucket, m_bucket) = shape;
  });
}

int iaskit_tune_gemm(int fp64, int M, int N, int K, int count, int shape, int reps, double* ms) {
  return guarded([&] {
    if (!ms) throw Error(IASKIT_ERR_ARG, "null pointer");
    if (M < 1 || N < 1 || K < 1 || count < 1 || reps < 1 || reps > 1000 || fp64 < 0 || fp64 > 1)
      throw Error(IASKIT_ERR_ARG, "bad GEMM size");
    if ((double)count * ((double)M * K + (double)K * N + (double)M * N) * (fp64 ? 8 : 4) > 4e9)
      throw Error(IASKIT_ERR_ARG, "tuning problem above 4 GB");
    if (shape < 0 || shape >= GEMM_NSHAPES || !gemm_shape_valid((GemmShape)shape, fp64 != 0))
      throw Error(IASKIT_ERR_ARG, "not a CUDA-core tile shape of this type");
    *ms = tune_gemm_ms(S(), fp64, M, N, K, count, (GemmShape)shape, reps);
  });
}

int iaskit_predict_device(const double* d_test, int64_t M, const double* d_w, int nrhs, double* d_scores) {
  return guarded([&] {
    Solver& s = S();
    if ((!d_test || !d_w || !d_scores) && M > 0) throw Error(IASKIT_ERR_ARG, "null pointer");
    const int q = s.opt.problem;
    if (q < 0 || q >= (int)s.pr.size()) throw Error(IASKIT_ERR_ARG, "selected problem out of range");
    s.predict_device(d_test, M, d_w, nrhs, d_scores, q);
  });
}

int iaskit_predict(const double* test, int64_t M, const double* w, int nrhs, double* scores) {
  return guarded([&] {
    Solver& s = S();
    if ((!test || !w || !scores) && M > 0) throw Error(IASKIT_ERR_ARG, "null pointer");
    const int q = s.opt.problem;
    if (q < 0 || q >= (int)s.pr.size()) throw Error(IASKIT_ERR_ARG, "selected problem out of range");
    if (M < 0 || M > INT_MAX / 2) throw Error(IASKIT_ERR_ARG, "bad number of test points");
    if (nrhs < 1 || nrhs > 4096) throw Error(IASKIT_ERR_ARG, "bad nrhs");
    if (M == 0) return;
    const int64_t nT = M * s.d, nW = (int64_t)s.pr[q].N * nrhs, nO = M * nrhs;
    double* dT = s.pred_io.ensure_n<double>(nT + nW + nO);
    double* dW = dT + nT;
    double* dO = dW + nW;
    h2d(dT, test, nT, s.st);
    h2d(dW, w, nW, s.st);
    s.predict_device(dT, M, dW, nrhs, dO, q);
    d2h(scores, dO, nO, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
}

int iaskit_apply(const double* w, double* u, int nrhs) {
  return guarded([&] {
    Solver& s = S();
    require_factored();
    if (!w || !u) throw Error(IASKIT_ERR_ARG, "null pointer");
    if (nrhs < 1) throw Error(IASKIT_ERR_ARG, "bad nrhs");
    const size_t n = (size_t)s.Ntot * nrhs;
    double* dw = s.io.ensure_n<double>(2 * n);
    double* du = dw + n;
    h2d(dw, w, n, s.st);
    s.apply_device(dw, du, nrhs);
    d2h(u, du, n, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
}

int iaskit_set_option(const char* key, double value) {
  return guarded([&] {
    if (!key) throw Error(IASKIT_ERR_ARG, "null key");
    Options& o = S().opt;
    std::string k(key);
    auto as_int = [&](double lo, double hi) {
      if (!(value >= lo && value <= hi) || value != std::floor(value))
        throw Error(IASKIT_ERR_ARG, "invalid value for " + k);
      return (int)value;
    };
    if (k == "kappa") o.kappa = as_int(1, 48);
    else if (k == "samp_factor") o.samp_factor = as_int(1, 64);
    else if (k == "seed") {
      if (!(value >= 0 && value <= 9007199254740992.0)) throw Error(IASKIT_ERR_ARG, "invalid seed");
      o.seed = (uint64_t)value;
    } else if (k == "refine") o.refine = as_int(0, 1000);
    else if (k == "refine_tol") {
      if (!(value > 0)) throw Error(IASKIT_ERR_ARG, "invalid refine_tol");
      o.refine_tol = value;
    } else if (k == "mem_cap_gb") {
      if (!(value >= 0)) throw Error(IASKIT_ERR_ARG, "invalid mem_cap_gb");
      o.mem_cap_gb = value;
    } else if (k == "precision") {
      o.precision = as_int(0, 1);
    } else if (k == "problem") {
      o.problem = as_int(0, 1 << 30);
    } else if (k == "mixed_cond_max") {
      if (!(value >= 1.0)) throw Error(IASKIT_ERR_ARG, "invalid mixed_cond_max");
      o.mixed_cond_max = value;
    } else if (k == "sampling") {
      o.sampling = as_int(0, 1);
    } else if (k == "cand_factor") {
      o.cand_factor = as_int(2, 64);
    } else if (k == "keep_candidates") {
      o.keep_candidates = as_int(0, 1);
    } else if (k == "train_batch") {
      o.train_batch = as_int(64, 1 << 20);
    } else if (k == "learned_temp") {
      if (!(value >= 0.0) || !std::isfinite(value)) throw Error(IASKIT_ERR_ARG, "invalid learned_temp");
      o.learned_temp = value;
    } else if (k == "gemm_tc") {
      o.gemm_tc = as_int(0, 1);
    } else if (k == "cpqr_cluster") {
      o.cpqr_cluster = as_int(0, 1);
    } else if (k == "lu_inverse") {
      o.lu_inverse = as_int(0, 2);
    } else if (k == "lu_inverse_zh") {
      o.lu_inverse_zh = as_int(0, 1 << 20);
    } else if (k == "pair_cond_max") {
      if (!(value >= 1.0)) throw Error(IASKIT_ERR_ARG, "invalid pair_cond_max");
      o.pair_cond_max = value;
    } else if (k == "near_field") {
      o.near_field = as_int(0, 1);
    } else if (k == "inject_status") {
      o.inject_status = as_int(0, 15);
    } else if (k == "knn_prune") {
      o.knn_prune = as_int(0, 1);
    } else if (k == "inner_pair") {
      o.inner_pair = as_int(0, 1);
    } else if (k == "op_slices") {
      o.op_slices = as_int(0, 1);
    } else if (k == "kernel") {
      o.kernel = as_int(0, 1);
    } else if (k == "poly_p") {
      o.poly_p = as_int(1, 16);
    } else if (k == "poly_c") {
      if (!(value >= 0.0) || !std::isfinite(value)) throw Error(IASKIT_ERR_ARG, "invalid poly_c");
      o.poly_c = value;
    } else if (k == "profile") {
      int v = as_int(0, 1);
      IA_CUDA(cudaStreamSynchronize(S().st));
      prof().reset();
      prof().enabled = v != 0;
    } else throw Error(IASKIT_ERR_ARG, "unknown option " + k);
  });
}

int iaskit_get_option(const char* key, double* value) {
  return guarded([&] {
    if (!key || !value) throw Error(IASKIT_ERR_ARG, "null argument");
    const Options& o = S().opt;
    std::string k(key);
    if (k == "kappa") *value = o.kappa;
    else if (k == "samp_factor") *value = o.samp_factor;
    else if (k == "seed") *value = (double)o.seed;
    else if (k == "refine") *value = o.refine;
    else if (k == "refine_tol") *value = o.refine_tol;
    else if (k == "mem_cap_gb") *value = o.mem_cap_gb;
    else if (k == "profile") *value = prof().enabled ? 1 : 0;
    else if (k == "precision") *value = o.precision;
    else if (k == "problem") *value = o.problem;
    else if (k == "mixed_cond_max") *value = o.mixed_cond_max;
    else if (k == "sampling") *value = o.sampling;
    else if (k == "cand_factor") *value = o.cand_factor;
    else if (k == "keep_candidates") *value = o.keep_candidates;
    else if (k == "train_batch") *value = o.train_batch;
    else if (k == "learned_temp") *value = o.learned_temp;
    else if (k == "gemm_tc") *value = o.gemm_tc;
    else if (k == "cpqr_cluster") *value = o.cpqr_cluster;
    else if (k == "lu_inverse") *value = o.lu_inverse;
    else if (k == "lu_inverse_zh") *value = o.lu_inverse_zh;
    else if (k == "pair_cond_max") *value = o.pair_cond_max;
    else if (k == "near_field") *value = o.near_field;
    else if (k == "inject_status") *value = o.inject_status;
    else if (k == "knn_prune") *value = o.knn_prune;
    else if (k == "inner_pair") *value = o.inner_pair;
    else if (k == "op_slices") *value = o.op_slices;
    else if (k == "kernel") *value = o.kernel;
    else if (k == "poly_p") *value = o.poly_p;
    else if (k == "poly_c") *value = o.poly_c;
    else throw Error(IASKIT_ERR_ARG, "unknown option " + k);
  });
}

int iaskit_set_stream(void* cuda_stream) {
  S().st = (cudaStream_t)cuda_stream;
  return IASKIT_OK;
}

int iaskit_stats(char* buf, size_t len) {
  Solver& s = S();
  std::string j = "{";
  char tmp[640];
  snprintf(tmp, sizeof tmp,
           "\"N\":%d,\"d\":%d,\"problems\":%d,\"L\":%d,\"factored\":%s,\"ms\":{\"tree\":%.3f,"
           "\"knn\":%.3f,\"skeletonize\":%.3f,\"leaf_lu\":%.3f,\"factor_levels\":%.3f,"
           "\"factor\":%.3f,\"solve\":%.3f,\"apply\":%.3f},\"knn_fallback\":%d,\"bytes\":{\"W\":%lld,"
           "\"LU\":%lld,\"P\":%lld,\"operator\":%lld,\"operator_slices\":%lld},\"precision\":\"%s\",\"refine_sweeps\":%d,",
           s.Ntot, s.d, (int)s.pr.size(), s.Hmax, s.factored ? "true" : "false", s.stats.t_tree,
           s.stats.t_knn, s.stats.t_skel, s.stats.t_leaf_lu, s.stats.t_factor_levels,
           s.stats.t_factor, s.stats.t_solve, s.stats.t_apply, s.stats.knn_fallback,
           (long long)s.stats.bytes_W, (long long)s.stats.bytes_LU, (long long)s.stats.bytes_P,
           (long long)s.stats.bytes_operator, (long long)s.stats.bytes_slices, s.prec == PREC_MIXED ? "mixed" : "fp64",
           s.stats.refine_sweeps);
  j += tmp;
  j += "\"refine_history\":[";
  for (size_t i = 0; i < s.stats.refine_hist.size(); ++i) {
    snprintf(tmp, sizeof tmp, "%s%.6g", i ? "," : "", s.stats.refine_hist[i]);
    j += tmp;
  }
  j += "],\"stagnated\":[";
  for (size_t i = 0; i < s.stats.stagnated.size() && i < 256; ++i) {
    const StagCol& c = s.stats.stagnated[i];
    snprintf(tmp, sizeof tmp, "%s{\"problem\":%d,\"column\":%d,\"residual\":%.4g,\"floor\":%.4g,\"op64\":%s}",
             i ? "," : "", c.prob, c.col, c.resid, c.floor, c.op64 ? "true" : "false");
    j += tmp;
  }
  snprintf(tmp, sizeof tmp, "],\"refine_iters\":%d,\"refine_stagnated\":%d,\"fp64_problems\":%d,"
           "\"fp64_operator_problems\":%d,\"operator_upgrades\":%d,",
           s.stats.refine_iters, s.stats.refine_stagnated, s.stats.fp64_problems, s.stats.fp64_operator_problems,
           s.stats.operator_upgrades);
  j += tmp;
  snprintf(tmp, sizeof tmp,
           "\"learned_nodes\":%d,\"fallback_nodes\":%d,\"judge_err_plain\":%.6g,\"judge_err_chosen\":%.6g,"
           "\"train_rows\":%lld,\"train_loss\":[",
           s.stats.learned_nodes, s.stats.fallback_nodes,
           s.stats.judged_nodes ? s.stats.judge_err_plain / s.stats.judged_nodes : 0.0,
           s.stats.judged_nodes ? s.stats.judge_err_chosen / s.stats.judged_nodes : 0.0,
           (long long)s.stats.train_rows);
  j += tmp;
  for (size_t i = 0; i < s.stats.train_loss.size(); ++i) {
    snprintf(tmp, sizeof tmp, "%s%.6g", i ? "," : "", s.stats.train_loss[i]);
    j += tmp;
  }
  j += "],";
  j += "\"cond_est\":[";
  for (size_t q = 0; q < s.pr.size() && s.factored; ++q) {
    snprintf(tmp, sizeof tmp, "%s%.17g", q ? "," : "", std::min(s.pr[q].cond_est, 1e300));
    j += tmp;
  }
  snprintf(tmp, sizeof tmp,
           "],\"knn_pairs_scanned\":%.17g,\"knn_pairs_all\":%.17g,\"knn_tiles_listed\":%lld,\"near_values\":%.17g",
           s.stats.knn_prune.pairs_scanned, s.stats.knn_prune.pairs_all, (long long)s.stats.knn_prune.tiles_scanned,
           s.stats.near_values);
  j += tmp;
  j += ",\"launches\":";
  j += std::to_string(prof().launches);
  j += ",\"kernels\":{";
  for (int k = 0; k < PK_COUNT; ++k) {
    snprintf(tmp, sizeof tmp, "%s\"%s\":{\"ms\":%.4f,\"calls\":%lld,\"flops\":%.6g,\"bytes\":%.6g}",
             k ? "," : "", prof_name(k), prof().ms[k], prof().calls[k], prof().flops[k], prof().bytes[k]);
    j += tmp;
  }
  // rank profile of the last skeletonization (also after a factorization that stopped
  // later, e.g. at mem_cap_gb): mean and largest rank per height, and the entries of
  // W (= of the U blocks) that profile implies, sum over non-root nodes of |c| s_sibling
  std::string mx = "],\"max_rank_per_height\":[";
  j += "},\"mean_rank_per_height\":[";
  double w_entries = 0;
  for (int hh = 0; hh < s.Hmax && s.skeletonized; ++hh) {
    double tot = 0;
    int cnt = 0, big = 0;
    for (int g : s.by_height[hh])
      if (!s.is_root(g)) {
        tot += s.nd[g].s;
        big = std::max(big, s.nd[g].s);
        w_entries += (double)s.nd[g].size * s.nd[s.sibling(g)].s;
        ++cnt;
      }
    snprintf(tmp, sizeof tmp, "%s%.3f", hh ? "," : "", cnt ? tot / cnt : 0.0);
    j += tmp;
    snprintf(tmp, sizeof tmp, "%s%d", hh ? "," : "", big);
    mx += tmp;
  }
  j += mx;
  snprintf(tmp, sizeof tmp, "],\"w_entries\":%.17g}", w_entries);
  j += tmp;
  if (buf && len > 0) {
    size_t n = std::min(len - 1, j.size());
    std::memcpy(buf, j.data(), n);
    buf[n] = 0;
  }
  return (int)j.size() + 1;
}

const char* iaskit_last_error(void) { return g_err.c_str(); }

void iaskit_free(void) { S().release(); }

int iaskit_depth(void) {
  if (!S().factored) return fail(IASKIT_ERR_NOT_FACTORED, "no factorization");
  int L = 0;
  const int rc = guarded([&] { L = selected_problem().L; });
  return rc == IASKIT_OK ? L : rc;
}

int iaskit_get_perm(int32_t* out) {
  return guarded([&] {
    require_factored();
    Solver& s = S();
    const Prob& P = selected_problem();
    d2h(out, s.perm.as<int>() + P.pbase, P.N, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
    for (int i = 0; i < P.N; ++i) out[i] -= P.pbase;
  });
}

int iaskit_get_knn(int32_t* out, int kappa_cap) {
  return guarded([&] {
    require_factored();
    Solver& s = S();
    const Prob& P = selected_problem();
    if (s.Hmax == 0) throw Error(IASKIT_ERR_ARG, "no kNN lists for single-leaf trees");
    if (kappa_cap < s.kappa) throw Error(IASKIT_ERR_ARG, "buffer too small");
    d2h(out, s.knn.as<int>() + (size_t)P.pbase * s.kappa, (size_t)P.N * s.kappa, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
    for (size_t i = 0; i < (size_t)P.N * s.kappa; ++i) out[i] -= P.pbase;
  });
}

int iaskit_get_ranks(int32_t* out, int count) {
  return guarded([&] {
    require_factored();
    Solver& s = S();
    const Prob& P = selected_problem();
    if (count < (2 << P.L)) throw Error(IASKIT_ERR_ARG, "buffer too small");
    for (int u = 0; u < (2 << P.L); ++u) out[u] = (u == 0 || u == 1) ? 0 : s.nd[P.nbase + u].s;
  });
}

int iaskit_get_skeleton(int level, int index, int32_t* out, int cap) {
  int rs = 0;
  int rc = guarded([&] {
    require_factored();
    Solver& s = S();
    const int g = check_node(level, index);
    const Prob& P = selected_problem();
    rs = s.nd[g].s;
    if (cap < rs) throw Error(IASKIT_ERR_ARG, "buffer too small");
    d2h(out, s.skel.as<int>() + (size_t)g * s.s_max, rs, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
    for (int i = 0; i < rs; ++i) out[i] -= P.pbase;
  });
  return rc == IASKIT_OK ? rs : rc;
}

int iaskit_get_samples(int level, int index, int32_t* out, int cap) {
  int ns = 0;
  int rc = guarded([&] {
    require_factored();
    Solver& s = S();
    const int g = check_node(level, index);
    const Prob& P = selected_problem();
    ns = s.nd[g].nsamp;
    if (cap < ns) throw Error(IASKIT_ERR_ARG, "buffer too small");
    d2h(out, s.samp.as<int>() + s.nd[g].samp_off, ns, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
    for (int i = 0; i < ns; ++i) out[i] -= P.pbase;
  });
  return rc == IASKIT_OK ? ns : rc;
}

int iaskit_get_P(int level, int index, double* out, int64_t cap) {
  int nc = 0;
  int rc = guarded([&] {
    require_factored();
    Solver& s = S();
    const int g = check_node(level, index);
    nc = s.nd[g].ncols;
    int64_t n = (int64_t)s.nd[g].s * nc;
    if (cap < n) throw Error(IASKIT_ERR_ARG, "buffer too small");
    d2h(out, s.Pd.as<double>() + s.nd[g].P_off, n, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
  return rc == IASKIT_OK ? nc : rc;
}

int iaskit_kernel_block(const double* points, int64_t N, int d, double h, const int32_t* rows, int nr,
                        const int32_t* cols, int nc, double diag, int form, double* out) {
  return guarded([&] {
    if (!points || !rows || !cols || !out) throw Error(IASKIT_ERR_ARG, "null argument");
    if (N < 1 || N > INT_MAX || d < 1 || nr < 1 || nc < 1 || !(h > 0) || form < 0 || form > 3)
      throw Error(IASKIT_ERR_ARG, "invalid size, bandwidth or form");
    for (int i = 0; i < nr; ++i)
      if (rows[i] < 0 || rows[i] >= N) throw Error(IASKIT_ERR_ARG, "row index out of range");
    for (int j = 0; j < nc; ++j)
      if (cols[j] < 0 || cols[j] >= N) throw Error(IASKIT_ERR_ARG, "column index out of range");
    for (int64_t e = 0; e < N * d; ++e)
      if (!std::isfinite(points[e])) throw Error(IASKIT_ERR_INPUT, "non-finite coordinate");
    cudaStream_t st = S().st;
    DevBuf X, aux, ri, ci, ob, db;
    double* Xd = X.ensure_n<double>((size_t)N * d);
    h2d(Xd, points, (size_t)N * d, st);
    int* rd = ri.ensure_n<int>(nr);
    int* cd = ci.ensure_n<int>(nc);
    h2d(rd, reinterpret_cast<const int*>(rows), nr, st);
    h2d(cd, reinterpret_cast<const int*>(cols), nc, st);
    const int64_t ne = (int64_t)nr * nc;
    const Options& o = S().opt;
    const KernelSpec ks{o.kernel, o.poly_p, o.poly_c};
    S().use_kernel(ks);
    const double scale = ks.poly ? 1.0 / (h * h) : -1.0 / (2.0 * h * h);
    if (form == 0) {
      double* xn = aux.ensure_n<double>(N);
      point_norms(Xd, (int)N, d, xn, st);
      double* o = ob.ensure_n<double>(ne);
      KDesc k{rd, cd, nullptr, o, 0, nr, 0, nc, nc, nr, diag, scale};
      KDesc* kd = db.ensure_n<KDesc>(1);
      h2d(kd, &k, 1, st);
      kernel_blocks<double>(Xd, xn, d, kd, 1, ne, st);
      d2h(out, o, ne, st);
      IA_CUDA(cudaStreamSynchronize(st));
    } else if (form == 1) {
      float2* xp = aux.ensure_n<float2>((size_t)N * d);
      split_pairs(Xd, xp, N * d, st);
      float2* o = ob.ensure_n<float2>(ne);
      KDescT<float2> k{rd, cd, nullptr, o, 0, nr, 0, nc, nc, nr, diag, scale};
      KDescT<float2>* kd = db.ensure_n<KDescT<float2>>(1);
      h2d(kd, &k, 1, st);
      kernel_blocks_pair(xp, d, kd, 1, ne, st);
      std::vector<float2> hv(ne);
      d2h(hv.data(), o, ne, st);
      IA_CUDA(cudaStreamSynchronize(st));
      for (int64_t e = 0; e < ne; ++e) out[e] = (double)hv[e].x + (double)hv[e].y;
    } else if (form == 3) {
      // sliced: the rows' points first (consecutive), then all points; identities for the
      // diagonal shift
      if (ks.poly || oz_dpad(d) == 0 || N + nr > INT_MAX)
        throw Error(IASKIT_ERR_UNSUPPORTED, "sliced kernel blocks: Gaussian kernel and d <= 64 only");
      const int64_t M = N + nr;
      std::vector<double> Y((size_t)M * d);
      for (int i = 0; i < nr; ++i)
        std::memcpy(&Y[(size_t)i * d], points + (size_t)rows[i] * d, sizeof(double) * d);
      std::memcpy(&Y[(size_t)nr * d], points, sizeof(double) * N * d);
      std::vector<int> ident(M), cs(nc);
      for (int i = 0; i < nr; ++i) ident[i] = rows[i];
      for (int64_t p = 0; p < N; ++p) ident[nr + p] = (int)p;
      for (int j = 0; j < nc; ++j) cs[j] = nr + cols[j];
      DevBuf Yb, yn, idb, xd, xe, cb, sb;
      double* Yd = Yb.ensure_n<double>((size_t)M * d);
      h2d(Yd, Y.data(), Y.size(), st);
      double* ynd = yn.ensure_n<double>(M);
      point_norms(Yd, (int)M, d, ynd, st);
      int* idd = idb.ensure_n<int>(M);
      h2d(idd, ident.data(), M, st);
      int* csd = cb.ensure_n<int>(nc);
      h2d(csd, cs.data(), nc, st);
      uint16_t* XD = xd.ensure_n<uint16_t>((size_t)M * OZ_S * oz_dpad(d));
      int* XE = xe.ensure_n<int>(M);
      oz_points(Yd, (int)M, d, XD, XE, st);
      double* o = ob.ensure_n<double>(ne);
      OzKDesc k{csd, nullptr, o, 0, nr, 0, nc, nc, nr, diag, scale, 0, idd};
      OzKDesc* kd = db.ensure_n<OzKDesc>(1);
      h2d(kd, &k, 1, st);
      int* stw = sb.ensure_n<int>(1);
      IA_CUDA(cudaMemsetAsync(stw, 0, sizeof(int), st));
      oz_kblocks(XD, XE, ynd, d, kd, 1, (int)ceil_div((size_t)nr, OZ_TM), stw, st);
      int sv = 0;
      d2h(&sv, stw, 1, st);
      d2h(out, o, ne, st);
      IA_CUDA(cudaStreamSynchronize(st));
      if (sv & DEV_TIMEOUT) throw Error(IASKIT_ERR_TIMEOUT, "bounded device wait expired");
    } else {
      float* o = ob.ensure_n<float>(ne);
      KDescT<float> k{rd, cd, nullptr, o, 0, nr, 0, nc, nc, nr, diag, scale};
      KDescT<float>* kd = db.ensure_n<KDescT<float>>(1);
      h2d(kd, &k, 1, st);
      kernel_blocks<float>(Xd, nullptr, d, kd, 1, ne, st);
      std::vector<float> hv(ne);
      d2h(hv.data(), o, ne, st);
      IA_CUDA(cudaStreamSynchronize(st));
      for (int64_t e = 0; e < ne; ++e) out[e] = hv[e];
    }
  });
}

int iaskit_sampler_train(const double* points, int64_t N, int d, double h, int leaf_m, int s_max,
                         double tol, int epochs, double lr) {
  return guarded([&] {
    if (!points) throw Error(IASKIT_ERR_ARG, "points is null");
    S().train_sampler(points, N, d, h, leaf_m, s_max, tol, epochs, lr);
  });
}

int iaskit_sampler_set_weights(const float* w, int n) {
  return guarded([&] {
    if (!w || n != MLP_NPARAM) throw Error(IASKIT_ERR_ARG, "weights must hold 17793 floats");
    for (int i = 0; i < n; ++i)
      if (!std::isfinite(w[i])) throw Error(IASKIT_ERR_INPUT, "non-finite weight");
    S().mlp_load(w);
  });
}

int iaskit_sampler_get_weights(float* w, int n) {
  return guarded([&] {
    Solver& s = S();
    if (!w || n != MLP_NPARAM) throw Error(IASKIT_ERR_ARG, "weights must hold 17793 floats");
    if (!s.mlp_ready) throw Error(IASKIT_ERR_NOT_FACTORED, "the sampler has no weights");
    d2h(w, s.mlp_master.as<float>(), n, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
}

namespace {
// round to nearest even BF16, NaN kept quiet
uint16_t host_bf16(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return (uint16_t)((u >> 16) | 0x40u);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
void upload_features(Solver& s, const float* feats, int64_t n, uint16_t* dst) {
  std::vector<uint16_t> hb((size_t)n * MLP_F);
  for (size_t i = 0; i < hb.size(); ++i) hb[i] = host_bf16(feats[i]);
  h2d(dst, hb.data(), hb.size(), s.st);
}
}  // namespace

int iaskit_mlp_forward(const float* feats, int64_t n, float* scores) {
  return guarded([&] {
    Solver& s = S();
    if (!feats || !scores || n < 1 || n > ((int64_t)1 << 28)) throw Error(IASKIT_ERR_ARG, "bad arguments");
    if (!s.mlp_ready) throw Error(IASKIT_ERR_NOT_FACTORED, "the sampler has no weights");
    uint16_t* X = s.tr_bx.ensure_n<uint16_t>((size_t)n * MLP_F);
    float* y = s.tr_y.ensure_n<float>(n);
    upload_features(s, feats, n, X);
    mlp_forward(X, n, s.mlp_dev(), y, nullptr, nullptr, s.st);
    d2h(scores, y, n, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
}

int iaskit_mlp_train_step(const float* feats, const float* targets, int64_t n, double lr, float* grad,
                          float* loss) {
  return guarded([&] {
    Solver& s = S();
    if (!feats || !targets || n < 1 || n > ((int64_t)1 << 24) || !(lr >= 0.0))
      throw Error(IASKIT_ERR_ARG, "bad arguments");
    if (!s.mlp_ready) throw Error(IASKIT_ERR_NOT_FACTORED, "the sampler has no weights");
    uint16_t* X = s.tr_bx.ensure_n<uint16_t>((size_t)n * MLP_F);
    float* t = s.tr_bt.ensure_n<float>(n);
    float* y = s.tr_y.ensure_n<float>(n);
    uint16_t* H1 = s.tr_H1.ensure_n<uint16_t>((size_t)n * MLP_W);
    uint16_t* H2 = s.tr_H2.ensure_n<uint16_t>((size_t)n * MLP_W);
    upload_features(s, feats, n, X);
    h2d(t, targets, n, s.st);
    IA_CUDA(cudaMemsetAsync(s.mlp_loss.p, 0, sizeof(float), s.st));
    const MlpDev w = s.mlp_dev();
    mlp_forward(X, n, w, y, H1, H2, s.st);
    mlp_backward(X, H1, H2, y, t, n, 1.0 / n, w, s.mlp_grad.as<float>(), s.mlp_loss.as<float>(), s.st);
    if (grad) d2h(grad, s.mlp_grad.as<float>(), MLP_NPARAM, s.st);
    if (loss) d2h(loss, s.mlp_loss.as<float>(), 1, s.st);
    mlp_adam(w, s.mlp_grad.as<float>(), s.mlp_m.as<float>(), s.mlp_v.as<float>(), ++s.mlp_step, lr, 0.9,
             0.999, 1e-8, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
}

int iaskit_get_learned(int level, int index, int32_t* cand, float* feat, float* value, int cap,
                       double* info) {
  int nc = 0;
  int rc = guarded([&] {
    require_factored();
    Solver& s = S();
    const int g = check_node(level, index);
    const Prob& P = selected_problem();
    if (s.kept.empty()) throw Error(IASKIT_ERR_ARG, "candidates were not kept (option keep_candidates)");
    const Solver::Kept& k = s.kept[g];
    nc = k.n;
    if (info) {
      info[0] = k.err_plain;
      info[1] = k.err_learned;
      info[2] = k.chosen;
      info[3] = k.n_samp;
    }
    if (k.off < 0) return;
    if (cap < nc) throw Error(IASKIT_ERR_ARG, "buffer too small");
    for (int i = 0; i < nc; ++i) {
      if (cand) cand[i] = s.kept_cand[k.off + i] - P.pbase;
      if (value) value[i] = s.kept_val[k.off + i];
      if (feat)
        for (int q = 0; q < MLP_F; ++q) {
          const uint32_t u = (uint32_t)s.kept_feat[(k.off + i) * MLP_F + q] << 16;
          float f;
          std::memcpy(&f, &u, 4);
          feat[(size_t)i * MLP_F + q] = f;
        }
    }
  });
  return rc == IASKIT_OK ? nc : rc;
}

}  // extern "C"
