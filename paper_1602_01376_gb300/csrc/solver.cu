// INV-ASKIT orchestration on one GPU and the C ABI of include/iaskit.h.
//
// Factorization (Sec. II-C, Alg. "Factorize", run bottom-up with loops over levels
// as the paper's implementation does):
//   tree -> kNN -> skeletonize levels L..1 (sample, kernel block, CPQR/ID, nested P)
//   -> leaf LU of lambda I + K_aa -> for l = L-1 .. 0: U blocks K_{l r~}, K_{r l~} of
//   every node of level l, W = Solve(child subtree, U) for all of them at once (a
//   "forest solve" rooted at level l+1), reduced systems Z and their LU.
// Solve (Alg. "Solve"): a forest solve rooted at level 0.
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
//    FP32 with FP64 pivot norms in the CPQR; the operator lambda I + K~ is kept in
//    FP64 (leaf blocks and U blocks evaluated once in FP64 and stored, P in FP64),
//    and the solve refines w += Solve32(u - (lambda I + K~) w) until the relative
//    residual of every column is below the target.  K~ is the one defined by the
//    skeletons and P this factorization chose, so the FP32 factorization is an
//    approximate inverse of exactly the operator the residual uses.
#include <algorithm>
#include <chrono>
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
};

struct Node {
  int off = 0, size = 0;
  int s = 0;          // rank (skeleton count); 0 for the root
  int ncols = 0;      // ID columns: size (leaf) or s_l + s_r
  int nsamp = 0;
  int64_t samp_off = 0, P_off = 0, W_off = 0, LU_off = 0, Z_off = 0, Zpiv_off = 0, CL_off = 0,
          CR_off = 0;
};

struct Stats {
  double t_tree = 0, t_knn = 0, t_skel = 0, t_leaf_lu = 0, t_factor_levels = 0, t_factor = 0;
  double t_solve = 0, t_apply = 0;
  int knn_fallback = 0;
  int64_t bytes_W = 0, bytes_LU = 0, bytes_P = 0, bytes_operator = 0;
  std::vector<double> refine_hist;
  int refine_sweeps = 0;
};

template <typename T>
struct RootBlock {
  int uid;
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
template <typename T>
double getrf_flops(const std::vector<LuDescT<T>>& v) {
  double f = 0;
  for (const auto& d : v) f += 2.0 / 3.0 * d.n * (double)d.n * d.n;
  return f;
}
template <typename T>
void add_gemm(std::vector<GemmDescT<T>>& g, const T* A, int lda, const T* B, int ldb, T* C,
              int ldc, int M, int Ncol, int K, double alpha, double beta) {
  if (M <= 0 || Ncol <= 0) return;
  g.push_back(GemmDescT<T>{A, B, C, M, Ncol, K, lda, ldb, ldc, alpha, beta});
}

// Tile list of one grouped launch: 256 x 16 tiles when no problem has more than 16
// columns (right-hand-side blocks of a solve), 64 x 64 tiles otherwise.
template <typename T>
GemmShape make_tiles(const std::vector<GemmDescT<T>>& g, std::vector<GemmTile>& t) {
  int maxn = 0;
  for (const auto& d : g) maxn = std::max(maxn, d.N);
  const GemmShape shape = maxn <= 16 ? GEMM_SKINNY : GEMM_SQUARE;
  const int tm_ = gemm_tile_m(shape), tn_ = gemm_tile_n(shape);
  t.clear();
  for (int idx = 0; idx < (int)g.size(); ++idx)
    for (int tn = 0; tn < (g[idx].N + tn_ - 1) / tn_; ++tn)
      for (int tm = 0; tm < (g[idx].M + tm_ - 1) / tm_; ++tm) t.push_back(GemmTile{idx, tm, tn});
  return shape;
}

class Solver {
 public:
  cudaStream_t st = nullptr;
  Options opt;
  Stats stats;
  bool factored = false;
  int prec = PREC_FP64;  // precision of the current factorization
  int N = 0, d = 0, L = 0, m_max = 0, s_max = 0, kappa = 0;
  double h = 0, lam = 0, tol = 0;
  std::vector<std::vector<int>> level_off;
  std::vector<Node> nd;  // heap ids 1 .. 2^(L+1) - 1
  DevBuf X, Xp, perm, iperm, split_dim, knn, knn_pos, samp, ranks, skel, piv_ws, A_ws, status,
      arena_dev, level_off_dev, tbuf, vbuf, vbuf32, ubuf, rbuf, wt, io, normbuf;
  // factorization storage: FP64 (plain) and FP32 (mixed)
  DevBuf LU, LUpiv, Wb, Zb, Zpiv, Cb, LU32, Wb32, Zb32, Cb32, tbuf32;
  // FP64 operator blocks kept by the mixed form: leaf blocks lambda I + K_aa and U blocks
  DevBuf Kleaf, Ustore;
  std::vector<std::unique_ptr<DevBuf>> Pl, Pl32;  // nested P per level (FP64; FP32 copy)
  TreeScratch tree_s;
  KnnScratch knn_s;
  SampleScratch samp_s;
  Arena arena;

  int uid(int l, int i) const { return (1 << l) + i; }
  int level_of(int u) const {
    int l = 0;
    while ((2 << l) <= u) ++l;
    return l;
  }

  // typed views of the factorization storage
  template <typename T>
  T* luP() { return std::is_same<T, float>::value ? (T*)LU32.p : (T*)LU.p; }
  template <typename T>
  T* wP() { return std::is_same<T, float>::value ? (T*)Wb32.p : (T*)Wb.p; }
  template <typename T>
  T* zP() { return std::is_same<T, float>::value ? (T*)Zb32.p : (T*)Zb.p; }
  template <typename T>
  T* cP() { return std::is_same<T, float>::value ? (T*)Cb32.p : (T*)Cb.p; }
  template <typename T>
  T* pP(int l) { return std::is_same<T, float>::value ? (T*)Pl32[l]->p : (T*)Pl[l]->p; }
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
  template <typename T>
  void run_gemms(const std::vector<GemmDescT<T>>& g) {
    if (g.empty()) return;
    std::vector<GemmTile> t;
    const GemmShape shape = make_tiles(g, t);
    arena.clear();
    size_t og = arena.push(g), ot = arena.push(t);
    char* base = upload_arena();
    prof().flops[pk_of<T>(PK_GEMM)] += gemm_flops(g);
    gemm_grouped((const GemmDescT<T>*)(base + og), (const GemmTile*)(base + ot), (int)t.size(),
                 shape, st);
  }

  // ------------------------------------------------------------- forest solve
  // Applies (lambda I + K~_cc)^{-1} to the block of every root c at level r, in
  // place, with the factorization stored in precision T.  Writes P_c v_c to
  // roots[].t_out when given.
  template <typename T>
  void forest_solve(int r, const std::vector<RootBlock<T>>& roots) {
    const bool need_t = !roots.empty() && roots[0].t_out != nullptr;
    std::vector<int> root_of(nd.size(), -1);
    std::vector<T*> Vp(nd.size(), nullptr);
    int max_nc = 0;
    for (size_t q = 0; q < roots.size(); ++q) {
      max_nc = std::max(max_nc, roots[q].nc);
      const int c = roots[q].uid;
      const int lc = level_of(c);
      for (int l = lc; l <= L; ++l) {
        int first = c << (l - lc), cnt = 1 << (l - lc);
        for (int u = first; u < first + cnt; ++u) {
          root_of[u] = (int)q;
          Vp[u] = roots[q].V + (nd[u].off - nd[c].off);
        }
      }
    }
    // T and Y scratch for internal forest nodes
    std::vector<int64_t> Toff(nd.size(), -1);
    int64_t tsz = 0;
    for (int l = r; l < L; ++l)
      for (int i = 0; i < (1 << l); ++i) {
        int u = uid(l, i);
        if (root_of[u] < 0) continue;
        int n2 = nd[2 * u].s + nd[2 * u + 1].s;
        Toff[u] = tsz;
        tsz += 2 * (int64_t)n2 * roots[root_of[u]].nc;
      }
    T* Tb = tB<T>().template ensure_n<T>(std::max<int64_t>(tsz, 1));
    auto Tp = [&](int u) { return Tb + Toff[u]; };
    auto Yp = [&](int u) {
      int n2 = nd[2 * u].s + nd[2 * u + 1].s;
      return Tb + Toff[u] + (int64_t)n2 * roots[root_of[u]].nc;
    };
    auto ldV = [&](int u) { return roots[root_of[u]].ld; };
    auto ncV = [&](int u) { return roots[root_of[u]].nc; };

    // 1. leaf LU solves
    {
      std::vector<LuSolveDescT<T>> ds;
      for (int i = 0; i < (1 << L); ++i) {
        int u = uid(L, i);
        if (root_of[u] < 0) continue;
        ds.push_back(LuSolveDescT<T>{luP<T>() + nd[u].LU_off, LUpiv.as<int>() + (int64_t)i * m_max,
                                     Vp[u], nd[u].size, nd[u].size, ldV(u), ncV(u)});
      }
      arena.clear();
      size_t o = arena.push(ds);
      char* base = upload_arena();
      prof().flops[pk_of<T>(PK_GETRS)] += getrs_flops(ds);
      getrs_batched((const LuSolveDescT<T>*)(base + o), (int)ds.size(), m_max, max_nc, st);
    }
    if (r == L) {
      if (need_t) {
        std::vector<GemmDescT<T>> g;
        for (const auto& rb : roots) {
          const Node& c = nd[rb.uid];
          add_gemm<T>(g, pP<T>(L) + c.P_off, c.s, rb.V, rb.ld, rb.t_out, rb.t_ld, c.s, rb.nc,
                      c.size, 1.0, 0.0);
        }
        run_gemms(g);
      }
      return;
    }
    // 2. leaf t = P v into the parent's T
    {
      std::vector<GemmDescT<T>> g;
      for (int i = 0; i < (1 << L); ++i) {
        int u = uid(L, i);
        if (root_of[u] < 0) continue;
        int par = u >> 1;
        int n2 = nd[2 * par].s + nd[2 * par + 1].s;
        int rowoff = (u & 1) ? nd[2 * par].s : 0;
        add_gemm<T>(g, pP<T>(L) + nd[u].P_off, nd[u].s, Vp[u], ldV(u), Tp(par) + rowoff, n2,
                    nd[u].s, ncV(u), nd[u].size, 1.0, 0.0);
      }
      run_gemms(g);
    }
    // 3. levels L-1 .. r
    for (int j = L - 1; j >= r; --j) {
      std::vector<CopyDescT<T>> cp;
      std::vector<LuSolveDescT<T>> zs;
      std::vector<GemmDescT<T>> g1, g2;
      std::vector<GemmTile> t1, t2;
      int64_t max_cp = 0;
      int max_n2 = 0;
      for (int i = 0; i < (1 << j); ++i) {
        int b = uid(j, i);
        if (root_of[b] < 0) continue;
        int a = 2 * b, c = 2 * b + 1;  // children: a left, c right
        int sa = nd[a].s, sc = nd[c].s, n2 = sa + sc, nc = ncV(b);
        max_n2 = std::max(max_n2, n2);
        max_cp = std::max<int64_t>(max_cp, (int64_t)n2 * nc);
        cp.push_back(CopyDescT<T>{Tp(b), Yp(b), n2, nc, n2, n2});
        zs.push_back(LuSolveDescT<T>{zP<T>() + nd[b].Z_off, Zpiv.as<int>() + nd[b].Zpiv_off, Yp(b),
                                     n2, n2, n2, nc});
        const T* W = wP<T>();
        // v_a -= W_{a c~} y1 (y1 = Y[sa : n2]);  v_c -= W_{c a~} y2 (y2 = Y[0 : sa])
        add_gemm<T>(g1, W + nd[a].W_off, nd[a].size, Yp(b) + sa, n2, Vp[a], ldV(b), nd[a].size,
                    nc, sc, -1.0, 1.0);
        add_gemm<T>(g1, W + nd[c].W_off, nd[c].size, Yp(b), n2, Vp[c], ldV(b), nd[c].size, nc,
                    sa, -1.0, 1.0);
        const bool carry = (j > r) || need_t;
        if (carry) {
          const T* C = cP<T>();
          add_gemm<T>(g1, C + nd[b].CL_off, sa, Yp(b) + sa, n2, Tp(b), n2, sa, nc, sc, -1.0, 1.0);
          add_gemm<T>(g1, C + nd[b].CR_off, sc, Yp(b), n2, Tp(b) + sa, n2, sc, nc, sa, -1.0, 1.0);
          T* dst;
          int ldd;
          if (j > r) {
            int par = b >> 1;
            int pn2 = nd[2 * par].s + nd[2 * par + 1].s;
            dst = Tp(par) + ((b & 1) ? nd[2 * par].s : 0);
            ldd = pn2;
          } else {
            dst = roots[root_of[b]].t_out;
            ldd = roots[root_of[b]].t_ld;
          }
          add_gemm<T>(g2, pP<T>(j) + nd[b].P_off, nd[b].s, Tp(b), n2, dst, ldd, nd[b].s, nc, n2,
                      1.0, 0.0);
        }
      }
      const GemmShape sh1 = make_tiles(g1, t1), sh2 = make_tiles(g2, t2);
      arena.clear();
      size_t ocp = arena.push(cp), ozs = arena.push(zs), og1 = arena.push(g1), ot1 = arena.push(t1),
             og2 = arena.push(g2), ot2 = arena.push(t2);
      char* base = upload_arena();
      prof().flops[pk_of<T>(PK_GETRS)] += getrs_flops(zs);
      prof().flops[pk_of<T>(PK_GEMM)] += gemm_flops(g1) + gemm_flops(g2);
      copy_batched((const CopyDescT<T>*)(base + ocp), (int)cp.size(), max_cp, st);
      getrs_batched((const LuSolveDescT<T>*)(base + ozs), (int)zs.size(), max_n2, max_nc, st);
      gemm_grouped((const GemmDescT<T>*)(base + og1), (const GemmTile*)(base + ot1), (int)t1.size(),
                   sh1, st);
      gemm_grouped((const GemmDescT<T>*)(base + og2), (const GemmTile*)(base + ot2), (int)t2.size(),
                   sh2, st);
    }
  }

  // ------------------------------------------------------------- factorization
  void factor(const double* points, bool on_device, int64_t N_, int d_, double h_, double lam_,
              int leaf_m, int s_max_, double tol_) {
    factored = false;
    if (N_ < 2 || N_ > (int64_t)1 << 30) throw Error(IASKIT_ERR_ARG, "N must be in [2, 2^30]");
    if (d_ < 1) throw Error(IASKIT_ERR_ARG, "d must be >= 1");
    if (!(h_ > 0.0) || !std::isfinite(h_)) throw Error(IASKIT_ERR_ARG, "h must be > 0");
    if (!(lam_ >= 0.0) || !std::isfinite(lam_)) throw Error(IASKIT_ERR_ARG, "lambda must be >= 0");
    if (leaf_m < 2) throw Error(IASKIT_ERR_ARG, "leaf_m must be >= 2");
    if (s_max_ < 1) throw Error(IASKIT_ERR_ARG, "s_max must be >= 1");
    if (!points) throw Error(IASKIT_ERR_ARG, "points is null");
    stats = Stats{};
    N = (int)N_;
    d = d_;
    h = h_;
    lam = lam_;
    s_max = s_max_;
    tol = tol_;
    prec = opt.precision;
    kappa = std::min(opt.kappa, N - 1);
    const double t0 = now_ms();
    // tree shape (data independent)
    L = 0;
    while ((N + (1 << L) - 1) / (1 << L) > leaf_m) ++L;
    if (L > 24) throw Error(IASKIT_ERR_UNSUPPORTED, "tree deeper than 24 levels");
    level_off.assign(L + 1, {});
    nd.assign((size_t)2 << L, Node{});
    nd[1].off = 0;
    nd[1].size = N;
    for (int l = 0; l < L; ++l)
      for (int i = 0; i < (1 << l); ++i) {
        Node& p = nd[uid(l, i)];
        Node& a = nd[2 * uid(l, i)];
        Node& b = nd[2 * uid(l, i) + 1];
        a.off = p.off;
        a.size = p.size / 2;
        b.off = p.off + a.size;
        b.size = p.size - a.size;
      }
    for (int l = 0; l <= L; ++l) {
      level_off[l].resize((1 << l) + 1);
      for (int i = 0; i < (1 << l); ++i) level_off[l][i] = nd[uid(l, i)].off;
      level_off[l][1 << l] = N;
    }
    m_max = 0;
    for (int i = 0; i < (1 << L); ++i) m_max = std::max(m_max, nd[uid(L, i)].size);
    if (m_max > 1536) throw Error(IASKIT_ERR_UNSUPPORTED, "leaf size above 1536");
    if (2 * s_max > 1536 && L > 0) throw Error(IASKIT_ERR_UNSUPPORTED, "s_max above 768");

    status.ensure_n<int>(1);
    IA_CUDA(cudaMemsetAsync(status.as<int>(), 0, sizeof(int), st));
    double* Xd = X.ensure_n<double>((size_t)N * d);
    IA_CUDA(cudaMemcpyAsync(Xd, points, (size_t)N * d * sizeof(double),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    check_finite(Xd, (int64_t)N * d, status.as<int>(), st);
    raise_status(read_status_and_clear());

    // a1: tree
    int* pm = perm.ensure_n<int>(N);
    build_tree(Xd, N, d, L, level_off, pm, split_dim.ensure_n<int>((size_t)1 << std::max(L, 1)),
               tree_s, st);
    permute_points(Xd, pm, N, d, iperm.ensure_n<int>(N), Xp.ensure_n<double>((size_t)N * d), st);
    IA_CUDA(cudaStreamSynchronize(st));
    const double t1 = now_ms();
    stats.t_tree = t1 - t0;

    Pl.clear();
    Pl32.clear();
    for (int l = 0; l <= L; ++l) {
      Pl.emplace_back(new DevBuf());
      Pl32.emplace_back(new DevBuf());
    }
    if (L > 0) {
      // a2: kNN
      stats.knn_fallback = knn_bruteforce(Xd, N, d, kappa, knn.ensure_n<int>((size_t)N * kappa), knn_s, st);
      IA_CUDA(cudaStreamSynchronize(st));
      const double t2 = now_ms();
      stats.t_knn = t2 - t1;
      if (prec == PREC_MIXED) skeletonize<float>();
      else skeletonize<double>();
      IA_CUDA(cudaStreamSynchronize(st));
      stats.t_skel = now_ms() - t2;
    }
    const double t3 = now_ms();
    leaf_lu();
    raise_status(read_status_and_clear());
    const double t4 = now_ms();
    stats.t_leaf_lu = t4 - t3;
    if (prec == PREC_MIXED) factor_levels<float>();
    else factor_levels<double>();
    raise_status(read_status_and_clear());
    stats.t_factor_levels = now_ms() - t4;
    stats.t_factor = now_ms() - t0;
    prof().resolve();
    factored = true;
  }

  // a3 + a4 + a5: skeletons, levels L .. 1; TS is the precision of the sampled
  // blocks and of the Householder updates (pivot norms are FP64 in both).
  template <typename TS>
  void skeletonize() {
    int* kp = knn_pos.ensure_n<int>((size_t)N * kappa);
    knn_to_positions(knn.as<int>(), perm.as<int>(), iperm.as<int>(), N, kappa, kp, st);
    const int samp_cap = opt.samp_factor * s_max;
    int64_t tot = 0;
    for (int l = 1; l <= L; ++l)
      for (int i = 0; i < (1 << l); ++i) {
        Node& n = nd[uid(l, i)];
        n.nsamp = std::min(samp_cap, N - n.size);
        n.samp_off = tot;
        tot += n.nsamp;
      }
    int* sp = samp.ensure_n<int>(tot);
    int* rk = ranks.ensure_n<int>(nd.size());
    IA_CUDA(cudaMemsetAsync(rk, 0, nd.size() * sizeof(int), st));
    int* sk = skel.ensure_n<int>(nd.size() * (size_t)s_max);
    for (int l = L; l >= 1; --l) {
      const int nn = 1 << l;
      // sampling
      std::vector<int> so(nn);
      for (int i = 0; i < nn; ++i) so[i] = (int)nd[uid(l, i)].samp_off;
      int* od = level_off_dev.ensure_n<int>(nn + 1 + nn);
      h2d(od, level_off[l].data(), nn + 1, st);
      h2d(od + nn + 1, so.data(), nn, st);
      sample_level(kp, N, kappa, l, od, level_off[l], samp_cap, od + nn + 1, opt.seed, sp,
                   status.as<int>(), samp_s, st);
      // sampled blocks
      int64_t asz = 0, pvsz = 0, max_e = 0;
      int max_r = 0, max_c = 0;
      std::vector<int64_t> aoff(nn), poff(nn);
      for (int i = 0; i < nn; ++i) {
        Node& n = nd[uid(l, i)];
        n.ncols = (l == L) ? n.size : nd[2 * uid(l, i)].s + nd[2 * uid(l, i) + 1].s;
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
      std::vector<KDescT<TS>> kd(nn);
      std::vector<CpqrDescT<TS>> qd(nn);
      for (int i = 0; i < nn; ++i) {
        const int u = uid(l, i);
        Node& n = nd[u];
        KDescT<TS> k{};
        k.rows = sp + n.samp_off;
        k.nrows = n.nsamp;
        k.out = A + aoff[i];
        k.ld = n.nsamp;
        k.ncols = n.ncols;
        k.diag = 0.0;
        if (l == L) {
          k.col0 = n.off;
        } else {
          k.colsA = sk + (size_t)(2 * u) * s_max;
          k.nA = nd[2 * u].s;
          k.colsB = sk + (size_t)(2 * u + 1) * s_max;
        }
        kd[i] = k;
        qd[i] = CpqrDescT<TS>{A + aoff[i], pv + poff[i], rk + u, n.nsamp, n.nsamp, n.ncols};
      }
      arena.clear();
      size_t ok = arena.push(kd), oq = arena.push(qd);
      char* base = upload_arena();
      kernel_blocks<TS>(Xp.as<double>(), d, h, (const KDescT<TS>*)(base + ok), nn, max_e, st);
      cpqr_id<TS>((const CpqrDescT<TS>*)(base + oq), nn, max_r, max_c, s_max, tol, st);
      // ranks of this level
      std::vector<int> rh(nn);
      d2h(rh.data(), rk + uid(l, 0), nn, st);
      IA_CUDA(cudaStreamSynchronize(st));
      raise_status(read_status_and_clear());
      int64_t psz = 0;
      double qr_flops = 0;
      for (int i = 0; i < nn; ++i) {
        Node& n = nd[uid(l, i)];
        n.s = rh[i];
        n.P_off = psz;
        psz += (int64_t)n.s * n.ncols;
        // Householder update (dot + axpy) and norm recomputation per step, then R11^{-1} R12
        for (int k = 0; k < n.s; ++k) qr_flops += 6.0 * (n.nsamp - k) * (double)(n.ncols - k);
        qr_flops += (double)n.s * n.s * (n.ncols - n.s);
      }
      prof().flops[pk_of<TS>(PK_CPQR)] += qr_flops;
      double* P = Pl[l]->ensure_n<double>(psz);
      std::vector<PDescT<TS>> pd(nn);
      for (int i = 0; i < nn; ++i) {
        const int u = uid(l, i);
        Node& n = nd[u];
        PDescT<TS> p{};
        p.A = A + aoff[i];
        p.piv = pv + poff[i];
        p.P = P + n.P_off;
        p.skel = sk + (size_t)u * s_max;
        p.ld = n.nsamp;
        p.ncols = n.ncols;
        p.s = n.s;
        if (l == L) {
          p.col0 = n.off;
        } else {
          p.colsA = sk + (size_t)(2 * u) * s_max;
          p.nA = nd[2 * u].s;
          p.colsB = sk + (size_t)(2 * u + 1) * s_max;
        }
        pd[i] = p;
      }
      arena.clear();
      size_t op = arena.push(pd);
      base = upload_arena();
      assemble_P<TS>((const PDescT<TS>*)(base + op), nn, max_c, st);
      if (prec == PREC_MIXED) convert_d2f(P, Pl32[l]->ensure_n<float>(psz), psz, st);
      stats.bytes_P += psz * 8;
    }
  }

  // a4 + a6: leaf LU of lambda I + K_aa.  Mixed: the FP64 blocks are kept for the
  // operator and their FP32 rounding is factored.
  void leaf_lu() {
    const int nl = 1 << L;
    int64_t tot = 0;
    for (int i = 0; i < nl; ++i) {
      Node& n = nd[uid(L, i)];
      n.LU_off = tot;
      tot += (int64_t)n.size * n.size;
    }
    const bool mixed = prec == PREC_MIXED;
    double* blocks = mixed ? Kleaf.ensure_n<double>(tot) : LU.ensure_n<double>(tot);
    int* lp = LUpiv.ensure_n<int>((size_t)nl * m_max);
    std::vector<KDesc> kd(nl);
    for (int i = 0; i < nl; ++i) {
      const Node& n = nd[uid(L, i)];
      KDesc k{};
      k.row0 = n.off;
      k.nrows = n.size;
      k.col0 = n.off;
      k.ncols = n.size;
      k.out = blocks + n.LU_off;
      k.ld = n.size;
      k.diag = lam;
      kd[i] = k;
    }
    arena.clear();
    size_t ok = arena.push(kd);
    char* base = upload_arena();
    kernel_blocks<double>(Xp.as<double>(), d, h, (const KDesc*)(base + ok), nl,
                          (int64_t)m_max * m_max, st);
    if (mixed) {
      float* lu = LU32.ensure_n<float>(tot);
      convert_d2f(blocks, lu, tot, st);
      std::vector<LuDescT<float>> ld(nl);
      for (int i = 0; i < nl; ++i) {
        const Node& n = nd[uid(L, i)];
        ld[i] = LuDescT<float>{lu + n.LU_off, lp + (int64_t)i * m_max, n.size, n.size};
      }
      arena.clear();
      size_t ol = arena.push(ld);
      base = upload_arena();
      prof().flops[PK_GETRF32] += getrf_flops(ld);
      getrf_batched<float>((const LuDescT<float>*)(base + ol), nl, m_max, status.as<int>(), st);
      stats.bytes_operator += tot * 8;
      stats.bytes_LU = tot * 4;
    } else {
      std::vector<LuDesc> ld(nl);
      for (int i = 0; i < nl; ++i) {
        const Node& n = nd[uid(L, i)];
        ld[i] = LuDesc{blocks + n.LU_off, lp + (int64_t)i * m_max, n.size, n.size};
      }
      arena.clear();
      size_t ol = arena.push(ld);
      base = upload_arena();
      prof().flops[PK_GETRF] += getrf_flops(ld);
      getrf_batched<double>((const LuDesc*)(base + ol), nl, m_max, status.as<int>(), st);
      stats.bytes_LU = tot * 8;
    }
  }

  // a7 + a8: W and Z, levels L-1 .. 0, factorization stored in precision T
  template <typename T>
  void factor_levels() {
    if (L == 0) return;
    const bool mixed = std::is_same<T, float>::value;
    int64_t wsz = 0, zsz = 0, zp = 0, csz = 0;
    for (int l = 1; l <= L; ++l)
      for (int i = 0; i < (1 << l); ++i) {
        int u = uid(l, i);
        Node& n = nd[u];
        n.W_off = wsz;
        wsz += (int64_t)n.size * nd[u ^ 1].s;
      }
    for (int l = 0; l < L; ++l)
      for (int i = 0; i < (1 << l); ++i) {
        int u = uid(l, i);
        Node& n = nd[u];
        int sa = nd[2 * u].s, sb = nd[2 * u + 1].s;
        n.Z_off = zsz;
        zsz += (int64_t)(sa + sb) * (sa + sb);
        n.Zpiv_off = zp;
        zp += sa + sb;
        n.CL_off = csz;
        csz += (int64_t)sa * sb;
        n.CR_off = csz;
        csz += (int64_t)sb * sa;
      }
    const double bytes = (double)(wsz + zsz + csz) * sizeof(T) + (mixed ? (double)wsz * 8 : 0.0);
    if (opt.mem_cap_gb > 0 && bytes > opt.mem_cap_gb * 1e9)
      throw Error(IASKIT_ERR_NOMEM, "factorization exceeds mem_cap_gb");
    T* W = (mixed ? Wb32 : Wb).template ensure_n<T>(wsz);
    double* U64 = mixed ? Ustore.ensure_n<double>(wsz) : (double*)W;
    (mixed ? Zb32 : Zb).template ensure_n<T>(zsz);
    Zpiv.ensure_n<int>(zp);
    (mixed ? Cb32 : Cb).template ensure_n<T>(csz);
    stats.bytes_W = wsz * (int64_t)sizeof(T);
    if (mixed) stats.bytes_operator += wsz * 8;
    int* sk = skel.as<int>();
    for (int l = L - 1; l >= 0; --l) {
      const int nn = 1 << l;
      // U blocks of the children of every node of level l (FP64)
      std::vector<KDesc> kd;
      int64_t max_e = 0, lo = INT64_MAX, hi = 0;
      for (int i = 0; i < 2 * nn; ++i) {
        int c = uid(l + 1, i);
        const Node& n = nd[c];
        KDesc k{};
        k.row0 = n.off;
        k.nrows = n.size;
        k.colsA = sk + (size_t)(c ^ 1) * s_max;
        k.nA = nd[c ^ 1].s;
        k.ncols = nd[c ^ 1].s;
        k.out = U64 + n.W_off;
        k.ld = n.size;
        k.diag = 0.0;
        kd.push_back(k);
        max_e = std::max<int64_t>(max_e, (int64_t)n.size * k.ncols);
        lo = std::min<int64_t>(lo, n.W_off);
        hi = std::max<int64_t>(hi, n.W_off + (int64_t)n.size * k.ncols);
      }
      arena.clear();
      size_t ok = arena.push(kd);
      char* base = upload_arena();
      kernel_blocks<double>(Xp.as<double>(), d, h, (const KDesc*)(base + ok), (int)kd.size(), max_e, st);
      if (mixed) convert_d2f(U64 + lo, (float*)W + lo, hi - lo, st);
      // W = Solve(child, U) for all children at once; C blocks come back as P_c W_c
      std::vector<RootBlock<T>> rb;
      T* C = cP<T>();
      for (int i = 0; i < 2 * nn; ++i) {
        int c = uid(l + 1, i);
        int par = c >> 1;
        const Node& n = nd[c];
        // left child: C_l = P_l W_{l r~} (s_l x s_r); right child: C_r = P_r W_{r l~}
        T* tout = C + ((c & 1) == 0 ? nd[par].CL_off : nd[par].CR_off);
        rb.push_back(RootBlock<T>{c, W + n.W_off, n.size, nd[c ^ 1].s, tout, n.s});
      }
      forest_solve<T>(l + 1, rb);
      // reduced systems Z'' = [[I, C_l], [C_r, I]] and their LU
      std::vector<ZDescT<T>> zd;
      std::vector<LuDescT<T>> ld;
      int64_t max_z = 0;
      int max_n = 0;
      for (int i = 0; i < nn; ++i) {
        int u = uid(l, i);
        int sa = nd[2 * u].s, sb = nd[2 * u + 1].s;
        zd.push_back(ZDescT<T>{C + nd[u].CL_off, C + nd[u].CR_off, zP<T>() + nd[u].Z_off, sa, sb});
        ld.push_back(LuDescT<T>{zP<T>() + nd[u].Z_off, Zpiv.as<int>() + nd[u].Zpiv_off, sa + sb, sa + sb});
        max_z = std::max<int64_t>(max_z, (int64_t)(sa + sb) * (sa + sb));
        max_n = std::max(max_n, sa + sb);
      }
      arena.clear();
      size_t oz = arena.push(zd), ol = arena.push(ld);
      base = upload_arena();
      form_Z<T>((const ZDescT<T>*)(base + oz), nn, max_z, st);
      prof().flops[pk_of<T>(PK_GETRF)] += getrf_flops(ld);
      getrf_batched<T>((const LuDescT<T>*)(base + ol), nn, max_n, status.as<int>(), st);
    }
  }

  // ------------------------------------------------------------------ solve
  void solve_device(double* rhs, int nrhs) {
    if (!factored) throw Error(IASKIT_ERR_NOT_FACTORED, "no factorization");
    if (nrhs < 1 || (int64_t)N * nrhs > ((int64_t)1 << 31)) throw Error(IASKIT_ERR_ARG, "bad nrhs");
    const double t0 = now_ms();
    check_finite(rhs, (int64_t)N * nrhs, status.as<int>(), st);
    raise_status(read_status_and_clear());
    stats.refine_hist.clear();
    stats.refine_sweeps = 0;
    const int sweeps = opt.refine > 0 ? opt.refine : (prec == PREC_MIXED ? 50 : 0);
    if (sweeps <= 0) {
      plain_solve(rhs, nrhs, rhs);
    } else {
      refine_solve(rhs, nrhs, sweeps);
    }
    IA_CUDA(cudaStreamSynchronize(st));
    prof().resolve();
    stats.t_solve = now_ms() - t0;
  }

  // out <- (lambda I + K~)^{-1} in with the stored factorization (ORIGINAL order,
  // N x nrhs, ld N); in and out may alias.
  void plain_solve(const double* in, int nrhs, double* out) {
    const size_t n = (size_t)N * nrhs;
    double* V = vbuf.ensure_n<double>(n);
    permute_rows<double>(in, N, V, N, perm.as<int>(), N, nrhs, false, st);
    if (prec == PREC_MIXED) {
      float* V32 = vbuf32.ensure_n<float>(n);
      convert_d2f(V, V32, (int64_t)n, st);
      std::vector<RootBlock<float>> rb{RootBlock<float>{1, V32, N, nrhs, nullptr, 0}};
      forest_solve<float>(0, rb);
      convert_f2d(V32, V, (int64_t)n, st);
    } else {
      std::vector<RootBlock<double>> rb{RootBlock<double>{1, V, N, nrhs, nullptr, 0}};
      forest_solve<double>(0, rb);
    }
    permute_rows<double>(V, N, out, N, perm.as<int>(), N, nrhs, true, st);
  }

  // Iterative refinement against the FP64 operator: w <- w + Solve(u - A w).
  void refine_solve(double* rhs, int nrhs, int sweeps) {
    const size_t n = (size_t)N * nrhs;
    double* u = rbuf.ensure_n<double>(2 * n);  // u copy, residual
    double* r = u + n;
    IA_CUDA(cudaMemcpyAsync(u, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    std::vector<double> un(nrhs), rn(nrhs);
    column_norms(u, nrhs, un);
    plain_solve(u, nrhs, rhs);
    auto worst_residual = [&]() {
      apply_device(rhs, r, nrhs);        // r = A w
      axpby(u, r, n);                    // r = u - A w
      column_norms(r, nrhs, rn);
      double worst = 0;
      for (int c = 0; c < nrhs; ++c) worst = std::max(worst, un[c] > 0 ? rn[c] / un[c] : rn[c]);
      stats.refine_hist.push_back(worst);
      return worst;
    };
    for (int it = 0; it < sweeps; ++it) {
      if (worst_residual() <= opt.refine_tol) return;
      plain_solve(r, nrhs, r);           // delta
      add_inplace(rhs, r, n);            // w += delta
      stats.refine_sweeps = it + 1;
    }
    if (worst_residual() > opt.refine_tol)
      throw Error(IASKIT_ERR_NOT_CONVERGED, "refinement did not converge");
  }

  void column_norms(const double* x, int nrhs, std::vector<double>& out);
  void axpby(const double* u, double* r, size_t n);
  void add_inplace(double* w, const double* dlt, size_t n);
  void scale_copy(const double* x, double* y, double a, size_t n);

  // ------------------------------------------------------- hierarchical apply
  // u = (lambda I + K~) w, ORIGINAL order, device pointers.  Skeletonize (w~ = P w
  // up the tree) then Evaluate (u_c += K_{c s~} w~_s for the sibling s of every
  // node c, and the leaf blocks).  The plain form recomputes the kernel entries in
  // FP64; the mixed form multiplies the FP64 blocks it stored.
  void apply_device(const double* w, double* u, int nrhs) {
    if (!factored) throw Error(IASKIT_ERR_NOT_FACTORED, "no factorization");
    if (nrhs < 1) throw Error(IASKIT_ERR_ARG, "bad nrhs");
    const double t0 = now_ms();
    const bool stored = prec == PREC_MIXED;
    const size_t n = (size_t)N * nrhs;
    double* Wp = ubuf.ensure_n<double>(2 * n);
    double* Up = Wp + n;
    permute_rows<double>(w, N, Wp, N, perm.as<int>(), N, nrhs, false, st);
    if (stored) IA_CUDA(cudaMemsetAsync(Up, 0, n * sizeof(double), st));
    else scale_copy(Wp, Up, lam, n);
    std::vector<int64_t> woff(nd.size(), 0);
    int64_t tot = 0;
    for (int l = 0; l < L; ++l)
      for (int i = 0; i < (1 << l); ++i) {
        int u_ = uid(l, i);
        woff[u_] = tot;
        tot += (int64_t)(nd[2 * u_].s + nd[2 * u_ + 1].s) * nrhs;
      }
    double* WT = wt.ensure_n<double>(std::max<int64_t>(tot, 1));
    auto n2 = [&](int u_) { return nd[2 * u_].s + nd[2 * u_ + 1].s; };
    auto wsib = [&](int c) {  // w~ of the sibling of c, inside the parent's [w~_a; w~_b]
      int par = c >> 1, sib = c ^ 1;
      return WT + woff[par] + ((sib & 1) ? nd[2 * par].s : 0);
    };
    if (L > 0) {
      std::vector<GemmDesc> g;
      for (int i = 0; i < (1 << L); ++i) {
        int u_ = uid(L, i), par = u_ >> 1;
        add_gemm<double>(g, Pl[L]->as<double>() + nd[u_].P_off, nd[u_].s, Wp + nd[u_].off, N,
                         WT + woff[par] + ((u_ & 1) ? nd[2 * par].s : 0), n2(par), nd[u_].s, nrhs,
                         nd[u_].size, 1.0, 0.0);
      }
      run_gemms(g);
      for (int l = L - 1; l >= 1; --l) {
        g.clear();
        for (int i = 0; i < (1 << l); ++i) {
          int u_ = uid(l, i), par = u_ >> 1;
          add_gemm<double>(g, Pl[l]->as<double>() + nd[u_].P_off, nd[u_].s, WT + woff[u_],
                           n2(u_), WT + woff[par] + ((u_ & 1) ? nd[2 * par].s : 0), n2(par),
                           nd[u_].s, nrhs, n2(u_), 1.0, 0.0);
        }
        run_gemms(g);
      }
    }
    // Evaluate: one launch per level keeps the rows written by a launch disjoint
    int* sk = skel.as<int>();
    for (int l = 1; l <= L + 1; ++l) {
      const bool leaves = l == L + 1;
      const int lev = leaves ? L : l;
      if (stored) {
        std::vector<GemmDesc> g;
        for (int i = 0; i < (1 << lev); ++i) {
          int c = uid(lev, i);
          if (leaves)
            add_gemm<double>(g, Kleaf.as<double>() + nd[c].LU_off, nd[c].size, Wp + nd[c].off, N,
                             Up + nd[c].off, N, nd[c].size, nrhs, nd[c].size, 1.0, 1.0);
          else
            add_gemm<double>(g, Ustore.as<double>() + nd[c].W_off, nd[c].size, wsib(c),
                             n2(c >> 1), Up + nd[c].off, N, nd[c].size, nrhs, nd[c ^ 1].s, 1.0, 1.0);
        }
        run_gemms(g);
      } else {
        std::vector<KMatvecDesc> md;
        int max_rows = 0;
        for (int i = 0; i < (1 << lev); ++i) {
          int c = uid(lev, i);
          if (leaves)
            md.push_back(KMatvecDesc{nullptr, Wp + nd[c].off, Up + nd[c].off, nd[c].off, nd[c].size,
                                     nd[c].off, nd[c].size, N, N});
          else
            md.push_back(KMatvecDesc{sk + (size_t)(c ^ 1) * s_max, wsib(c), Up + nd[c].off, nd[c].off,
                                     nd[c].size, 0, nd[c ^ 1].s, n2(c >> 1), N});
          max_rows = std::max(max_rows, nd[c].size);
        }
        arena.clear();
        size_t om = arena.push(md);
        char* base = upload_arena();
        kernel_matvec(Xp.as<double>(), d, h, nrhs, (const KMatvecDesc*)(base + om), (int)md.size(),
                      max_rows, st);
      }
    }
    permute_rows<double>(Up, N, u, N, perm.as<int>(), N, nrhs, true, st);
    IA_CUDA(cudaStreamSynchronize(st));
    prof().resolve();
    stats.t_apply = now_ms() - t0;
  }

  void release() {
    factored = false;
    DevBuf* all[] = {&X, &Xp, &perm, &iperm, &split_dim, &knn, &knn_pos, &samp, &ranks, &skel,
                     &piv_ws, &A_ws, &status, &arena_dev, &level_off_dev, &tbuf, &vbuf, &vbuf32,
                     &ubuf, &rbuf, &wt, &io, &normbuf, &LU, &LUpiv, &Wb, &Zb, &Zpiv, &Cb, &LU32,
                     &Wb32, &Zb32, &Cb32, &tbuf32, &Kleaf, &Ustore};
    for (DevBuf* b : all) b->release();
    Pl.clear();
    Pl32.clear();
    tree_s.release();
    knn_s.release();
    samp_s.release();
  }
};

__global__ void axpby_kernel(const double* u, double* r, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    r[i] = u[i] - r[i];
}
__global__ void add_kernel(double* w, const double* dl, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    w[i] += dl[i];
}
__global__ void scale_kernel(const double* x, double* y, double a, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}
__global__ void colnorm_kernel(const double* x, int N, double* out) {
  __shared__ double red[32];
  const double* c = x + (size_t)blockIdx.x * N;
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s = fma(c[i], c[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(s);
  }
}

void Solver::column_norms(const double* x, int nrhs, std::vector<double>& out) {
  double* dn = normbuf.ensure_n<double>(nrhs);
  {
    ProfScope _ps(PK_MISC, st);
    colnorm_kernel<<<nrhs, 256, 0, st>>>(x, N, dn);
    IA_LAUNCH_CHECK();
  }
  out.resize(nrhs);
  d2h(out.data(), dn, nrhs, st);
  IA_CUDA(cudaStreamSynchronize(st));
}
void Solver::axpby(const double* u, double* r, size_t n) {
  ProfScope _ps(PK_MISC, st);
  axpby_kernel<<<std::min<size_t>(ceil_div(n, 256), 8192), 256, 0, st>>>(u, r, n);
  IA_LAUNCH_CHECK();
}
void Solver::add_inplace(double* w, const double* dl, size_t n) {
  ProfScope _ps(PK_MISC, st);
  add_kernel<<<std::min<size_t>(ceil_div(n, 256), 8192), 256, 0, st>>>(w, dl, n);
  IA_LAUNCH_CHECK();
}
void Solver::scale_copy(const double* x, double* y, double a, size_t n) {
  ProfScope _ps(PK_MISC, st);
  scale_kernel<<<std::min<size_t>(ceil_div(n, 256), 8192), 256, 0, st>>>(x, y, a, n);
  IA_LAUNCH_CHECK();
}

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

int check_node(int level, int index) {
  Solver& s = S();
  if (level < 1 || level > s.L || index < 0 || index >= (1 << level))
    throw Error(IASKIT_ERR_ARG, "node out of range");
  return (1 << level) + index;
}

}  // namespace

// Records a failure for iaskit_last_error() and returns its code.
int report_error(int code, const std::string& msg) { return fail(code, msg); }

}  // namespace iaskit

using namespace iaskit;

extern "C" {

int iaskit_factor(const double* points, int64_t N, int d, double h, double lambda, int leaf_m,
                  int s_max, double tol) {
  int rc = guarded([&] { S().factor(points, false, N, d, h, lambda, leaf_m, s_max, tol); });
  if (rc != IASKIT_OK) S().factored = false;
  return rc;
}

int iaskit_factor_device(const double* d_points, int64_t N, int d, double h, double lambda,
                         int leaf_m, int s_max, double tol) {
  int rc = guarded([&] { S().factor(d_points, true, N, d, h, lambda, leaf_m, s_max, tol); });
  if (rc != IASKIT_OK) S().factored = false;
  return rc;
}

int iaskit_solve_device(double* d_rhs, int nrhs) {
  return guarded([&] {
    if (!d_rhs) throw Error(IASKIT_ERR_ARG, "rhs is null");
    S().solve_device(d_rhs, nrhs);
  });
}

int iaskit_solve(double* rhs, int nrhs) {
  return guarded([&] {
    Solver& s = S();
    require_factored();
    if (!rhs) throw Error(IASKIT_ERR_ARG, "rhs is null");
    if (nrhs < 1) throw Error(IASKIT_ERR_ARG, "bad nrhs");
    const size_t n = (size_t)s.N * nrhs;
    double* d = s.io.ensure_n<double>(n);
    h2d(d, rhs, n, s.st);
    s.solve_device(d, nrhs);
    d2h(rhs, d, n, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
}

int iaskit_apply_device(const double* d_w, double* d_u, int nrhs) {
  return guarded([&] {
    if (!d_w || !d_u) throw Error(IASKIT_ERR_ARG, "null pointer");
    S().apply_device(d_w, d_u, nrhs);
  });
}

int iaskit_apply(const double* w, double* u, int nrhs) {
  return guarded([&] {
    Solver& s = S();
    require_factored();
    if (!w || !u) throw Error(IASKIT_ERR_ARG, "null pointer");
    if (nrhs < 1) throw Error(IASKIT_ERR_ARG, "bad nrhs");
    const size_t n = (size_t)s.N * nrhs;
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
  char tmp[512];
  snprintf(tmp, sizeof tmp,
           "\"N\":%d,\"d\":%d,\"L\":%d,\"factored\":%s,\"ms\":{\"tree\":%.3f,\"knn\":%.3f,"
           "\"skeletonize\":%.3f,\"leaf_lu\":%.3f,\"factor_levels\":%.3f,\"factor\":%.3f,"
           "\"solve\":%.3f,\"apply\":%.3f},\"knn_fallback\":%d,\"bytes\":{\"W\":%lld,\"LU\":%lld,"
           "\"P\":%lld,\"operator\":%lld},\"precision\":\"%s\",\"refine_sweeps\":%d,",
           s.N, s.d, s.L, s.factored ? "true" : "false", s.stats.t_tree, s.stats.t_knn,
           s.stats.t_skel, s.stats.t_leaf_lu, s.stats.t_factor_levels, s.stats.t_factor,
           s.stats.t_solve, s.stats.t_apply, s.stats.knn_fallback, (long long)s.stats.bytes_W,
           (long long)s.stats.bytes_LU, (long long)s.stats.bytes_P,
           (long long)s.stats.bytes_operator, s.prec == PREC_MIXED ? "mixed" : "fp64",
           s.stats.refine_sweeps);
  j += tmp;
  j += "\"refine_history\":[";
  for (size_t i = 0; i < s.stats.refine_hist.size(); ++i) {
    snprintf(tmp, sizeof tmp, "%s%.6g", i ? "," : "", s.stats.refine_hist[i]);
    j += tmp;
  }
  j += "],\"launches\":";
  j += std::to_string(prof().launches);
  j += ",\"kernels\":{";
  for (int k = 0; k < PK_COUNT; ++k) {
    snprintf(tmp, sizeof tmp, "%s\"%s\":{\"ms\":%.4f,\"calls\":%lld,\"flops\":%.6g}", k ? "," : "",
             prof_name(k), prof().ms[k], prof().calls[k], prof().flops[k]);
    j += tmp;
  }
  j += "},\"mean_rank_per_level\":[";
  for (int l = 1; l <= s.L && s.factored; ++l) {
    double tot = 0;
    for (int i = 0; i < (1 << l); ++i) tot += s.nd[(1 << l) + i].s;
    snprintf(tmp, sizeof tmp, "%s%.3f", l > 1 ? "," : "", tot / (1 << l));
    j += tmp;
  }
  j += "]}";
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
  return S().L;
}

int iaskit_get_perm(int32_t* out) {
  return guarded([&] {
    require_factored();
    Solver& s = S();
    d2h(out, s.perm.as<int>(), s.N, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
}

int iaskit_get_knn(int32_t* out, int kappa_cap) {
  return guarded([&] {
    require_factored();
    Solver& s = S();
    if (s.L == 0) throw Error(IASKIT_ERR_ARG, "no kNN lists for a single-leaf tree");
    if (kappa_cap < s.kappa) throw Error(IASKIT_ERR_ARG, "buffer too small");
    d2h(out, s.knn.as<int>(), (size_t)s.N * s.kappa, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
}

int iaskit_get_ranks(int32_t* out, int count) {
  return guarded([&] {
    require_factored();
    Solver& s = S();
    if (count < (2 << s.L)) throw Error(IASKIT_ERR_ARG, "buffer too small");
    for (int u = 0; u < (2 << s.L); ++u) out[u] = u == 0 ? 0 : s.nd[u].s;
  });
}

int iaskit_get_skeleton(int level, int index, int32_t* out, int cap) {
  int rs = 0;
  int rc = guarded([&] {
    require_factored();
    Solver& s = S();
    int u = check_node(level, index);
    rs = s.nd[u].s;
    if (cap < rs) throw Error(IASKIT_ERR_ARG, "buffer too small");
    d2h(out, s.skel.as<int>() + (size_t)u * s.s_max, rs, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
  return rc == IASKIT_OK ? rs : rc;
}

int iaskit_get_samples(int level, int index, int32_t* out, int cap) {
  int ns = 0;
  int rc = guarded([&] {
    require_factored();
    Solver& s = S();
    int u = check_node(level, index);
    ns = s.nd[u].nsamp;
    if (cap < ns) throw Error(IASKIT_ERR_ARG, "buffer too small");
    d2h(out, s.samp.as<int>() + s.nd[u].samp_off, ns, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
  return rc == IASKIT_OK ? ns : rc;
}

int iaskit_get_P(int level, int index, double* out, int64_t cap) {
  int nc = 0;
  int rc = guarded([&] {
    require_factored();
    Solver& s = S();
    int u = check_node(level, index);
    nc = s.nd[u].ncols;
    int64_t n = (int64_t)s.nd[u].s * nc;
    if (cap < n) throw Error(IASKIT_ERR_ARG, "buffer too small");
    d2h(out, s.Pl[level]->as<double>() + s.nd[u].P_off, n, s.st);
    IA_CUDA(cudaStreamSynchronize(s.st));
  });
  return rc == IASKIT_OK ? nc : rc;
}

}  // extern "C"
