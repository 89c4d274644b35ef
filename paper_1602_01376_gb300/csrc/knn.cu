// Brute-force kNN lists (the nearest-neighbour input of ASKIT, Sec. II-B).
//
// The lists are defined on the FP64 squared distance sum_k (x_k - y_k)^2 with the
// coordinates summed in order and every operation rounded (no FMA), ties broken by
// the lower index.  The search runs in three steps:
//   1. FP32 prefilter: every query keeps its KP smallest FP32 squared distances
//      (FMA accumulation) over all points, in registers;
//   2. exact re-rank: the KP candidates get their FP64 distances, sorted by
//      (distance, index); the first kappa form the list.  A rounding bound proves
//      that no excluded point can come before the kappa-th: with |x| <= M for all
//      coordinates, u = 2^-24 and e = 4.01 u M, every FP32 difference is within e of
//      the exact one, so ||t|| >= sqrt(S32 / (1 + gamma_d)) - sqrt(d) e for the exact
//      difference vector t and the FP32 sum S32 (gamma_d = d u / (1 - d u)); every
//      excluded point has S32 >= the largest kept FP32 value;
//   3. queries whose bound fails (near-ties at the cut) are redone by an exact FP64
//      scan over all points.
#include <cfloat>
#include <climits>

#include "kernels.cuh"

namespace iaskit {

namespace {


__global__ void to_float_kernel(const double* X, float* X32, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) X32[i] = (float)X[i];
}

__global__ void maxabs_kernel(const double* X, size_t n, unsigned long long* out) {
  double m = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(X[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// FP32 prefilter.  A block owns KT_QB = 256 queries (one per thread for the
// selection) and streams the points in tiles of KT_RB = 32:
//   phase 1: every thread computes 8 queries x 4 points of the tile's squared
//            distances, sum_k fma(q_k - r_k, q_k - r_k, acc) in coordinate order
//            (coordinates d..D-1 are zero on both sides and add exact zeros), into
//            shared memory;
//   phase 2: every thread scans its query's row and updates its register list.
// 8 x 4 keeps the kernel at two resident blocks per SM, so one block's selection
// and barriers overlap the other's arithmetic.
constexpr int KT_QB = 256;
constexpr int KT_RB = 32;
template <int D, int KP>
__global__ void __launch_bounds__(KT_QB) knn_prefilter_tiled_kernel(const float* X32, int d,
                                                                   const KnnTile* tiles,
                                                                   float* cand_d, int* cand_i) {
  extern __shared__ float kt_sh[];
  float* Qs = kt_sh;                      // [D][KT_QB]
  float* Rs = Qs + D * KT_QB;             // [D][KT_RB]
  float* Dt = Rs + D * KT_RB;             // [KT_QB][KT_RB + 1]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const KnnTile tl = tiles[blockIdx.x];
  const int q0 = tl.q0, qend = tl.q0 + tl.qn;
  for (int e = tid; e < D * KT_QB; e += KT_QB) {
    const int i = e / D, k = e % D;
    Qs[k * KT_QB + i] = (q0 + i < qend && k < d) ? X32[(size_t)(q0 + i) * d + k] : 0.0f;
  }
  const int my_q = q0 + tid;
  const bool active = my_q < qend;
  float bd[KP];
  int bi[KP];
#pragma unroll
  for (int t = 0; t < KP; ++t) {
    bd[t] = FLT_MAX;
    bi[t] = INT_MAX;
  }
  const int rend = tl.rb + tl.rn;
  for (int r0 = tl.rb; r0 < rend; r0 += KT_RB) {
    const int nt = min(KT_RB, rend - r0);
    __syncthreads();
    for (int e = tid; e < D * KT_RB; e += KT_QB) {
      const int j = e / D, k = e % D;
      Rs[k * KT_RB + j] = (j < nt && k < d) ? X32[(size_t)(r0 + j) * d + k] : 0.0f;
    }
    __syncthreads();
    float acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
#pragma unroll 4
    for (int k = 0; k < D; ++k) {
      float qa[8], rb[4];
#pragma unroll
      for (int a = 0; a < 8; ++a) qa[a] = Qs[k * KT_QB + lane + 32 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) rb[b] = Rs[k * KT_RB + warp * 4 + b];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          float df = qa[a] - rb[b];
          acc[a][b] = fmaf(df, df, acc[a][b]);
        }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) Dt[(lane + 32 * a) * (KT_RB + 1) + warp * 4 + b] = acc[a][b];
    __syncthreads();
    if (active) {
      for (int j = 0; j < nt; ++j) {
        const float v = Dt[tid * (KT_RB + 1) + j];
        const int ref = r0 + j;
        if (v <= bd[KP - 1] && ref != my_q) {
          float cv = v;
          int cj = ref;
#pragma unroll
          for (int t = 0; t < KP; ++t) {
            bool less = cv < bd[t] || (cv == bd[t] && cj < bi[t]);
            float tv = less ? bd[t] : cv;
            int tj = less ? bi[t] : cj;
            bd[t] = less ? cv : bd[t];
            bi[t] = less ? cj : bi[t];
            cv = tv;
            cj = tj;
          }
        }
      }
    }
  }
  if (active) {
#pragma unroll
    for (int t = 0; t < KP; ++t) {
      cand_d[(size_t)my_q * KP + t] = bd[t];
      cand_i[(size_t)my_q * KP + t] = bi[t];
    }
  }
}

// Exact FP64 squared distance in coordinate order, no contraction.
__device__ __forceinline__ double exact_sqdist(const double* a, const double* b, int d) {
  double acc = 0.0;
  for (int k = 0; k < d; ++k) {
    double df = __dsub_rn(a[k], b[k]);
    acc = __dadd_rn(acc, __dmul_rn(df, df));
  }
  return acc;
}

__device__ __forceinline__ bool pair_less(double a, int ia, double b, int ib) {
  return a < b || (a == b && ia < ib);
}

// One block of KT_QB threads per work tile, one thread per query.
template <int KP>
__global__ void knn_rerank_kernel(const double* X, int d, int kappa, const KnnTile* tiles,
                                  const float* cand_d, const int* cand_i,
                                  const unsigned long long* maxabs_bits, int* knn, int2* flagged,
                                  int* nflagged) {
  const KnnTile tl = tiles[blockIdx.x];
  if ((int)threadIdx.x >= tl.qn) return;
  const int i = tl.q0 + threadIdx.x;
  const int N = tl.rn, rb = tl.rb;
  double dd[KP];
  int ii[KP];
  const double* xi = X + (size_t)i * d;
  const int nc = min(KP, N - 1);
  for (int t = 0; t < nc; ++t) {
    int j = cand_i[(size_t)i * KP + t];
    if (j < rb || j >= rb + N) {  // an FP32 distance overflowed: redo this query exactly
      int slot = atomicAdd(nflagged, 1);
      flagged[slot] = make_int2(i, blockIdx.x);
      return;
    }
    ii[t] = j;
    dd[t] = exact_sqdist(xi, X + (size_t)j * d, d);
  }
  for (int a = 1; a < nc; ++a) {  // insertion sort by (distance, index)
    double v = dd[a];
    int j = ii[a];
    int b = a - 1;
    while (b >= 0 && pair_less(v, j, dd[b], ii[b])) {
      dd[b + 1] = dd[b];
      ii[b + 1] = ii[b];
      --b;
    }
    dd[b + 1] = v;
    ii[b + 1] = j;
  }
  for (int t = 0; t < kappa; ++t) knn[(size_t)i * kappa + t] = ii[t];
  if (N - 1 <= KP) return;  // every other point was a candidate
  const double M = __longlong_as_double((long long)*maxabs_bits);
  const double u = 5.9604644775390625e-08;  // 2^-24
  const double e = 4.01 * u * M;
  const double gam = d * u / (1.0 - d * u);
  const double Dkept = (double)cand_d[(size_t)i * KP + KP - 1];
  const double r_lo = sqrt(Dkept / (1.0 + gam)) * (1.0 - 1e-15) - sqrt((double)d) * e;
  const bool ok = r_lo > 0.0 && r_lo * r_lo * (1.0 - 1e-12) > dd[kappa - 1];
  if (!ok) {
    int slot = atomicAdd(nflagged, 1);
    flagged[slot] = make_int2(i, blockIdx.x);
  }
}

// Exact scan for one flagged query per block: every thread keeps a sorted top-kappa
// list of its strided share of the points, then kappa rounds of a block-wide argmin
// over the list heads merge them.
constexpr int FB_THREADS = 128;
constexpr int FB_MAXK = 64;
__global__ void knn_fallback_kernel(const double* X, int d, int kappa, const KnnTile* tiles,
                                    const int2* flagged, int* knn) {
  __shared__ double sd[FB_THREADS];
  __shared__ int si[FB_THREADS];
  __shared__ int st[FB_THREADS];
  __shared__ int chosen[FB_MAXK];
  const int i = flagged[blockIdx.x].x;
  const KnnTile tl = tiles[flagged[blockIdx.x].y];
  const int r_begin = tl.rb, r_end = tl.rb + tl.rn;
  const double* xi = X + (size_t)i * d;
  double ld[FB_MAXK];
  int li[FB_MAXK];
  for (int t = 0; t < kappa; ++t) {
    ld[t] = DBL_MAX;
    li[t] = INT_MAX;
  }
  for (int j = r_begin + threadIdx.x; j < r_end; j += FB_THREADS) {
    if (j == i) continue;
    double v = exact_sqdist(xi, X + (size_t)j * d, d);
    if (!pair_less(v, j, ld[kappa - 1], li[kappa - 1])) continue;
    int b = kappa - 1;
    while (b > 0 && pair_less(v, j, ld[b - 1], li[b - 1])) {
      ld[b] = ld[b - 1];
      li[b] = li[b - 1];
      --b;
    }
    ld[b] = v;
    li[b] = j;
  }
  int head = 0;
  for (int t = 0; t < kappa; ++t) {
    sd[threadIdx.x] = head < kappa ? ld[head] : DBL_MAX;
    si[threadIdx.x] = head < kappa ? li[head] : INT_MAX;
    st[threadIdx.x] = threadIdx.x;
    __syncthreads();
    for (int s = FB_THREADS / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s && pair_less(sd[threadIdx.x + s], si[threadIdx.x + s], sd[threadIdx.x],
                                       si[threadIdx.x])) {
        sd[threadIdx.x] = sd[threadIdx.x + s];
        si[threadIdx.x] = si[threadIdx.x + s];
        st[threadIdx.x] = st[threadIdx.x + s];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) chosen[t] = si[0];
    if (threadIdx.x == st[0]) ++head;
    __syncthreads();
  }
  for (int t = threadIdx.x; t < kappa; t += FB_THREADS) knn[(size_t)i * kappa + t] = chosen[t];
}

template <int D, int KP>
void launch_prefilter(const float* X32, int d, const KnnTile* tiles, int ntiles, float* cd, int* ci,
                      cudaStream_t st) {
  const size_t smem = sizeof(float) * ((size_t)D * KT_QB + (size_t)D * KT_RB + (size_t)KT_QB * (KT_RB + 1));
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(knn_prefilter_tiled_kernel<D, KP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  knn_prefilter_tiled_kernel<D, KP><<<ntiles, KT_QB, smem, st>>>(X32, d, tiles, cd, ci);
  IA_LAUNCH_CHECK();
}

template <int KP>
void prefilter_dispatch(const float* X32, int d, const KnnTile* tl, int nt, float* cd, int* ci,
                        cudaStream_t st) {
  if (d <= 8) launch_prefilter<8, KP>(X32, d, tl, nt, cd, ci, st);
  else if (d <= 16) launch_prefilter<16, KP>(X32, d, tl, nt, cd, ci, st);
  else if (d <= 24) launch_prefilter<24, KP>(X32, d, tl, nt, cd, ci, st);
  else if (d <= 32) launch_prefilter<32, KP>(X32, d, tl, nt, cd, ci, st);
  else if (d <= 40) launch_prefilter<40, KP>(X32, d, tl, nt, cd, ci, st);
  else if (d <= 48) launch_prefilter<48, KP>(X32, d, tl, nt, cd, ci, st);
  else if (d <= 56) launch_prefilter<56, KP>(X32, d, tl, nt, cd, ci, st);
  else if (d <= 64) launch_prefilter<64, KP>(X32, d, tl, nt, cd, ci, st);
  else throw Error(IASKIT_ERR_UNSUPPORTED, "kNN supports d <= 64");
}

}  // namespace

std::vector<KnnTile> knn_tiles(const std::vector<std::pair<int, int>>& problems) {
  std::vector<KnnTile> t;
  for (const auto& pr : problems)
    for (int q = 0; q < pr.second; q += KT_QB)
      t.push_back(KnnTile{pr.first + q, std::min(KT_QB, pr.second - q), pr.first, pr.second});
  return t;
}

int knn_bruteforce(const double* X, int N, int d, int kappa, int* knn,
                   const std::vector<std::pair<int, int>>& problems, KnnScratch& s,
                   cudaStream_t st) {
  ProfScope _ps(PK_KNN, st);
  int min_n = N;
  for (const auto& pr : problems) min_n = std::min(min_n, pr.second);
  if (kappa < 1 || kappa > min_n - 1) throw Error(IASKIT_ERR_ARG, "kappa must be in [1, N-1]");
  if (kappa > FB_MAXK - 16) throw Error(IASKIT_ERR_UNSUPPORTED, "kappa > 48");
  const size_t nd = (size_t)N * d;
  float* X32 = s.x32.ensure_n<float>(nd);
  to_float_kernel<<<ceil_div(nd, 256), 256, 0, st>>>(X, X32, nd);
  IA_LAUNCH_CHECK();
  unsigned long long* mx = s.maxabs.ensure_n<unsigned long long>(1);
  IA_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st));
  maxabs_kernel<<<304, 256, 0, st>>>(X, nd, mx);
  IA_LAUNCH_CHECK();
  int2* flagged = s.flagged.ensure_n<int2>(N);
  int* nfl = s.counter.ensure_n<int>(1);
  IA_CUDA(cudaMemsetAsync(nfl, 0, sizeof(int), st));
  const std::vector<KnnTile> tiles = knn_tiles(problems);
  KnnTile* dt = s.tiles.ensure_n<KnnTile>(tiles.size());
  h2d(dt, tiles.data(), tiles.size(), st);
  const int nt = (int)tiles.size();
  const bool wide = kappa + 8 > 32;
  const int KP = wide ? 64 : 32;
  // algorithmic work of the FP32 prefilter: a subtraction and an FMA per pair and coordinate
  for (const auto& pr : problems) prof().flops[PK_KNN] += 3.0 * (double)pr.second * pr.second * d;
  float* cd = s.cand_d.ensure_n<float>((size_t)N * KP);
  int* ci = s.cand_i.ensure_n<int>((size_t)N * KP);
  if (wide) {
    prefilter_dispatch<64>(X32, d, dt, nt, cd, ci, st);
    knn_rerank_kernel<64><<<nt, KT_QB, 0, st>>>(X, d, kappa, dt, cd, ci, mx, knn, flagged, nfl);
  } else {
    prefilter_dispatch<32>(X32, d, dt, nt, cd, ci, st);
    knn_rerank_kernel<32><<<nt, KT_QB, 0, st>>>(X, d, kappa, dt, cd, ci, mx, knn, flagged, nfl);
  }
  IA_LAUNCH_CHECK();
  int nf = 0;
  d2h(&nf, nfl, 1, st);
  IA_CUDA(cudaStreamSynchronize(st));
  if (nf > 0) {
    knn_fallback_kernel<<<nf, FB_THREADS, 0, st>>>(X, d, kappa, dt, flagged, knn);
    IA_LAUNCH_CHECK();
  }
  return nf;
}

}  // namespace iaskit

// ---------------------------------------------------------------------------
// kNN without device allocation (iaskit_knn_noalloc in include/iaskit.h).
//
// Its scratch lives in one file-scope device array that every GPU loading this
// library holds until the process exits.  Host code must not pass the array's
// name to a kernel (on the host it is only a stand-in symbol); the device address
// is looked up once per device with cudaGetSymbolAddress and cached.
namespace iaskit {
namespace {

constexpr int64_t NA_MAX_N = 32768;             // points
constexpr int64_t NA_MAX_ND = int64_t(1) << 20;  // N * d coordinates
constexpr int NA_KP = 32;                        // candidates kept per query (kappa <= 24)
constexpr size_t NA_X32 = 0;
constexpr size_t NA_CD = NA_X32 + sizeof(float) * NA_MAX_ND;
constexpr size_t NA_CI = NA_CD + sizeof(float) * NA_MAX_N * NA_KP;
constexpr size_t NA_FLAGGED = NA_CI + sizeof(int) * NA_MAX_N * NA_KP;
constexpr size_t NA_TILES = NA_FLAGGED + sizeof(int2) * NA_MAX_N;
constexpr size_t NA_COUNTER = NA_TILES + sizeof(KnnTile) * (NA_MAX_N / KT_QB);
constexpr size_t NA_MAXABS = NA_COUNTER + 256;
constexpr size_t NA_BYTES = NA_MAXABS + 256;   // about 12.3 MiB

__device__ __align__(256) unsigned char g_knn_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
void* g_knn_noalloc_base[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once).
unsigned char* noalloc_scratch() {
  int dev = 0;
  IA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEVICES) throw Error(IASKIT_ERR_UNSUPPORTED, "device ordinal >= 64");
  if (!g_knn_noalloc_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_knn_noalloc_scratch);
    if (e != cudaSuccess || !p)
      throw Error(IASKIT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_knn_noalloc_base[dev] = p;
  }
  return static_cast<unsigned char*>(g_knn_noalloc_base[dev]);
}

void knn_noalloc(const double* X, int N, int d, int kappa, int* knn, cudaStream_t st) {
  unsigned char* base = noalloc_scratch();
  float* X32 = reinterpret_cast<float*>(base + NA_X32);
  float* cd = reinterpret_cast<float*>(base + NA_CD);
  int* ci = reinterpret_cast<int*>(base + NA_CI);
  int2* flagged = reinterpret_cast<int2*>(base + NA_FLAGGED);
  KnnTile* dt = reinterpret_cast<KnnTile*>(base + NA_TILES);
  int* nfl = reinterpret_cast<int*>(base + NA_COUNTER);
  unsigned long long* mx = reinterpret_cast<unsigned long long*>(base + NA_MAXABS);
  const size_t nd = (size_t)N * d;
  const std::vector<KnnTile> tiles = knn_tiles({{0, N}});
  const int nt = (int)tiles.size();
  // the array keeps the previous call's contents: clear what must start at zero
  IA_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st));
  IA_CUDA(cudaMemsetAsync(nfl, 0, sizeof(int), st));
  to_float_kernel<<<ceil_div(nd, 256), 256, 0, st>>>(X, X32, nd);
  IA_LAUNCH_CHECK();
  maxabs_kernel<<<304, 256, 0, st>>>(X, nd, mx);
  IA_LAUNCH_CHECK();
  IA_CUDA(cudaMemcpyAsync(dt, tiles.data(), nt * sizeof(KnnTile), cudaMemcpyHostToDevice, st));
  prefilter_dispatch<NA_KP>(X32, d, dt, nt, cd, ci, st);
  knn_rerank_kernel<NA_KP><<<nt, KT_QB, 0, st>>>(X, d, kappa, dt, cd, ci, mx, knn, flagged, nfl);
  IA_LAUNCH_CHECK();
  int nf = 0;
  IA_CUDA(cudaMemcpyAsync(&nf, nfl, sizeof(int), cudaMemcpyDeviceToHost, st));
  IA_CUDA(cudaStreamSynchronize(st));
  if (nf > 0) {
    knn_fallback_kernel<<<nf, FB_THREADS, 0, st>>>(X, d, kappa, dt, flagged, knn);
    IA_LAUNCH_CHECK();
  }
  IA_CUDA(cudaStreamSynchronize(st));
}

}  // namespace

int report_error(int code, const std::string& msg);

}  // namespace iaskit

extern "C" int iaskit_knn_noalloc(const double* d_points, int64_t N, int d, int kappa,
                                  int32_t* d_knn, void* cuda_stream) {
  using namespace iaskit;
  try {
    if (!d_points || !d_knn) return report_error(IASKIT_ERR_ARG, "null pointer");
    if (N < 2 || d < 1) return report_error(IASKIT_ERR_ARG, "need N >= 2 and d >= 1");
    if (N > NA_MAX_N)
      return report_error(IASKIT_ERR_ARG, "N exceeds the no-allocation limit of 32768 points");
    if (d > 64) return report_error(IASKIT_ERR_ARG, "d exceeds the no-allocation limit of 64");
    if (N * (int64_t)d > NA_MAX_ND)
      return report_error(IASKIT_ERR_ARG, "N*d exceeds the no-allocation limit of 1048576");
    if (kappa < 1 || kappa > 24 || kappa > N - 1)
      return report_error(IASKIT_ERR_ARG, "kappa must be in [1, min(24, N-1)]");
    knn_noalloc(d_points, (int)N, d, kappa, d_knn, (cudaStream_t)cuda_stream);
    return IASKIT_OK;
  } catch (const Error& e) {
    return report_error(e.code, e.what());
  }
}
