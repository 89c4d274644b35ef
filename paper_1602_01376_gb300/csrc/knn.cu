// Brute-force kNN lists (the nearest-neighbour input of ASKIT, Sec. II-B).
//
// The lists are defined on the FP64 squared distance sum_k (x_k - y_k)^2 with the
// coordinates summed in order and every operation rounded (no FMA), ties broken by
// the lower index.  The search runs in three steps:
//   1. FP32 prefilter: the points of each problem are centred on the problem's mean and
//      rounded to FP32 (a = fl32(x - mean)); every query keeps the KP smallest values
//      D = fl(fl(|a|^2 + |b|^2) - 2 a.b) (Gram form: one FMA per pair and coordinate,
//      the dot product accumulated in coordinate order, the norms rounded up);
//   2. exact re-rank: the KP candidates get their FP64 distances, sorted by
//      (distance, index); the first kappa form the list.  A rounding bound proves that
//      no excluded point comes before the kappa-th: for every pair,
//      |D - |x - y|^2| <= E = (4K + 16) 2^-23 (|a|^2 + |b|^2)  (K = padded dimension:
//      FP32 accumulation of K products K 2^-24, norm and final roundings 2.5 2^-23, FP32
//      centring 2 2^-23, all relative to |a|^2 + |b|^2, with room to spare), so an
//      excluded point, whose D is at least the largest kept D_KP, lies at FP64 distance
//      >= (D_KP - E(q, |b|^2 <= max_b |b|^2)) (1 - 1e-12);
//   3. queries whose bound fails (near-ties at the cut) are redone by an exact FP64
//      scan over all points.
#include <cfloat>
#include <climits>

#include "kernels.cuh"

namespace iaskit {

namespace {

constexpr int KT_QB = 256;    // queries per tile, one thread each
constexpr int KT_RB = 32;     // points per streamed tile
constexpr int KC_CHUNKS = 64; // partial sums per problem for the mean

// Per problem and chunk of its points, the coordinate sums (FP64, in point order).
__global__ void center_partial_kernel(const double* X, int d, const int2* probs, double* part) {
  const int2 P = probs[blockIdx.y];
  const int per = (P.y + KC_CHUNKS - 1) / KC_CHUNKS;
  const int i0 = blockIdx.x * per, i1 = min(P.y, i0 + per);
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double s = 0.0;
    for (int i = i0; i < i1; ++i) s += X[(size_t)(P.x + i) * d + k];
    part[((size_t)blockIdx.y * KC_CHUNKS + blockIdx.x) * d + k] = s;
  }
}
__global__ void center_mean_kernel(int d, const int2* probs, const double* part, double* mean) {
  const int2 P = probs[blockIdx.x];
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < KC_CHUNKS; ++c) s += part[((size_t)blockIdx.x * KC_CHUNKS + c) * d + k];
    mean[(size_t)blockIdx.x * d + k] = s / P.y;
  }
}
// Centred FP32 coordinates, their squared norms rounded up, and the largest norm of
// each problem (as the bit pattern of a non-negative float, ordered like the value).
__global__ void center_points_kernel(const double* X, int d, const KnnTile* tiles, const double* mean,
                                     float* Xc, float* qn, unsigned* rmax) {
  const KnnTile tl = tiles[blockIdx.x];
  if ((int)threadIdx.x >= tl.qn) return;
  const int i = tl.q0 + threadIdx.x;
  const double* m = mean + (size_t)tl.prob * d;
  double nrm = 0.0;
  for (int k = 0; k < d; ++k) {
    const float c = (float)(X[(size_t)i * d + k] - m[k]);
    Xc[(size_t)i * d + k] = c;
    nrm = fma((double)c, (double)c, nrm);
  }
  const float q = __double2float_ru(nrm);
  qn[i] = q;
  atomicMax(&rmax[tl.prob], __float_as_uint(q));
}

// Prefilter.  A block owns KT_QB queries (one thread each for the selection) and
// streams the points in tiles of KT_RB:
//   phase 1: every thread computes the dot products of 8 queries x 4 points of the
//            tile, acc = fma(q_k, r_k, acc) in coordinate order (coordinates d..D-1 are
//            zero on both sides), then D = (|q|^2 + |r|^2) - 2 acc, into shared memory;
//   phase 2: every thread scans its query's row and updates its register list.
// 8 x 4 keeps the kernel at two resident blocks per SM, so one block's selection and
// barriers overlap the other's arithmetic.
template <int D, int KP>
__global__ void __launch_bounds__(KT_QB) knn_prefilter_kernel(const float* Xc, const float* qnorm, int d,
                                                              const KnnTile* tiles, float* cand_d,
                                                              int* cand_i) {
  extern __shared__ float kt_sh[];
  float* Qs = kt_sh;                      // [D][KT_QB]
  float* Rs = Qs + D * KT_QB;             // [D][KT_RB]
  float* qn_s = Rs + D * KT_RB;           // [KT_QB]
  float* rn_s = qn_s + KT_QB;             // [KT_RB]
  float* Dt = rn_s + KT_RB;               // [KT_QB][KT_RB + 1]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const KnnTile tl = tiles[blockIdx.x];
  const int q0 = tl.q0, qend = tl.q0 + tl.qn;
  for (int e = tid; e < D * KT_QB; e += KT_QB) {
    const int i = e / D, k = e % D;
    Qs[k * KT_QB + i] = (q0 + i < qend && k < d) ? Xc[(size_t)(q0 + i) * d + k] : 0.0f;
  }
  const int my_q = q0 + tid;
  const bool active = my_q < qend;
  qn_s[tid] = active ? qnorm[my_q] : 0.0f;
  float bd[KP];
  int bi[KP];
#pragma unroll
  for (int u = 0; u < KP; ++u) {
    bd[u] = FLT_MAX;
    bi[u] = INT_MAX;
  }
  const int rend = tl.rb + tl.rn;
  for (int r0 = tl.rb; r0 < rend; r0 += KT_RB) {
    const int nt = min(KT_RB, rend - r0);
    __syncthreads();
    for (int e = tid; e < D * KT_RB; e += KT_QB) {
      const int j = e / D, k = e % D;
      Rs[k * KT_RB + j] = (j < nt && k < d) ? Xc[(size_t)(r0 + j) * d + k] : 0.0f;
    }
    if (tid < KT_RB) rn_s[tid] = tid < nt ? qnorm[r0 + tid] : 0.0f;
    __syncthreads();
    float acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
#pragma unroll 4
    for (int k = 0; k < D; ++k) {
      float qa[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) qa[a] = Qs[k * KT_QB + lane + 32 * a];
      const float4 rb = *reinterpret_cast<const float4*>(Rs + k * KT_RB + warp * 4);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        acc[a][0] = fmaf(qa[a], rb.x, acc[a][0]);
        acc[a][1] = fmaf(qa[a], rb.y, acc[a][1]);
        acc[a][2] = fmaf(qa[a], rb.z, acc[a][2]);
        acc[a][3] = fmaf(qa[a], rb.w, acc[a][3]);
      }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int q = lane + 32 * a;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = warp * 4 + b;
        Dt[q * (KT_RB + 1) + c] = (qn_s[q] + rn_s[c]) - 2.0f * acc[a][b];
      }
    }
    __syncthreads();
    if (active) {
      for (int j = 0; j < nt; ++j) {
        const float v = Dt[tid * (KT_RB + 1) + j];
        const int ref = r0 + j;
        if (v <= bd[KP - 1] && ref != my_q) {
          float cv = v;
          int cj = ref;
#pragma unroll
          for (int u = 0; u < KP; ++u) {
            bool less = cv < bd[u] || (cv == bd[u] && cj < bi[u]);
            float tv = less ? bd[u] : cv;
            int tj = less ? bi[u] : cj;
            bd[u] = less ? cv : bd[u];
            bi[u] = less ? cj : bi[u];
            cv = tv;
            cj = tj;
          }
        }
      }
    }
  }
  if (active) {
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      cand_d[(size_t)my_q * KP + u] = bd[u];
      cand_i[(size_t)my_q * KP + u] = bi[u];
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

// One block of KT_QB threads per work tile, one thread per query.  Kdim is the
// padded dimension of the prefilter (its accumulation length).
template <int KP>
__global__ void knn_rerank_kernel(const double* X, int d, int kappa, int Kdim, const KnnTile* tiles,
                                  const float* cand_d, const int* cand_i, const float* qnorm,
                                  const unsigned* rmax_bits, int* knn, int2* flagged, int* nflagged) {
  const KnnTile tl = tiles[blockIdx.x];
  if ((int)threadIdx.x >= tl.qn) return;
  const int i = tl.q0 + threadIdx.x;
  const int N = tl.rn, rb = tl.rb;
  double dd[KP];
  int ii[KP];
  const double* xi = X + (size_t)i * d;
  const int nc = min(KP, N - 1);
  for (int u = 0; u < nc; ++u) {
    int j = cand_i[(size_t)i * KP + u];
    if (j < rb || j >= rb + N) {  // an FP32 distance overflowed: redo this query exactly
      int slot = atomicAdd(nflagged, 1);
      flagged[slot] = make_int2(i, blockIdx.x);
      return;
    }
    ii[u] = j;
    dd[u] = exact_sqdist(xi, X + (size_t)j * d, d);
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
  for (int u = 0; u < kappa; ++u) knn[(size_t)i * kappa + u] = ii[u];
  if (N - 1 <= KP) return;  // every other point was a candidate
  const double c = (4.0 * Kdim + 16.0) * 1.1920928955078125e-07;  // (4K + 16) 2^-23
  const double E = c * ((double)qnorm[i] + (double)__uint_as_float(rmax_bits[tl.prob]));
  const double Dkept = (double)cand_d[(size_t)i * KP + KP - 1];
  const double lo = (Dkept - E) * (1.0 - 1e-12);
  const bool ok = lo > dd[kappa - 1];
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
void launch_prefilter(const float* Xc, const float* qn, int d, const KnnTile* tiles, int ntiles, float* cd,
                      int* ci, cudaStream_t st) {
  const size_t smem = sizeof(float) * ((size_t)D * KT_QB + (size_t)D * KT_RB + KT_QB + KT_RB +
                                       (size_t)KT_QB * (KT_RB + 1));
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(knn_prefilter_kernel<D, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  knn_prefilter_kernel<D, KP><<<ntiles, KT_QB, smem, st>>>(Xc, qn, d, tiles, cd, ci);
  IA_LAUNCH_CHECK();
}

// Padded dimension (multiple of 8) of the prefilter for d.
int padded_dim(int d) { return (d + 7) / 8 * 8; }

template <int KP>
void prefilter_dispatch(const float* Xc, const float* qn, int d, const KnnTile* tl, int nt, float* cd, int* ci,
                        cudaStream_t st) {
  switch (padded_dim(d)) {
    case 8: launch_prefilter<8, KP>(Xc, qn, d, tl, nt, cd, ci, st); break;
    case 16: launch_prefilter<16, KP>(Xc, qn, d, tl, nt, cd, ci, st); break;
    case 24: launch_prefilter<24, KP>(Xc, qn, d, tl, nt, cd, ci, st); break;
    case 32: launch_prefilter<32, KP>(Xc, qn, d, tl, nt, cd, ci, st); break;
    case 40: launch_prefilter<40, KP>(Xc, qn, d, tl, nt, cd, ci, st); break;
    case 48: launch_prefilter<48, KP>(Xc, qn, d, tl, nt, cd, ci, st); break;
    case 56: launch_prefilter<56, KP>(Xc, qn, d, tl, nt, cd, ci, st); break;
    case 64: launch_prefilter<64, KP>(Xc, qn, d, tl, nt, cd, ci, st); break;
    default: throw Error(IASKIT_ERR_UNSUPPORTED, "kNN supports d <= 64");
  }
}

// Scratch pointers of one kNN run (the allocating and the allocation-free callers).
struct KnnBufs {
  float* Xc;
  float* qn;
  double* part;
  double* mean;
  unsigned* rmax;
  int2* probs;
  KnnTile* tiles;
  float* cd;
  int* ci;
  int2* flagged;
  int* nfl;
};

// The whole search; returns the number of queries redone by the exact scan.
template <int KP>
int knn_run(const double* X, int d, int kappa, const std::vector<std::pair<int, int>>& problems,
            const std::vector<KnnTile>& tiles, const KnnBufs& b, int* knn, cudaStream_t st) {
  const int np = (int)problems.size(), nt = (int)tiles.size();
  std::vector<int2> hp(np);
  for (int q = 0; q < np; ++q) hp[q] = make_int2(problems[q].first, problems[q].second);
  IA_CUDA(cudaMemcpyAsync(b.probs, hp.data(), np * sizeof(int2), cudaMemcpyHostToDevice, st));
  IA_CUDA(cudaMemcpyAsync(b.tiles, tiles.data(), nt * sizeof(KnnTile), cudaMemcpyHostToDevice, st));
  IA_CUDA(cudaMemsetAsync(b.rmax, 0, np * sizeof(unsigned), st));
  IA_CUDA(cudaMemsetAsync(b.nfl, 0, sizeof(int), st));
  center_partial_kernel<<<dim3(KC_CHUNKS, np), 64, 0, st>>>(X, d, b.probs, b.part);
  IA_LAUNCH_CHECK();
  center_mean_kernel<<<np, 64, 0, st>>>(d, b.probs, b.part, b.mean);
  IA_LAUNCH_CHECK();
  center_points_kernel<<<nt, KT_QB, 0, st>>>(X, d, b.tiles, b.mean, b.Xc, b.qn, b.rmax);
  IA_LAUNCH_CHECK();
  prefilter_dispatch<KP>(b.Xc, b.qn, d, b.tiles, nt, b.cd, b.ci, st);
  knn_rerank_kernel<KP><<<nt, KT_QB, 0, st>>>(X, d, kappa, padded_dim(d), b.tiles, b.cd, b.ci, b.qn, b.rmax,
                                              knn, b.flagged, b.nfl);
  IA_LAUNCH_CHECK();
  int nf = 0;
  IA_CUDA(cudaMemcpyAsync(&nf, b.nfl, sizeof(int), cudaMemcpyDeviceToHost, st));
  IA_CUDA(cudaStreamSynchronize(st));
  if (nf > 0) {
    knn_fallback_kernel<<<nf, FB_THREADS, 0, st>>>(X, d, kappa, b.tiles, b.flagged, knn);
    IA_LAUNCH_CHECK();
  }
  return nf;
}

}  // namespace

std::vector<KnnTile> knn_tiles(const std::vector<std::pair<int, int>>& problems) {
  std::vector<KnnTile> t;
  for (size_t p = 0; p < problems.size(); ++p) {
    const auto& pr = problems[p];
    for (int q = 0; q < pr.second; q += KT_QB)
      t.push_back(KnnTile{pr.first + q, std::min(KT_QB, pr.second - q), pr.first, pr.second, (int)p});
  }
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
  if (d > 64) throw Error(IASKIT_ERR_UNSUPPORTED, "kNN supports d <= 64");
  const int np = (int)problems.size();
  const std::vector<KnnTile> tiles = knn_tiles(problems);
  const bool wide = kappa + 8 > 32;
  const int KP = wide ? 64 : 32;
  KnnBufs b{};
  b.Xc = s.x32.ensure_n<float>((size_t)N * d);
  b.qn = s.qnorm.ensure_n<float>(N);
  b.part = s.part.ensure_n<double>((size_t)np * KC_CHUNKS * d);
  b.mean = s.mean.ensure_n<double>((size_t)np * d);
  b.rmax = s.rmax.ensure_n<unsigned>(np);
  b.probs = s.probs.ensure_n<int2>(np);
  b.tiles = s.tiles.ensure_n<KnnTile>(tiles.size());
  b.cd = s.cand_d.ensure_n<float>((size_t)N * KP);
  b.ci = s.cand_i.ensure_n<int>((size_t)N * KP);
  b.flagged = s.flagged.ensure_n<int2>(N);
  b.nfl = s.counter.ensure_n<int>(1);
  // algorithmic work of the prefilter: one multiply-add per pair and coordinate
  for (const auto& pr : problems) prof().flops[PK_KNN] += 2.0 * (double)pr.second * pr.second * d;
  return wide ? knn_run<64>(X, d, kappa, problems, tiles, b, knn, st)
              : knn_run<32>(X, d, kappa, problems, tiles, b, knn, st);
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
constexpr size_t NA_QN = NA_X32 + sizeof(float) * NA_MAX_ND;
constexpr size_t NA_PART = NA_QN + sizeof(float) * NA_MAX_N;
constexpr size_t NA_MEAN = NA_PART + sizeof(double) * KC_CHUNKS * 64;
constexpr size_t NA_CD = NA_MEAN + sizeof(double) * 64;
constexpr size_t NA_CI = NA_CD + sizeof(float) * NA_MAX_N * NA_KP;
constexpr size_t NA_FLAGGED = NA_CI + sizeof(int) * NA_MAX_N * NA_KP;
constexpr size_t NA_TILES = NA_FLAGGED + sizeof(int2) * NA_MAX_N;
constexpr size_t NA_COUNTER = NA_TILES + sizeof(KnnTile) * (NA_MAX_N / KT_QB);
constexpr size_t NA_RMAX = NA_COUNTER + 256;
constexpr size_t NA_PROBS = NA_RMAX + 256;
constexpr size_t NA_BYTES = NA_PROBS + 256;   // about 12.5 MiB

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
  KnnBufs b{};
  b.Xc = reinterpret_cast<float*>(base + NA_X32);
  b.qn = reinterpret_cast<float*>(base + NA_QN);
  b.part = reinterpret_cast<double*>(base + NA_PART);
  b.mean = reinterpret_cast<double*>(base + NA_MEAN);
  b.rmax = reinterpret_cast<unsigned*>(base + NA_RMAX);
  b.probs = reinterpret_cast<int2*>(base + NA_PROBS);
  b.tiles = reinterpret_cast<KnnTile*>(base + NA_TILES);
  b.cd = reinterpret_cast<float*>(base + NA_CD);
  b.ci = reinterpret_cast<int*>(base + NA_CI);
  b.flagged = reinterpret_cast<int2*>(base + NA_FLAGGED);
  b.nfl = reinterpret_cast<int*>(base + NA_COUNTER);
  const std::vector<std::pair<int, int>> probs{{0, N}};
  knn_run<NA_KP>(X, d, kappa, probs, knn_tiles(probs), b, knn, st);
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
