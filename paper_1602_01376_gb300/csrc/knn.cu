// Brute-force kNN lists (the nearest-neighbour input of ASKIT, Sec. II-B).
//
// The lists are defined on the FP64 squared distance sum_k (x_k - y_k)^2 with the
// coordinates summed in order and every operation rounded (no FMA), ties broken by
// the lower index.  The search runs in three steps:
//   1. tensor-core prefilter: the points of each problem are centred on the problem's
//      mean and rounded to FP32 (a = fl32(x - mean)); every query keeps the KP smallest
//      values D = fl(fl(|a|^2 + |b|^2) - 2 a.b), the norms rounded up and the dot
//      products on the fifth-generation tensor cores (tcgen05.mma kind::tf32, TMEM
//      accumulators) in 3xTF32: a = a_hi + a_lo with TF32 terms, a.b ~ a_lo.b_hi +
//      a_hi.b_lo + a_hi.b_hi accumulated in FP32;
//   2. exact re-rank: the KP candidates get their FP64 distances, sorted by
//      (distance, index); the first kappa form the list.  A rounding bound proves that
//      no excluded point comes before the kappa-th: for every pair,
//      |D - |x - y|^2| <= E = (8K + 32) 2^-23 (|a|^2 + |b|^2)  (K = padded dimension:
//      TF32 split remainders 3 2^-22, accumulation of 3K products 3K 2^-23 even with
//      truncating adds, norm and final roundings 2.5 2^-23, FP32 centring 2 2^-23, all
//      relative to |a|^2 + |b|^2, then doubled), so an excluded point, whose D is at
//      least the largest kept D_KP, lies at FP64 distance
//      >= (D_KP - E(q, |b|^2 <= max_b |b|^2)) (1 - 1e-12);
//   3. queries whose bound fails (near-ties at the cut) are redone by an exact FP64
//      scan over all points.
#include <atomic>
#include <cfloat>
#include <climits>
#include <mutex>
#include <type_traits>

#include "kernels.cuh"
#include "tc.cuh"

namespace iaskit {

namespace {

constexpr int KT_QB = 128;    // queries per tile: TMEM lanes
constexpr int KT_RB = 128;    // points per streamed tile: accumulator columns
constexpr int KT_SUB = 4;     // threads per query, one per quarter of a tile's columns
constexpr int KT_NTH = KT_QB * KT_SUB;
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
__global__ void center_points_kernel(const double* X, int d, int Dp, const KnnTile* tiles, const double* mean,
                                     float* Xc, float* qn, unsigned* rmax) {
  const KnnTile tl = tiles[blockIdx.x];
  if ((int)threadIdx.x >= tl.qn) return;
  const int i = tl.q0 + threadIdx.x;
  const double* m = mean + (size_t)tl.prob * d;
  double nrm = 0.0;
  for (int k = 0; k < Dp; ++k) {
    const float c = k < d ? (float)(X[(size_t)i * d + k] - m[k]) : 0.0f;
    Xc[(size_t)i * Dp + k] = c;
    nrm = fma((double)c, (double)c, nrm);
  }
  const float q = __double2float_ru(nrm);
  qn[i] = q;
  atomicMax(&rmax[tl.prob], __float_as_uint(q));
}

// Prefilter on the tensor cores.  A block owns KT_QB = 128 queries (TMEM lanes) and
// streams its problem's points in tiles of KT_RB = 128:
//   * the query block (TF32 hi and lo parts) stays in shared memory; point tiles are
//     staged into one of two buffers while the tensor core works on the other;
//   * thread 0 issues 3 MMAs (lo.hi, hi.lo, hi.hi) per 8 coordinates into one of two
//     TMEM accumulator tiles (128 x 128 FP32) and commits them to that tile's mbarrier;
//   * warp w reads TMEM lanes 32 (w % 4) .. + 31 (its queries) and columns
//     32 (w / 4) .. + 31 of the finished tile: four threads per query, each keeping its
//     own list of the KP smallest D = (|q|^2 + |r|^2) - 2 q.r over its quarter of the
//     columns.  The re-rank merges the four lists.
// Xc rows are padded to D floats (zeros), so a row is whole 16-byte chunks.  Waits are
// bounded; a wait that gives up sets DEV_TIMEOUT and the block stops issuing.
constexpr long KT_WAIT = 1L << 22;
template <int D>
__device__ __forceinline__ void stage_operand(const float* Xc, int row0, int nrows, uint32_t* H, uint32_t* L) {
  constexpr int KC = D / 4;
  for (int e = threadIdx.x; e < KT_QB * KC; e += KT_NTH) {
    const int g = e / (8 * KC), rem = e % (8 * KC);
    const int kc = rem / 8, rr = rem % 8;
    const int r = g * 8 + rr;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < nrows) v = *reinterpret_cast<const float4*>(Xc + (size_t)(row0 + r) * D + kc * 4);
    uint4 h, l;
    h.x = tc::to_tf32(v.x);
    h.y = tc::to_tf32(v.y);
    h.z = tc::to_tf32(v.z);
    h.w = tc::to_tf32(v.w);
    l.x = tc::to_tf32(v.x - __uint_as_float(h.x));
    l.y = tc::to_tf32(v.y - __uint_as_float(h.y));
    l.z = tc::to_tf32(v.z - __uint_as_float(h.z));
    l.w = tc::to_tf32(v.w - __uint_as_float(h.w));
    const uint32_t w = (uint32_t)((g * KC + kc) * 32 + rr * 4);  // 32-bit words
    *reinterpret_cast<uint4*>(H + w) = h;
    *reinterpret_cast<uint4*>(L + w) = l;
  }
}

// The next-but-one point tile arrives as raw FP32 rows through asynchronous 16-byte
// copies (cp.async, zero-filled past the end), overlapping the scan of the current
// tile; split_raw then forms its TF32 hi/lo operand from shared memory.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_addr(smem)), "l"(gmem),
               "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
template <int D>
__device__ __forceinline__ void fetch_raw(const float* Xc, int row0, int nrows, float* raw) {
  constexpr int KC = D / 4;
  for (int e = threadIdx.x; e < KT_RB * KC; e += KT_NTH) {
    const int r = e / KC, kc = e % KC;
    const bool ok = r < nrows;
    cp_async16(raw + r * D + kc * 4, ok ? Xc + (size_t)(row0 + r) * D + kc * 4 : Xc, ok);
  }
  cp_async_commit();
}
template <int D>
__device__ __forceinline__ void split_raw(const float* raw, uint32_t* H, uint32_t* L) {
  constexpr int KC = D / 4;
  for (int e = threadIdx.x; e < KT_RB * KC; e += KT_NTH) {
    const int g = e / (8 * KC), rem = e % (8 * KC);
    const int kc = rem / 8, rr = rem % 8;
    const float4 v = *reinterpret_cast<const float4*>(raw + (g * 8 + rr) * D + kc * 4);
    uint4 h, l;
    h.x = tc::to_tf32(v.x);
    h.y = tc::to_tf32(v.y);
    h.z = tc::to_tf32(v.z);
    h.w = tc::to_tf32(v.w);
    l.x = tc::to_tf32(v.x - __uint_as_float(h.x));
    l.y = tc::to_tf32(v.y - __uint_as_float(h.y));
    l.z = tc::to_tf32(v.z - __uint_as_float(h.z));
    l.w = tc::to_tf32(v.w - __uint_as_float(h.w));
    const uint32_t w = (uint32_t)((g * KC + kc) * 32 + rr * 4);  // 32-bit words
    *reinterpret_cast<uint4*>(H + w) = h;
    *reinterpret_cast<uint4*>(L + w) = l;
  }
}

template <int D>
constexpr size_t prefilter_smem() {
  return (size_t)6 * KT_QB * D * 4 + (size_t)KT_RB * D * 4 + 2 * KT_RB * 4 + 64;
}

// With a tile list (tlist, toff: CSR per work tile) the block scans the listed point
// tiles of its problem (local tile t = rows tl.rb + 128 t ..) instead of the whole
// range [tl.rb, tl.rb + tl.rn); with load_init its lists start from the candidates
// already in cand_d / cand_i (an earlier pass over other tiles) instead of empty.
template <int D, int KP>
__global__ void __launch_bounds__(KT_NTH) knn_prefilter_kernel(const float* Xc, const float* qnorm,
                                                               const KnnTile* tiles, const int* tlist,
                                                               const int* toff, int load_init,
                                                               float* cand_d, int* cand_i, int* status) {
  extern __shared__ __align__(1024) unsigned char kt_sh[];
  constexpr int OPW = KT_QB * D;  // 32-bit words of one operand
  uint32_t* Ah = reinterpret_cast<uint32_t*>(kt_sh);
  uint32_t* Al = Ah + OPW;
  uint32_t* Bh0 = Al + OPW;
  uint32_t* Bl0 = Bh0 + OPW;
  uint32_t* Bh1 = Bl0 + OPW;
  uint32_t* Bl1 = Bh1 + OPW;
  float* raw = reinterpret_cast<float*>(Bl1 + OPW);                 // [KT_RB][D]
  float* rn_s = raw + KT_RB * D;                                     // [2][KT_RB]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(rn_s + 2 * KT_RB);   // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  __shared__ int abort_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lq = warp & 3, cq = warp >> 2;  // lane quarter (queries) and column quarter
  const int qi = lq * 32 + lane;
  const KnnTile tl = tiles[blockIdx.x];
  const int my_q = tl.q0 + qi;
  const bool active = qi < tl.qn;
  const int rend = tl.rb + tl.rn;
  const int lbeg = tlist ? toff[blockIdx.x] : 0;
  const int ntile = tlist ? toff[blockIdx.x + 1] - lbeg : (tl.rn + KT_RB - 1) / KT_RB;
  if (ntile == 0) return;  // block-uniform: nothing to scan, the lists stay as they are
  auto tile_row = [&](int t) { return tl.rb + (tlist ? tlist[lbeg + t] : t) * KT_RB; };
  stage_operand<D>(Xc, tl.q0, tl.qn, Ah, Al);
  stage_operand<D>(Xc, tile_row(0), min(KT_RB, rend - tile_row(0)), Bh0, Bl0);
  if (tid < KT_RB) rn_s[tid] = tid < min(KT_RB, rend - tile_row(0)) ? qnorm[tile_row(0) + tid] : 0.0f;
  if (ntile > 1) fetch_raw<D>(Xc, tile_row(1), min(KT_RB, rend - tile_row(1)), raw);
  const float qv = active ? qnorm[my_q] : 0.0f;
  if (warp == 0) tc::tmem_alloc(tslot, 2 * KT_RB);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    abort_s = 0;
  }
  cp_async_wait_all();
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = tc::idesc_tf32(KT_QB, KT_RB);
  constexpr uint32_t SBO = (D / 4) * 128;
  auto issue = [&](int b) {
    const uint32_t* Bh = b ? Bh1 : Bh0;
    const uint32_t* Bl = b ? Bl1 : Bl0;
    const uint32_t dt = tmem + (uint32_t)(b * KT_RB);
#pragma unroll 1
    for (int ks = 0; ks < D / 8; ++ks) {
      const uint32_t ko = (uint32_t)ks * 256;
      const uint64_t ah = tc::smem_desc(tc::smem_addr(Ah) + ko, 128, SBO);
      const uint64_t al = tc::smem_desc(tc::smem_addr(Al) + ko, 128, SBO);
      const uint64_t bh = tc::smem_desc(tc::smem_addr(Bh) + ko, 128, SBO);
      const uint64_t bl = tc::smem_desc(tc::smem_addr(Bl) + ko, 128, SBO);
      tc::mma_tf32(dt, al, bh, idesc, ks > 0);
      tc::mma_tf32(dt, ah, bl, idesc, true);
      tc::mma_tf32(dt, ah, bh, idesc, true);
    }
    tc::mma_commit(&mbar[b]);
  };
  if (tid == 0) issue(0);
  float bd[KP];
  int bi[KP];
#pragma unroll
  for (int u = 0; u < KP; ++u) {
    bd[u] = FLT_MAX;
    bi[u] = INT_MAX;
  }
  if (load_init && active) {
    const size_t o = (size_t)my_q * (KT_SUB * KP) + (size_t)cq * KP;
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      bd[u] = cand_d[o + u];
      bi[u] = cand_i[o + u];
    }
  }
  for (int t = 0; t < ntile; ++t) {
    const int b = t & 1;
    const int r0 = tile_row(t), nt = min(KT_RB, rend - r0);
    if (t + 1 < ntile) {  // the other buffer's last reader, MMA t-1, has completed
      const int r1 = tile_row(t + 1), n1 = min(KT_RB, rend - r1);
      split_raw<D>(raw, b ? Bh0 : Bh1, b ? Bl0 : Bl1);
      if (tid < KT_RB) rn_s[(b ^ 1) * KT_RB + tid] = tid < n1 ? qnorm[r1 + tid] : 0.0f;
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const bool stop = abort_s != 0;
    if (!stop && t + 1 < ntile && tid == 0) issue(b ^ 1);
    if (t + 2 < ntile) {  // every thread is past split_raw: the raw buffer is free
      const int r2 = tile_row(t + 2);
      fetch_raw<D>(Xc, r2, min(KT_RB, rend - r2), raw);
    }
    bool got = false;
    if (!stop) {
      got = tc::mbar_wait(&mbar[b], (uint32_t)((t >> 1) & 1), KT_WAIT);
      if (!got) {
        atomicOr(status, DEV_TIMEOUT);
        abort_s = 1;
      }
    }
    tc::fence_after_sync();
    const bool use = __all_sync(0xffffffffu, got);  // tcgen05.ld needs the whole warp
    if (use) {
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int c0 = cq * 32 + h * 16;
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(b * KT_RB + c0), v);
        // distances of the 16 columns, and the mask of those below the list's bound: the
        // columns that may enter (in range, not the query itself) form one mask per
        // chunk, so a column costs a distance, a compare and a bit
        unsigned ok = !active || c0 >= nt ? 0u : (nt - c0 >= 16 ? 0xFFFFu : (1u << (nt - c0)) - 1u);
        const int self = my_q - (r0 + c0);
        if (self >= 0 && self < 16) ok &= ~(1u << self);
        const float bound = bd[KP - 1];
        const float4* rn4 = reinterpret_cast<const float4*>(rn_s + b * KT_RB + c0);
        unsigned mask = 0;
#pragma unroll
        for (int j4 = 0; j4 < 4; ++j4) {
          const float4 r4 = rn4[j4];
          const float rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = 4 * j4 + u;
            v[j] = (qv + rr[u]) - 2.0f * v[j];
            mask |= (v[j] <= bound ? 1u : 0u) << j;
          }
        }
        mask &= ok;
        // insertions are rare: one copy of the insertion chain, column by column
        while (mask) {
          const int j = __ffs(mask) - 1;
          mask &= mask - 1;
          float cv = v[0];
#pragma unroll
          for (int u = 1; u < 16; ++u) cv = (u == j) ? v[u] : cv;
          int cj = r0 + c0 + j;
          if (!(cv <= bd[KP - 1])) continue;
#pragma unroll
          for (int u = 0; u < KP; ++u) {
            const bool less = cv < bd[u] || (cv == bd[u] && cj < bi[u]);
            const float tv = less ? bd[u] : cv;
            const int tj = less ? bi[u] : cj;
            bd[u] = less ? cv : bd[u];
            bi[u] = less ? cj : bi[u];
            cv = tv;
            cj = tj;
          }
        }
      }
    }
    cp_async_wait_all();  // the next tile's raw rows have landed (this thread's copies)
    tc::fence_before_sync();
    __syncthreads();  // rn_s and the TMEM tile are reused two tiles later; raw is complete
  }
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_free(tmem, 2 * KT_RB);
  if (active) {
    const size_t o = (size_t)my_q * (KT_SUB * KP) + (size_t)cq * KP;
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      cand_d[o + u] = bd[u];
      cand_i[o + u] = bi[u];
    }
  }
}

// ------------------------------------------------- prefilter on pre-split tile records
// The tree-order search converts every 128-row tile once per call into a record: the
// TF32 hi and lo parts of its centred FP32 rows in the operand layout of the tensor-core
// descriptors (8-row x 16-byte core matrices), then (separately) the tile's 128 row
// norms, rows past the tile's end zero.  A block then brings each point tile in with
// one bulk copy (cp.async.bulk, mbarrier completion) instead of splitting it itself.
template <int D>
constexpr uint32_t rec_bytes() { return (uint32_t)(2 * KT_RB * D * 4); }

template <int D>
__global__ void knn_records_kernel(const float* Xc, const float* qnorm, const KnnTile* tiles, uint32_t* rec,
                                   float* tnorm) {
  constexpr int KC = D / 4;
  const KnnTile tl = tiles[blockIdx.x];
  uint32_t* H = rec + (size_t)blockIdx.x * (rec_bytes<D>() / 4);
  uint32_t* L = H + KT_RB * D;
  for (int e = threadIdx.x; e < KT_RB * KC; e += blockDim.x) {
    const int g = e / (8 * KC), rem = e % (8 * KC);
    const int kc = rem / 8, rr = rem % 8;
    const int r = g * 8 + rr;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < tl.qn) v = *reinterpret_cast<const float4*>(Xc + (size_t)(tl.q0 + r) * D + kc * 4);
    uint4 h, l;
    h.x = tc::to_tf32(v.x);
    h.y = tc::to_tf32(v.y);
    h.z = tc::to_tf32(v.z);
    h.w = tc::to_tf32(v.w);
    l.x = tc::to_tf32(v.x - __uint_as_float(h.x));
    l.y = tc::to_tf32(v.y - __uint_as_float(h.y));
    l.z = tc::to_tf32(v.z - __uint_as_float(h.z));
    l.w = tc::to_tf32(v.w - __uint_as_float(h.w));
    const uint32_t w = (uint32_t)((g * KC + kc) * 32 + rr * 4);
    *reinterpret_cast<uint4*>(H + w) = h;
    *reinterpret_cast<uint4*>(L + w) = l;
  }
  for (int r = threadIdx.x; r < KT_RB; r += blockDim.x)
    tnorm[(size_t)blockIdx.x * KT_RB + r] = r < tl.qn ? qnorm[tl.q0 + r] : 0.0f;
}

// The prefilter of knn_prefilter_kernel (same lists, same arithmetic) over tile records:
// the query block is the record of its own tile; the point tile of step t (local index
// tlist[..] or t, record first_tile[prob] + local) arrives by bulk copy into one of two
// operand buffers, its norms into one of PF_NSLOT slots.  Warp 16 (one thread) issues
// the copies and the MMAs: tile t's products go to accumulator t % NACC (NACC = 4 TMEM
// accumulators of 128 columns for D >= 32, else 2) as soon as its operands have arrived
// and every warp has finished scanning the tile that used that accumulator before
// (mbarrier arrivals, one per warp), and tile t + 2's copy starts once MMA t has read
// its operand buffer.  Warps 0-15 scan accumulator after accumulator at their own pace:
// no block barrier per tile, so a warp whose list insertions run long no longer holds up
// the others, and the products run up to NACC - 1 tiles ahead of the slowest warp.
// Waits are bounded; a wait that gives up sets DEV_TIMEOUT, the block stops issuing,
// waits (bounded) for its MMAs and copies in flight, frees its TMEM and returns.
constexpr int PF_NSLOT = 8;  // norm slots: refilled only after every warp scanned their tile
template <int D>
constexpr int pf_nacc() { return D >= 32 ? 4 : 2; }
template <int D>
constexpr size_t prefilter2_smem() {
  return (size_t)3 * rec_bytes<D>() + (size_t)PF_NSLOT * KT_RB * 4 + 64;
}
static_assert(PF_NSLOT - 2 >= 4, "a norm slot is refilled after the scans of its tile");

template <int D, int KP>
__global__ void __launch_bounds__(KT_NTH + 32) knn_prefilter2_kernel(const uint32_t* rec, const float* tnorm,
                                                                     const KnnTile* tiles, const int* first_tile,
                                                                     const int* tlist, const int* toff,
                                                                     int load_init, float* cand_d, int* cand_i,
                                                                     int* status) {
  extern __shared__ __align__(1024) unsigned char kt_sh[];
  constexpr uint32_t RB = rec_bytes<D>();
  constexpr int OPW = KT_QB * D;  // 32-bit words of one operand (hi or lo)
  constexpr int NACC = pf_nacc<D>();
  uint32_t* Ah = reinterpret_cast<uint32_t*>(kt_sh);
  uint32_t* Al = Ah + OPW;
  uint32_t* B0 = Al + OPW;  // operand buffer b at B0 + 2 b OPW: hi, then lo
  float* rns = reinterpret_cast<float*>(Al + OPW + 4 * OPW);  // [PF_NSLOT][KT_RB]
  __shared__ uint64_t qbar, full[2], opfree[2], nfull[PF_NSLOT], mmadone[NACC], accfree[NACC], fin;
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lq = warp & 3, cq = (warp >> 2) & 3;
  const int qi = lq * 32 + lane;
  const KnnTile tl = tiles[blockIdx.x];
  const int my_q = tl.q0 + qi;
  const bool scanner = warp < 16;
  const bool active = scanner && qi < tl.qn;
  const int rend = tl.rb + tl.rn;
  const int lbeg = tlist ? toff[blockIdx.x] : 0;
  const int ntile = tlist ? toff[blockIdx.x + 1] - lbeg : (tl.rn + KT_RB - 1) / KT_RB;
  if (ntile == 0) return;  // block-uniform: nothing to scan, the lists stay as they are
  const int ft = first_tile[tl.prob];
  auto local = [&](int t) { return tlist ? tlist[lbeg + t] : t; };
  if (warp == 0) tc::tmem_alloc(&tslot, NACC * KT_RB);
  if (tid == 0) {
    tc::mbar_init(&qbar, 1);
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&opfree[i], 1);
    }
    for (int i = 0; i < PF_NSLOT; ++i) tc::mbar_init(&nfull[i], 1);
    for (int i = 0; i < NACC; ++i) {
      tc::mbar_init(&mmadone[i], 1);
      tc::mbar_init(&accfree[i], 16);
    }
    tc::mbar_init(&fin, 1);
    abort_s = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  float bd[KP];
  int bi[KP];
  if (warp == 16) {
    if (lane == 0) {
      // tile t: operands into buffer t & 1 (full), norms into slot t % PF_NSLOT (nfull)
      auto load = [&](int t) {
        const int b = t & 1, r = ft + local(t);
        tc::mbar_expect_tx(&full[b], RB);
        tc::bulk_g2s(B0 + 2 * b * OPW, rec + (size_t)r * (RB / 4), RB, &full[b]);
        tc::mbar_expect_tx(&nfull[t % PF_NSLOT], KT_RB * 4);
        tc::bulk_g2s(rns + (t % PF_NSLOT) * KT_RB, tnorm + (size_t)r * KT_RB, KT_RB * 4, &nfull[t % PF_NSLOT]);
      };
      auto wait = [&](uint64_t* bar, uint32_t par) {
        for (long it = 0; it < KT_WAIT; it += 64) {
          if (tc::mbar_wait(bar, par, 64)) return true;
          if (abort_s) return false;
        }
        return false;
      };
      constexpr uint32_t idesc = tc::idesc_tf32(KT_QB, KT_RB);
      constexpr uint32_t SBO = (D / 4) * 128;
      tc::mbar_expect_tx(&qbar, RB);
      tc::bulk_g2s(Ah, rec + (size_t)blockIdx.x * (RB / 4), RB, &qbar);
      int loaded = 0, issued = 0;
      load(0);
      loaded = 1;
      if (ntile > 1) {
        load(1);
        loaded = 2;
      }
      bool ok = wait(&qbar, 0);
      for (int t = 0; t < ntile && ok; ++t) {
        const int b = t & 1, a = t % NACC;
        ok = wait(&full[b], (uint32_t)((t >> 1) & 1));
        // the accumulator's previous tile (t - NACC) has been scanned by every warp; that
        // also frees the norm slot of tile t + 2 (PF_NSLOT - 2 >= NACC)
        if (ok && t >= NACC) ok = wait(&accfree[a], (uint32_t)((t / NACC - 1) & 1));
        if (!ok) break;
        tc::fence_after_sync();
        const uint32_t dt = tmem + (uint32_t)(a * KT_RB);
#pragma unroll 1
        for (int ks = 0; ks < D / 8; ++ks) {
          const uint32_t ko = (uint32_t)ks * 256;
          const uint64_t ah = tc::smem_desc(tc::smem_addr(Ah) + ko, 128, SBO);
          const uint64_t al = tc::smem_desc(tc::smem_addr(Al) + ko, 128, SBO);
          const uint64_t bh = tc::smem_desc(tc::smem_addr(B0 + 2 * b * OPW) + ko, 128, SBO);
          const uint64_t bl = tc::smem_desc(tc::smem_addr(B0 + 2 * b * OPW + OPW) + ko, 128, SBO);
          tc::mma_tf32(dt, al, bh, idesc, ks > 0);
          tc::mma_tf32(dt, ah, bl, idesc, true);
          tc::mma_tf32(dt, ah, bh, idesc, true);
        }
        tc::mma_commit(&mmadone[a]);
        tc::mma_commit(&opfree[b]);
        issued = t + 1;
        if (t + 2 < ntile) {  // MMA t releases operand buffer b for tile t + 2
          ok = wait(&opfree[b], (uint32_t)((t >> 1) & 1));
          if (!ok) break;
          load(t + 2);
          loaded = t + 3;
        }
      }
      if (!ok) {
        if (!abort_s) {
          atomicOr(status, DEV_TIMEOUT);
          abort_s = 1;
        }
        tc::mma_commit(&fin);  // every MMA issued so far, then the copies that may be in flight:
        tc::mbar_wait(&fin, 0, KT_WAIT);  // operands not yet consumed, norms of the last slots
        for (int u = issued; u < loaded; ++u)
          if (!tc::mbar_wait(&full[u & 1], (uint32_t)((u >> 1) & 1), KT_WAIT)) break;
        for (int u = max(0, loaded - PF_NSLOT); u < loaded; ++u)
          if (!tc::mbar_wait(&nfull[u % PF_NSLOT], (uint32_t)((u / PF_NSLOT) & 1), KT_WAIT)) break;
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      bd[u] = FLT_MAX;
      bi[u] = INT_MAX;
    }
    if (load_init && active) {
      const size_t o = (size_t)my_q * (KT_SUB * KP) + (size_t)cq * KP;
#pragma unroll
      for (int u = 0; u < KP; ++u) {
        bd[u] = cand_d[o + u];
        bi[u] = cand_i[o + u];
      }
    }
    const float qv = active ? tnorm[(size_t)blockIdx.x * KT_RB + qi] : 0.0f;
    for (int t = 0; t < ntile; ++t) {
      const int a = t % NACC, slot = t % PF_NSLOT;
      bool got = false;
      for (long it = 0; it < KT_WAIT && !got; it += 64) {
        got = tc::mbar_wait(&mmadone[a], (uint32_t)((t / NACC) & 1), 64) &&
              tc::mbar_wait(&nfull[slot], (uint32_t)((t / PF_NSLOT) & 1), 64);
        if (abort_s) break;
      }
      if (!__all_sync(0xffffffffu, got)) {  // tcgen05.ld needs the whole warp
        if (lane == 0 && !abort_s) {
          atomicOr(status, DEV_TIMEOUT);
          abort_s = 1;
        }
        break;
      }
      tc::fence_after_sync();
      const int r0 = tl.rb + local(t) * KT_RB, nt = min(KT_RB, rend - r0);
      const float* rn_t = rns + slot * KT_RB;
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int c0 = cq * 32 + h * 16;
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(a * KT_RB + c0), v);
        unsigned ok = !active || c0 >= nt ? 0u : (nt - c0 >= 16 ? 0xFFFFu : (1u << (nt - c0)) - 1u);
        const int self = my_q - (r0 + c0);
        if (self >= 0 && self < 16) ok &= ~(1u << self);
        const float bound = bd[KP - 1];
        const float4* rn4 = reinterpret_cast<const float4*>(rn_t + c0);
        unsigned mask = 0;
#pragma unroll
        for (int j4 = 0; j4 < 4; ++j4) {
          const float4 r4 = rn4[j4];
          const float rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = 4 * j4 + u;
            v[j] = (qv + rr[u]) - 2.0f * v[j];
            mask |= (v[j] <= bound ? 1u : 0u) << j;
          }
        }
        mask &= ok;
        while (mask) {
          const int j = __ffs(mask) - 1;
          mask &= mask - 1;
          float cv = v[0];
#pragma unroll
          for (int u = 1; u < 16; ++u) cv = (u == j) ? v[u] : cv;
          int cj = r0 + c0 + j;
          if (!(cv <= bd[KP - 1])) continue;
#pragma unroll
          for (int u = 0; u < KP; ++u) {
            const bool less = cv < bd[u] || (cv == bd[u] && cj < bi[u]);
            const float tv = less ? bd[u] : cv;
            const int tj = less ? bi[u] : cj;
            bd[u] = less ? cv : bd[u];
            bi[u] = less ? cj : bi[u];
            cv = tv;
            cj = tj;
          }
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&accfree[a]);  // this warp is done with accumulator a and slot
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_free(tmem, NACC * KT_RB);
  if (active) {
    const size_t o = (size_t)my_q * (KT_SUB * KP) + (size_t)cq * KP;
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      cand_d[o + u] = bd[u];
      cand_i[o + u] = bi[u];
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

// One block of KT_QB threads per work tile, one thread per query.  Its KT_SUB lists of
// KP candidates are merged: exact FP64 distances, the kappa smallest by (distance,
// index) kept by insertion.  Every point outside the lists has D >= the smallest of
// the lists' last values (a list that is not full holds all of its quarter's points).
// Kdim is the padded dimension of the prefilter (its accumulation length).
constexpr int RR_MAXK = 48;
// Rows may be in any order: ids[r] is the original index of row r (null: r itself);
// ties are broken and the lists written in original indices, at row ids[i].  With
// tau (the pruned search) the points of the tiles that were not scanned are known to
// lie farther than tau[i] (exact FP64), so a list is certified only if its kappa-th
// distance is <= tau[i] as well.
template <int KP, int KAP>  // KAP >= kappa: size of the sorted list
__global__ void knn_rerank_kernel(const double* X, int d, int kappa, int Kdim, const KnnTile* tiles,
                                  const float* cand_d, const int* cand_i, const float* qnorm,
                                  const unsigned* rmax_bits, const int* ids, const double* tau, int* knn,
                                  int2* flagged, int* nflagged) {
  const KnnTile tl = tiles[blockIdx.x];
  if ((int)threadIdx.x >= tl.qn) return;
  const int i = tl.q0 + threadIdx.x;
  const int N = tl.rn, rb = tl.rb;
  double dd[KAP];
  int ii[KAP];
#pragma unroll
  for (int u = 0; u < KAP; ++u) {
    dd[u] = DBL_MAX;
    ii[u] = INT_MAX;
  }
  const double* xi = X + (size_t)i * d;
  const size_t o = (size_t)i * (KT_SUB * KP);
  const double c = (8.0 * Kdim + 32.0) * 1.1920928955078125e-07;  // (8K + 32) 2^-23
  const double a2 = (double)qnorm[i];
  // pass 1: every candidate's exact distance lies within D +- E_j, E_j = c (|a|^2 + |b_j|^2);
  // U = the kappa-th smallest D + E_j bounds the kappa-th smallest exact distance
  float cut = FLT_MAX;
  int found = 0;
  double ub[KAP];
#pragma unroll
  for (int u = 0; u < KAP; ++u) ub[u] = DBL_MAX;
  for (int q = 0; q < KT_SUB; ++q) {
    cut = fminf(cut, cand_d[o + (size_t)q * KP + KP - 1]);
    for (int u = 0; u < KP; ++u) {
      const int j = cand_i[o + (size_t)q * KP + u];
      if (j == INT_MAX) break;  // the rest of this list is empty
      if (j < rb || j >= rb + N) {  // cannot happen with finite norms; redo exactly
        int slot = atomicAdd(nflagged, 1);
        flagged[slot] = make_int2(i, blockIdx.x);
        return;
      }
      ++found;
      double v = (double)cand_d[o + (size_t)q * KP + u] + c * (a2 + (double)qnorm[j]);
      if (!(v < ub[kappa - 1])) continue;
#pragma unroll
      for (int w = 0; w < KAP; ++w) {
        if (w >= kappa) break;
        if (v < ub[w]) {
          const double tv = ub[w];
          ub[w] = v;
          v = tv;
        }
      }
    }
  }
  const double U = found >= kappa ? ub[kappa - 1] * (1.0 + 1e-12) : DBL_MAX;
  // pass 2: exact distances of the candidates that can be among the kappa nearest; one
  // whose D - E_j exceeds U is strictly farther than the kappa-th (no tie with it)
  for (int q = 0; q < KT_SUB; ++q) {
    for (int u = 0; u < KP; ++u) {
      const int j = cand_i[o + (size_t)q * KP + u];
      if (j == INT_MAX) break;
      const double lbj = ((double)cand_d[o + (size_t)q * KP + u] - c * (a2 + (double)qnorm[j])) * (1.0 - 1e-12);
      if (lbj > U) continue;
      double v = exact_sqdist(xi, X + (size_t)j * d, d);
      int jj = ids ? ids[j] : j;
      if (!pair_less(v, jj, dd[kappa - 1], ii[kappa - 1])) continue;
#pragma unroll
      for (int w = 0; w < KAP; ++w) {  // insertion into the sorted kappa list
        if (w >= kappa) break;
        if (pair_less(v, jj, dd[w], ii[w])) {
          const double tv = dd[w];
          const int tj = ii[w];
          dd[w] = v;
          ii[w] = jj;
          v = tv;
          jj = tj;
        }
      }
    }
  }
  const double E = c * ((double)qnorm[i] + (double)__uint_as_float(rmax_bits[tl.prob]));
  const bool all_in = found >= N - 1;  // every other point was a candidate
  const double lo = ((double)cut - E) * (1.0 - 1e-12);
  const bool ok = found >= kappa && isfinite(E) && (all_in || lo > dd[kappa - 1]) &&
                  (tau == nullptr || all_in || dd[kappa - 1] <= tau[i]);
  if (!ok) {
    int slot = atomicAdd(nflagged, 1);
    flagged[slot] = make_int2(i, blockIdx.x);
    return;
  }
  const size_t orow = (size_t)(ids ? ids[i] : i);
  for (int u = 0; u < kappa; ++u) knn[orow * kappa + u] = ii[u];
}

// Exact scan for one flagged query per block: every thread keeps a sorted top-kappa
// list of its strided share of the points, then kappa rounds of a block-wide argmin
// over the list heads merge them.
constexpr int FB_THREADS = 128;
constexpr int FB_MAXK = 64;
__global__ void knn_fallback_kernel(const double* X, int d, int kappa, const KnnTile* tiles,
                                    const int2* flagged, const int* ids, int* knn) {
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
  for (int r = r_begin + threadIdx.x; r < r_end; r += FB_THREADS) {
    if (r == i) continue;
    double v = exact_sqdist(xi, X + (size_t)r * d, d);
    const int j = ids ? ids[r] : r;
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
  const size_t orow = (size_t)(ids ? ids[i] : i);
  for (int t = threadIdx.x; t < kappa; t += FB_THREADS) knn[orow * kappa + t] = chosen[t];
}

// Tile list of one prefilter pass: none (every block scans its whole range), or CSR
// per block with the lists starting from the candidates of an earlier pass.
struct TileList {
  const int* tlist = nullptr;
  const int* toff = nullptr;
  int load_init = 0;
};

template <int D, int KP>
void launch_prefilter(const float* Xc, const float* qn, const KnnTile* tiles, int ntiles, float* cd, int* ci,
                      int* status, cudaStream_t st, TileList tl = TileList{}) {
  // at least 80 KB so that at most two blocks share an SM's 512 TMEM columns
  const size_t smem = std::max<size_t>(prefilter_smem<D>(), 80 * 1024);
  IA_CUDA(cudaFuncSetAttribute(knn_prefilter_kernel<D, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  knn_prefilter_kernel<D, KP><<<ntiles, KT_NTH, smem, st>>>(Xc, qn, tiles, tl.tlist, tl.toff, tl.load_init, cd,
                                                             ci, status);
  IA_LAUNCH_CHECK();
}

// Padded dimension (multiple of 8) of the prefilter for d.
int padded_dim(int d) { return (d + 7) / 8 * 8; }

template <int KP>
void prefilter_dispatch(const float* Xc, const float* qn, int d, const KnnTile* tl, int nt, float* cd, int* ci,
                        int* status, cudaStream_t st, TileList list = TileList{}) {
  switch (padded_dim(d)) {
    case 8: launch_prefilter<8, KP>(Xc, qn, tl, nt, cd, ci, status, st, list); break;
    case 16: launch_prefilter<16, KP>(Xc, qn, tl, nt, cd, ci, status, st, list); break;
    case 24: launch_prefilter<24, KP>(Xc, qn, tl, nt, cd, ci, status, st, list); break;
    case 32: launch_prefilter<32, KP>(Xc, qn, tl, nt, cd, ci, status, st, list); break;
    case 40: launch_prefilter<40, KP>(Xc, qn, tl, nt, cd, ci, status, st, list); break;
    case 48: launch_prefilter<48, KP>(Xc, qn, tl, nt, cd, ci, status, st, list); break;
    case 56: launch_prefilter<56, KP>(Xc, qn, tl, nt, cd, ci, status, st, list); break;
    case 64: launch_prefilter<64, KP>(Xc, qn, tl, nt, cd, ci, status, st, list); break;
    default: throw Error(IASKIT_ERR_UNSUPPORTED, "kNN supports d <= 64");
  }
}

// Records of every tile for the tree-order search, and its prefilter on them.
template <int D, int KP>
void launch_prefilter2(const uint32_t* rec, const float* tn, const KnnTile* tiles, const int* first, int ntiles,
                       float* cd, int* ci, int* status, cudaStream_t st, TileList tl) {
  // with 4 accumulators (512 TMEM columns) a block must hold its SM alone: at least 116 KB
  const size_t smem = std::max<size_t>(prefilter2_smem<D>(), pf_nacc<D>() > 2 ? 116 * 1024 : 80 * 1024);
  IA_CUDA(cudaFuncSetAttribute(knn_prefilter2_kernel<D, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  knn_prefilter2_kernel<D, KP><<<ntiles, KT_NTH + 32, smem, st>>>(rec, tn, tiles, first, tl.tlist, tl.toff, tl.load_init,
                                                              cd, ci, status);
  IA_LAUNCH_CHECK();
}

template <int D>
void make_records(const float* Xc, const float* qn, const KnnTile* tiles, int ntiles, uint32_t* rec, float* tn,
                  cudaStream_t st) {
  knn_records_kernel<D><<<ntiles, 256, 0, st>>>(Xc, qn, tiles, rec, tn);
  IA_LAUNCH_CHECK();
}

#define IA_KNN_DIMS(X) X(8) X(16) X(24) X(32) X(40) X(48) X(56) X(64)

void records_dispatch(int Dp, const float* Xc, const float* qn, const KnnTile* tiles, int ntiles, uint32_t* rec,
                      float* tn, cudaStream_t st) {
  switch (Dp) {
#define IA_CASE(D) \
  case D: make_records<D>(Xc, qn, tiles, ntiles, rec, tn, st); break;
    IA_KNN_DIMS(IA_CASE)
#undef IA_CASE
    default: throw Error(IASKIT_ERR_UNSUPPORTED, "kNN supports d <= 64");
  }
}

template <int KP>
void prefilter2_dispatch(int Dp, const uint32_t* rec, const float* tn, const KnnTile* tiles, const int* first,
                         int ntiles, float* cd, int* ci, int* status, cudaStream_t st, TileList tl) {
  switch (Dp) {
#define IA_CASE(D) \
  case D: launch_prefilter2<D, KP>(rec, tn, tiles, first, ntiles, cd, ci, status, st, tl); break;
    IA_KNN_DIMS(IA_CASE)
#undef IA_CASE
    default: throw Error(IASKIT_ERR_UNSUPPORTED, "kNN supports d <= 64");
  }
}

// Scratch pointers of one kNN run (the allocating and the allocation-free callers).
struct KnnBufs {
  int* status;  // device word: DEV_TIMEOUT when a bounded wait gave up
  float* Xc;    // N x padded_dim(d)
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
  IA_CUDA(cudaMemsetAsync(b.status, 0, sizeof(int), st));
  center_partial_kernel<<<dim3(KC_CHUNKS, np), 64, 0, st>>>(X, d, b.probs, b.part);
  IA_LAUNCH_CHECK();
  center_mean_kernel<<<np, 64, 0, st>>>(d, b.probs, b.part, b.mean);
  IA_LAUNCH_CHECK();
  center_points_kernel<<<nt, KT_QB, 0, st>>>(X, d, padded_dim(d), b.tiles, b.mean, b.Xc, b.qn, b.rmax);
  IA_LAUNCH_CHECK();
  prefilter_dispatch<KP>(b.Xc, b.qn, d, b.tiles, nt, b.cd, b.ci, b.status, st);
  if (kappa <= 16)
    knn_rerank_kernel<KP, 16><<<nt, KT_QB, 0, st>>>(X, d, kappa, padded_dim(d), b.tiles, b.cd, b.ci, b.qn,
                                                    b.rmax, nullptr, nullptr, knn, b.flagged, b.nfl);
  else if (kappa <= 32)
    knn_rerank_kernel<KP, 32><<<nt, KT_QB, 0, st>>>(X, d, kappa, padded_dim(d), b.tiles, b.cd, b.ci, b.qn,
                                                    b.rmax, nullptr, nullptr, knn, b.flagged, b.nfl);
  else
    knn_rerank_kernel<KP, RR_MAXK><<<nt, KT_QB, 0, st>>>(X, d, kappa, padded_dim(d), b.tiles, b.cd, b.ci,
                                                         b.qn, b.rmax, nullptr, nullptr, knn, b.flagged, b.nfl);
  IA_LAUNCH_CHECK();
  int nf = 0, dev_status = 0;
  IA_CUDA(cudaMemcpyAsync(&nf, b.nfl, sizeof(int), cudaMemcpyDeviceToHost, st));
  IA_CUDA(cudaMemcpyAsync(&dev_status, b.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  IA_CUDA(cudaStreamSynchronize(st));
  if (dev_status & DEV_TIMEOUT) throw Error(IASKIT_ERR_TIMEOUT, "kNN tensor-core wait expired");
  if (nf > 0) {
    knn_fallback_kernel<<<nf, FB_THREADS, 0, st>>>(X, d, kappa, b.tiles, b.flagged, nullptr, knn);
    IA_LAUNCH_CHECK();
  }
  return nf;
}

// ----------------------------------------------------- tree-order search with pruning
// The points are searched in the order of a tree with leaves of at most 128 points, so
// every 128-row tile is a compact box.  Each block of 128 queries first scans its seed
// tiles (the SEED_TILES tiles whose boxes lie nearest to its own, its own first), which
// gives every query an upper bound tau on its kappa-th distance; a point tile whose box
// lies farther than the block's largest tau from the block's own box cannot hold a
// neighbour of any of its queries and is not scanned.
constexpr int SEED_TILES = 8;

// FP32 lower bound of the squared distance between two boxes (minima, then maxima),
// every operation rounded down.
__device__ __forceinline__ float box_lower_bound(const float* a, const float* b, int d) {
  float lb = 0.0f;
  for (int k = 0; k < d; ++k) {
    const float gap = fmaxf(0.0f, fmaxf(__fsub_rd(b[k], a[d + k]), __fsub_rd(a[k], b[d + k])));
    lb = __fadd_rd(lb, __fmul_rd(gap, gap));
  }
  return lb;
}

// Bounding box of every 128-row tile in FP32, rounded outward (minima rounded down,
// maxima up, so the box contains the FP64 points): box[g][0 .. d) = minima,
// box[g][d .. 2d) = maxima; the same coordinate-major in boxT[k NT + g] (minima) and
// boxT[(d + k) NT + g] (maxima), NT tiles, for scans of many tiles by one warp.
__global__ void tile_box_kernel(const double* X, int d, const KnnTile* tiles, int NT, float* box, float* boxT) {
  const KnnTile tl = tiles[blockIdx.x];
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double lo = DBL_MAX, hi = -DBL_MAX;
    for (int r = 0; r < tl.qn; ++r) {
      const double v = X[(size_t)(tl.q0 + r) * d + k];
      lo = fmin(lo, v);
      hi = fmax(hi, v);
    }
    const float flo = __double2float_rd(lo), fhi = __double2float_ru(hi);
    box[(size_t)blockIdx.x * 2 * d + k] = flo;
    box[(size_t)blockIdx.x * 2 * d + d + k] = fhi;
    boxT[(size_t)k * NT + blockIdx.x] = flo;
    boxT[(size_t)(d + k) * NT + blockIdx.x] = fhi;
  }
}

// Box of every group of SEL_GROUP consecutive tiles of a problem (the union of their
// boxes): grp[j] = (first global tile, count); sbox[j][0 .. 2d) as box.
constexpr int SEL_GROUP = 32;
__global__ void super_box_kernel(const float* box, int d, const int2* grp, float* sbox) {
  const int2 G = grp[blockIdx.x];
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    float lo = FLT_MAX, hi = -FLT_MAX;
    for (int t = 0; t < G.y; ++t) {
      lo = fminf(lo, box[(size_t)(G.x + t) * 2 * d + k]);
      hi = fmaxf(hi, box[(size_t)(G.x + t) * 2 * d + d + k]);
    }
    sbox[(size_t)blockIdx.x * 2 * d + k] = lo;
    sbox[(size_t)blockIdx.x * 2 * d + d + k] = hi;
  }
}

// box_lower_bound of box a against tile g of the coordinate-major boxes.
__device__ __forceinline__ float box_lower_bound_T(const float* a, const float* boxT, size_t NT, int g, int d) {
  float lb = 0.0f;
  for (int k = 0; k < d; ++k) {
    const float blo = boxT[(size_t)k * NT + g], bhi = boxT[(size_t)(d + k) * NT + g];
    const float gap = fmaxf(0.0f, fmaxf(__fsub_rd(blo, a[d + k]), __fsub_rd(a[k], bhi)));
    lb = __fadd_rd(lb, __fmul_rd(gap, gap));
  }
  return lb;
}

// Seed tiles of block g: the min(SEED_TILES, tiles of its problem) tiles whose boxes have
// the smallest lower bound from g's box, by (bound, tile index), g's own tile first;
// written as local tile indices at soff[g].
__global__ void knn_seed_pick_kernel(const KnnTile* tiles, const int* first_tile, const float* box,
                                     const float* boxT, int NT, int d, const int* soff, int* seeds) {
  __shared__ float hv[KT_QB];
  __shared__ int ht[KT_QB], hs[KT_QB];
  __shared__ int chosen_s;
  const int g = blockIdx.x;
  const KnnTile tl = tiles[g];
  const int ft = first_tile[tl.prob];
  const int nt = (tl.rn + KT_RB - 1) / KT_RB;
  const int ns = min(SEED_TILES, nt);
  const float* bq = box + (size_t)g * 2 * d;
  float lv[SEED_TILES];
  int lt[SEED_TILES];
#pragma unroll
  for (int u = 0; u < SEED_TILES; ++u) {
    lv[u] = FLT_MAX;
    lt[u] = INT_MAX;
  }
  for (int t = threadIdx.x; t < nt; t += KT_QB) {
    float v = ft + t == g ? -1.0f : box_lower_bound_T(bq, boxT, NT, ft + t, d);
    int tt = t;
#pragma unroll
    for (int u = 0; u < SEED_TILES; ++u) {  // sorted insertion by (bound, index)
      const bool less = v < lv[u] || (v == lv[u] && tt < lt[u]);
      const float pv = lv[u];
      const int pt = lt[u];
      lv[u] = less ? v : pv;
      lt[u] = less ? tt : pt;
      v = less ? pv : v;
      tt = less ? pt : tt;
    }
  }
  int head = 0;
  for (int r = 0; r < ns; ++r) {  // ns rounds of a block-wide argmin over the list heads
    hv[threadIdx.x] = head < SEED_TILES ? lv[head] : FLT_MAX;
    ht[threadIdx.x] = head < SEED_TILES ? lt[head] : INT_MAX;
    hs[threadIdx.x] = threadIdx.x;
    __syncthreads();
    for (int w = KT_QB / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        const int o = threadIdx.x + w;
        if (hv[o] < hv[threadIdx.x] || (hv[o] == hv[threadIdx.x] && ht[o] < ht[threadIdx.x])) {
          hv[threadIdx.x] = hv[o];
          ht[threadIdx.x] = ht[o];
          hs[threadIdx.x] = hs[o];
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      seeds[soff[g] + r] = ht[0];
      chosen_s = hs[0];
    }
    __syncthreads();
    if ((int)threadIdx.x == chosen_s) ++head;
    __syncthreads();
  }
}

// tau[i] = an upper bound on the kappa-th smallest exact FP64 distance among the
// candidates of the seed pass (so on the true kappa-th distance; DBL_MAX when fewer than
// kappa), and Tq[g] = the largest tau of block g.  It needs no FP64 distance: by the
// prefilter's rounding bound every candidate's exact distance is at most
// D + E, E = (8 K + 32) 2^-23 (|a|^2 + |b|^2) (K = Kdim, the norms those of the centred
// FP32 rows), so the kappa-th smallest D + E bounds the kappa-th smallest exact distance
// (a factor 1 + 1e-12 covers the FP64 distances' own rounding).  A larger tau only scans
// a few more tiles; the re-rank certifies every list against it as before.
template <int KP, int KAP>
__global__ void knn_seed_bound_kernel(const float* qnorm, int Kdim, int kappa, const KnnTile* tiles,
                                      const float* cand_d, const int* cand_i, double* tau, double* Tq) {
  __shared__ double red[KT_QB];
  const KnnTile tl = tiles[blockIdx.x];
  const int t = threadIdx.x;
  const double ef = (8.0 * Kdim + 32.0) * 0x1p-23;
  double bound = 0.0;
  if (t < tl.qn) {
    const int i = tl.q0 + t;
    const double a2 = (double)qnorm[i];
    double dd[KAP];
#pragma unroll
    for (int u = 0; u < KAP; ++u) dd[u] = DBL_MAX;
    const size_t o = (size_t)i * (KT_SUB * KP);
    int found = 0;
    for (int q = 0; q < KT_SUB; ++q)
      for (int u = 0; u < KP; ++u) {
        const int j = cand_i[o + (size_t)q * KP + u];
        if (j == INT_MAX) break;
        ++found;
        double v = (double)cand_d[o + (size_t)q * KP + u] + ef * (a2 + (double)qnorm[j]);
        if (!(v < dd[kappa - 1])) continue;
#pragma unroll
        for (int w = 0; w < KAP; ++w) {
          if (w >= kappa) break;
          if (v < dd[w]) {
            const double tv = dd[w];
            dd[w] = v;
            v = tv;
          }
        }
      }
    bound = found >= kappa ? dd[kappa - 1] * (1.0 + 1e-12) : DBL_MAX;
    tau[i] = bound;
  }
  red[t] = bound;
  __syncthreads();
  for (int s = KT_QB / 2; s > 0; s >>= 1) {
    if (t < s) red[t] = fmax(red[t], red[t + s]);
    __syncthreads();
  }
  if (t == 0) Tq[blockIdx.x] = red[0];
}

// Point tiles that block g must scan after its seed tiles: every other tile t of its
// problem that may hold a neighbour of one of g's queries.  A tile is skipped when, for
// every query q of g, the distance from q to the tile's box, a lower bound on q's
// distance to any point of the tile, exceeds tau_q (1 + 1e-9): first the cheap test on
// g's whole box against the largest tau (Tq), then, for the tiles it keeps, query by
// query (one warp per tile, four queries per lane).  Bounds are formed in FP32 with
// every operation rounded down, from the outward-rounded boxes and the queries rounded
// toward the box, against thresholds rounded up; so a skipped tile lies farther than
// tau_q from every query q of g in exact arithmetic, and so (by more than the FP64
// rounding of a squared distance) in the FP64 distances that define the lists.
// Writes block g's selection as bits (word c of bits[g * mstride ..] for tiles 32 c ..)
// and their count.
constexpr int SEL_WARPS = KT_QB / 32;
__global__ void __launch_bounds__(KT_QB) knn_select_kernel(const double* Xp, const KnnTile* tiles, const int* soff,
                                                           const int* seeds, const int* first_tile, const float* box,
                                                           const float* boxT, int NT, const float* sbox,
                                                           const int* first_grp, int d, const double* Tq,
                                                           const double* tau, size_t mstride, unsigned* bits,
                                                           int* cnt) {
  extern __shared__ float sel_q[];  // [d][KT_QB] queries rounded down, then rounded up
  float* qlo = sel_q;
  float* qhi = sel_q + (size_t)d * KT_QB;
  __shared__ float tq_s[KT_QB];
  __shared__ unsigned char cand[KT_QB], keep[KT_QB];
  __shared__ int wcount[SEL_WARPS];
  __shared__ int base_s;
  __shared__ int sd[SEED_TILES];
  const int g = blockIdx.x;
  const KnnTile tl = tiles[g];
  const int ft = first_tile[tl.prob];
  const int nt = (tl.rn + KT_RB - 1) / KT_RB;
  const int ns = soff[g + 1] - soff[g];
  const float T = __double2float_ru(Tq[g] * (1.0 + 1e-9));
  const float* bq = box + (size_t)g * 2 * d;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) base_s = 0;
  if (tid < ns) sd[tid] = seeds[soff[g] + tid];
  for (int e = tid; e < d * KT_QB; e += KT_QB) {
    const int k = e / KT_QB, q = e % KT_QB;
    const double x = q < tl.qn ? Xp[(size_t)(tl.q0 + q) * d + k] : 0.0;
    qlo[e] = __double2float_rd(x);
    qhi[e] = __double2float_ru(x);
  }
  // absent rows get a negative threshold, which no bound meets
  tq_s[tid] = tid < tl.qn ? __double2float_ru(tau[tl.q0 + tid] * (1.0 + 1e-9)) : -1.0f;
  __syncthreads();
  // the four sub-blocks of 32 queries (lane + 32 j: queries consecutive in tree order):
  // their boxes and largest thresholds
  __shared__ float sub_lo[4][64], sub_hi[4][64], Tj_s[4];
  {
    const int j = tid >> 5;
    for (int k = lane; k < d; k += 32) {
      float lo = FLT_MAX, hi = -FLT_MAX;
      for (int q = 32 * j; q < min(32 * j + 32, tl.qn); ++q) {
        lo = fminf(lo, qlo[(size_t)k * KT_QB + q]);
        hi = fmaxf(hi, qhi[(size_t)k * KT_QB + q]);
      }
      sub_lo[j][k] = lo;
      sub_hi[j][k] = hi;
    }
    float tm = tq_s[tid];
#pragma unroll
    for (int o = 16; o; o >>= 1) tm = fmaxf(tm, __shfl_xor_sync(0xffffffffu, tm, o));
    if (lane == 0) Tj_s[j] = tm;
  }
  __syncthreads();
  const int fg = first_grp[tl.prob];
  for (int c0 = 0; c0 < nt; c0 += KT_QB) {
    const int t = c0 + tid;
    bool c = false;
    // the warp's SEL_GROUP tiles first as one group: a group box beyond T (every
    // lane computes the same bound from broadcast loads) rejects them all, as each
    // tile's own bound, rounded the same way, is at least the group's
    const bool grp_live = c0 + 32 * w < nt &&
                          !(box_lower_bound(bq, sbox + (size_t)(fg + ((c0 + 32 * w) / SEL_GROUP)) * 2 * d, d) > T);
    if (t < nt && grp_live) {
      bool seeded = false;
      for (int r = 0; r < ns; ++r) seeded = seeded || sd[r] == t;
      c = !seeded && !(box_lower_bound_T(bq, boxT, NT, ft + t, d) > T);
    }
    cand[tid] = c ? 1 : 0;
    __syncthreads();
    for (int i = w; i < KT_QB; i += SEL_WARPS) {
      if (!cand[i]) {  // warp-uniform
        if (lane == 0) keep[i] = 0;
        continue;
      }
      const float* bt = box + (size_t)(ft + c0 + i) * 2 * d;
      // a sub-block whose box lies beyond its largest threshold has no query that can
      // reach the tile (its lower bound, rounded down in any order, bounds every one of
      // its queries' true distances from below): the lanes share its dimensions
      float ps[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      for (int k = lane; k < d; k += 32) {
        const float lo = bt[k], hi = bt[d + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float gap = fmaxf(0.0f, fmaxf(__fsub_rd(lo, sub_hi[j][k]), __fsub_rd(sub_lo[j][k], hi)));
          ps[j] = __fadd_rd(ps[j], __fmul_rd(gap, gap));
        }
      }
      bool live[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
#pragma unroll
        for (int o = 16; o; o >>= 1) ps[j] = __fadd_rd(ps[j], __shfl_xor_sync(0xffffffffu, ps[j], o));
        live[j] = ps[j] <= Tj_s[j];  // the same in every lane (symmetric butterfly)
      }
      float lb[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (live[0] || live[1] || live[2] || live[3])
        for (int k = 0; k < d; ++k) {
          const float lo = bt[k], hi = bt[d + k];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (!live[j]) continue;  // warp-uniform
            const int q = lane + 32 * j;
            const float gap =
                fmaxf(0.0f, fmaxf(__fsub_rd(lo, qhi[(size_t)k * KT_QB + q]), __fsub_rd(qlo[(size_t)k * KT_QB + q], hi)));
            lb[j] = __fadd_rd(lb[j], __fmul_rd(gap, gap));
          }
        }
      bool hit = false;
#pragma unroll
      for (int j = 0; j < 4; ++j) hit = hit || (live[j] && lb[j] <= tq_s[lane + 32 * j]);
      const bool any = __any_sync(0xffffffffu, hit);
      if (lane == 0) keep[i] = any ? 1 : 0;
    }
    __syncthreads();
    const bool take = t < nt && keep[tid];
    const unsigned m = __ballot_sync(0xffffffffu, take);
    if (lane == 0) {
      wcount[w] = __popc(m);
      if (c0 + 32 * w < nt) bits[(size_t)g * mstride + (c0 >> 5) + w] = m;  // tiles c0 + 32 w ..
    }
    __syncthreads();
    if (tid == 0) {
      int tot = 0;
      for (int ww = 0; ww < SEL_WARPS; ++ww) tot += wcount[ww];
      base_s += tot;
    }
    __syncthreads();
  }
  if (tid == 0) cnt[g] = base_s;
}

// Block g's tile list, in tile order at toff[g], from its selection bits.
__global__ void knn_list_kernel(const KnnTile* tiles, const unsigned* bits, size_t mstride, const int* toff,
                                int* tlist) {
  __shared__ int wbase[KT_QB / 32];
  __shared__ int base_s;
  const int g = blockIdx.x;
  const KnnTile tl = tiles[g];
  const int nt = (tl.rn + KT_RB - 1) / KT_RB;
  const int nw = (nt + 31) / 32;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) base_s = 0;
  __syncthreads();
  for (int w0 = 0; w0 < nw; w0 += KT_QB) {  // one word per thread
    const unsigned word = w0 + tid < nw ? bits[(size_t)g * mstride + w0 + tid] : 0u;
    int c = __popc(word), incl = c;
    for (int o = 1; o < 32; o <<= 1) {  // inclusive scan of the counts over the warp
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) wbase[w] = incl;
    __syncthreads();
    int off = base_s;
    for (int ww = 0; ww < w; ++ww) off += wbase[ww];
    off += incl - c;
    unsigned m = word;
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      tlist[toff[g] + off++] = (w0 + tid) * 32 + b;
    }
    __syncthreads();
    if (tid == 0) {
      int tot = 0;
      for (int ww = 0; ww < KT_QB / 32; ++ww) tot += wbase[ww];
      base_s += tot;
    }
    __syncthreads();
  }
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
  if (kappa > RR_MAXK) throw Error(IASKIT_ERR_UNSUPPORTED, "kappa > 48");
  if (d > 64) throw Error(IASKIT_ERR_UNSUPPORTED, "kNN supports d <= 64");
  const int np = (int)problems.size();
  const std::vector<KnnTile> tiles = knn_tiles(problems);
  const bool wide = kappa + 8 > 32;
  // candidates kept per sub-list: kappa <= 16 keeps 16 (the kappa nearest are among
  // the 16 smallest of their own sub-lists; a shorter list halves the insertion work)
  const int KP = kappa <= 16 ? 16 : wide ? 64 : 32;
  KnnBufs b{};
  b.status = s.status.ensure_n<int>(1);
  b.Xc = s.x32.ensure_n<float>((size_t)N * padded_dim(d));
  b.qn = s.qnorm.ensure_n<float>(N);
  b.part = s.part.ensure_n<double>((size_t)np * KC_CHUNKS * d);
  b.mean = s.mean.ensure_n<double>((size_t)np * d);
  b.rmax = s.rmax.ensure_n<unsigned>(np);
  b.probs = s.probs.ensure_n<int2>(np);
  b.tiles = s.tiles.ensure_n<KnnTile>(tiles.size());
  b.cd = s.cand_d.ensure_n<float>((size_t)N * KT_SUB * KP);
  b.ci = s.cand_i.ensure_n<int>((size_t)N * KT_SUB * KP);
  b.flagged = s.flagged.ensure_n<int2>(N);
  b.nfl = s.counter.ensure_n<int>(1);
  // algorithmic work of the prefilter: one multiply-add per pair and coordinate
  for (const auto& pr : problems) prof().flops[PK_KNN] += 2.0 * (double)pr.second * pr.second * d;
  return KP == 16 ? knn_run<16>(X, d, kappa, problems, tiles, b, knn, st)
         : wide     ? knn_run<64>(X, d, kappa, problems, tiles, b, knn, st)
                    : knn_run<32>(X, d, kappa, problems, tiles, b, knn, st);
}

// Exact kNN lists of points held in tree order (see the pruning note above the
// tile_box kernel).  Xp: N x d row-major FP64 rows in permuted order, perm[r] = the
// original index of row r; problems = (first row, row count) in that order; knn is
// written in original indices at original rows, bit for bit the lists of
// knn_bruteforce on the original order.
int knn_tree(const double* Xp, const int* perm, int N, int d, int kappa, int* knn,
             const std::vector<std::pair<int, int>>& problems, KnnScratch& s, cudaStream_t st,
             KnnPruneStats* pstats) {
  ProfScope _ps(PK_KNN, st);
  int min_n = N;
  for (const auto& pr : problems) min_n = std::min(min_n, pr.second);
  if (kappa < 1 || kappa > min_n - 1) throw Error(IASKIT_ERR_ARG, "kappa must be in [1, N-1]");
  if (kappa > RR_MAXK) throw Error(IASKIT_ERR_UNSUPPORTED, "kappa > 48");
  if (d > 64) throw Error(IASKIT_ERR_UNSUPPORTED, "kNN supports d <= 64");
  const int np = (int)problems.size();
  const std::vector<KnnTile> tiles = knn_tiles(problems);
  const int nt = (int)tiles.size();
  // seed list offsets and the first tile of every problem
  std::vector<int> first(np, 0), soff(nt + 1, 0);
  for (int g = 0; g < nt; ++g) {
    const KnnTile& t = tiles[g];
    if (g == 0 || tiles[g - 1].prob != t.prob) first[t.prob] = g;
    soff[g + 1] = soff[g] + std::min(SEED_TILES, (t.rn + KT_RB - 1) / KT_RB);
  }
  const bool wide = kappa + 8 > 32;
  const int KP = kappa <= 16 ? 16 : wide ? 64 : 32;
  KnnBufs b{};
  b.status = s.status.ensure_n<int>(1);
  b.Xc = s.x32.ensure_n<float>((size_t)N * padded_dim(d));
  b.qn = s.qnorm.ensure_n<float>(N);
  b.part = s.part.ensure_n<double>((size_t)np * KC_CHUNKS * d);
  b.mean = s.mean.ensure_n<double>((size_t)np * d);
  b.rmax = s.rmax.ensure_n<unsigned>(np);
  b.probs = s.probs.ensure_n<int2>(np);
  b.tiles = s.tiles.ensure_n<KnnTile>(tiles.size());
  b.cd = s.cand_d.ensure_n<float>((size_t)N * KT_SUB * KP);
  b.ci = s.cand_i.ensure_n<int>((size_t)N * KT_SUB * KP);
  b.flagged = s.flagged.ensure_n<int2>(N);
  b.nfl = s.counter.ensure_n<int>(1);
  int* soff_d = s.seed_tiles.ensure_n<int>(nt + 1);
  int* seeds_d = s.seeds.ensure_n<int>(soff[nt]);
  int* first_d = s.first.ensure_n<int>(np);
  float* box = s.box.ensure_n<float>((size_t)nt * 2 * d);
  double* tau = s.tau.ensure_n<double>(N);
  double* Tq = s.tq.ensure_n<double>(nt);
  int* cnt = s.cnt.ensure_n<int>(nt);
  int* toff = s.toff.ensure_n<int>(nt + 1);
  std::vector<int2> hp(np);
  for (int q = 0; q < np; ++q) hp[q] = make_int2(problems[q].first, problems[q].second);
  h2d(b.probs, hp.data(), np, st);
  h2d(b.tiles, tiles.data(), tiles.size(), st);
  h2d(soff_d, soff.data(), soff.size(), st);
  h2d(first_d, first.data(), first.size(), st);
  IA_CUDA(cudaMemsetAsync(b.rmax, 0, np * sizeof(unsigned), st));
  IA_CUDA(cudaMemsetAsync(b.nfl, 0, sizeof(int), st));
  IA_CUDA(cudaMemsetAsync(b.status, 0, sizeof(int), st));
  center_partial_kernel<<<dim3(KC_CHUNKS, np), 64, 0, st>>>(Xp, d, b.probs, b.part);
  IA_LAUNCH_CHECK();
  center_mean_kernel<<<np, 64, 0, st>>>(d, b.probs, b.part, b.mean);
  IA_LAUNCH_CHECK();
  center_points_kernel<<<nt, KT_QB, 0, st>>>(Xp, d, padded_dim(d), b.tiles, b.mean, b.Xc, b.qn, b.rmax);
  IA_LAUNCH_CHECK();
  float* boxT = s.boxT.ensure_n<float>((size_t)nt * 2 * d);
  tile_box_kernel<<<nt, 64, 0, st>>>(Xp, d, b.tiles, nt, box, boxT);
  IA_LAUNCH_CHECK();
  // groups of SEL_GROUP consecutive tiles of each problem and their boxes
  std::vector<int2> grp;
  std::vector<int> fgrp(np, 0);
  for (int q = 0; q < np; ++q) {
    fgrp[q] = (int)grp.size();
    const int ntq = (problems[q].second + KT_RB - 1) / KT_RB;
    for (int j = 0; j < ntq; j += SEL_GROUP) grp.push_back(make_int2(first[q] + j, std::min(SEL_GROUP, ntq - j)));
  }
  int2* grp_d = s.grps.ensure_n<int2>(grp.size());
  int* fgrp_d = s.fgrp.ensure_n<int>(np);
  float* sbox = s.sbox.ensure_n<float>(grp.size() * 2 * d);
  h2d(grp_d, grp.data(), grp.size(), st);
  h2d(fgrp_d, fgrp.data(), np, st);
  super_box_kernel<<<(unsigned)grp.size(), 64, 0, st>>>(box, d, grp_d, sbox);
  IA_LAUNCH_CHECK();
  const int Dp = padded_dim(d);
  uint32_t* rec = s.rec.ensure_n<uint32_t>((size_t)nt * 2 * KT_RB * Dp);
  float* tn = s.tnorm.ensure_n<float>((size_t)nt * KT_RB);
  records_dispatch(Dp, b.Xc, b.qn, b.tiles, nt, rec, tn, st);
  // 1. seed tiles: the nearest boxes
  knn_seed_pick_kernel<<<nt, KT_QB, 0, st>>>(b.tiles, first_d, box, boxT, nt, d, soff_d, seeds_d);
  IA_LAUNCH_CHECK();
  auto prefilter = [&](TileList list) {
    if (KP == 16) prefilter2_dispatch<16>(Dp, rec, tn, b.tiles, first_d, nt, b.cd, b.ci, b.status, st, list);
    else if (wide) prefilter2_dispatch<64>(Dp, rec, tn, b.tiles, first_d, nt, b.cd, b.ci, b.status, st, list);
    else prefilter2_dispatch<32>(Dp, rec, tn, b.tiles, first_d, nt, b.cd, b.ci, b.status, st, list);
  };
  prefilter(TileList{seeds_d, soff_d, 0});
  // 2. bounds and the tiles left to scan
  auto seed_bound = [&](auto kp_tag, auto kap_tag) {
    constexpr int kp = decltype(kp_tag)::value, kap = decltype(kap_tag)::value;
    knn_seed_bound_kernel<kp, kap><<<nt, KT_QB, 0, st>>>(b.qn, padded_dim(d), kappa, b.tiles, b.cd, b.ci, tau, Tq);
  };
  using I16 = std::integral_constant<int, 16>;
  using I32 = std::integral_constant<int, 32>;
  using I48 = std::integral_constant<int, RR_MAXK>;
  using I64 = std::integral_constant<int, 64>;
  if (KP == 16) seed_bound(I16{}, I16{});
  else if (!wide) seed_bound(I32{}, I32{});
  else seed_bound(I64{}, I48{});
  IA_LAUNCH_CHECK();
  const size_t sel_smem = (size_t)2 * d * KT_QB * sizeof(float);
  if (sel_smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(knn_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sel_smem));
  int max_nt = 0;
  for (const auto& pr : problems) max_nt = std::max(max_nt, (pr.second + KT_RB - 1) / KT_RB);
  const size_t mstride = (size_t)(max_nt + 31) / 32 + 4;  // words per block, padded to the last chunk
  unsigned* bits = s.bits.ensure_n<unsigned>((size_t)nt * mstride);
  knn_select_kernel<<<nt, KT_QB, sel_smem, st>>>(Xp, b.tiles, soff_d, seeds_d, first_d, box, boxT, nt, sbox,
                                                 fgrp_d, d, Tq, tau, mstride, bits, cnt);
  IA_LAUNCH_CHECK();
  std::vector<int> hc(nt), ho(nt + 1, 0);
  d2h(hc.data(), cnt, nt, st);
  IA_CUDA(cudaStreamSynchronize(st));
  int64_t total = 0;
  double seed_pairs = 0.0, main_pairs = 0.0;
  for (int g = 0; g < nt; ++g) {
    ho[g] = (int)total;
    total += hc[g];
    seed_pairs += (double)tiles[g].qn * KT_RB * (soff[g + 1] - soff[g]);
    main_pairs += (double)tiles[g].qn * KT_RB * hc[g];
  }
  if (total > INT_MAX) throw Error(IASKIT_ERR_UNSUPPORTED, "kNN tile list too long");
  ho[nt] = (int)total;
  prof().flops[PK_KNN] += 2.0 * (seed_pairs + main_pairs) * d;
  if (pstats) {
    pstats->tiles_scanned = total;
    pstats->pairs_scanned = seed_pairs + main_pairs;
    double all = 0.0;
    for (const auto& pr : problems) all += (double)pr.second * pr.second;
    pstats->pairs_all = all;
  }
  // 3. the selected tiles, continuing the seed lists
  if (total > 0) {
    h2d(toff, ho.data(), nt + 1, st);
    int* tlist = s.tlist.ensure_n<int>((size_t)total);
    knn_list_kernel<<<nt, KT_QB, 0, st>>>(b.tiles, bits, mstride, toff, tlist);
    IA_LAUNCH_CHECK();
    prefilter(TileList{tlist, toff, 1});
  }
  // 4. exact re-rank (original indices), certified against the scanned and skipped points
  if (kappa <= 16)
    knn_rerank_kernel<16, 16><<<nt, KT_QB, 0, st>>>(Xp, d, kappa, padded_dim(d), b.tiles, b.cd, b.ci, b.qn,
                                                    b.rmax, perm, tau, knn, b.flagged, b.nfl);
  else if (!wide)
    knn_rerank_kernel<32, 32><<<nt, KT_QB, 0, st>>>(Xp, d, kappa, padded_dim(d), b.tiles, b.cd, b.ci, b.qn,
                                                    b.rmax, perm, tau, knn, b.flagged, b.nfl);
  else
    knn_rerank_kernel<64, RR_MAXK><<<nt, KT_QB, 0, st>>>(Xp, d, kappa, padded_dim(d), b.tiles, b.cd, b.ci,
                                                         b.qn, b.rmax, perm, tau, knn, b.flagged, b.nfl);
  IA_LAUNCH_CHECK();
  int nf = 0, dev_status = 0;
  d2h(&nf, b.nfl, 1, st);
  d2h(&dev_status, b.status, 1, st);
  IA_CUDA(cudaStreamSynchronize(st));
  if (dev_status & DEV_TIMEOUT) throw Error(IASKIT_ERR_TIMEOUT, "kNN tensor-core wait expired");
  if (nf > 0) {
    knn_fallback_kernel<<<nf, FB_THREADS, 0, st>>>(Xp, d, kappa, b.tiles, b.flagged, perm, knn);
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
constexpr size_t NA_X32 = 0;                     // rows padded to a multiple of 8 floats
constexpr size_t NA_QN = NA_X32 + sizeof(float) * (NA_MAX_ND + 7 * NA_MAX_N);
constexpr size_t NA_PART = NA_QN + sizeof(float) * NA_MAX_N;
constexpr size_t NA_MEAN = NA_PART + sizeof(double) * KC_CHUNKS * 64;
constexpr size_t NA_CD = NA_MEAN + sizeof(double) * 64;
constexpr size_t NA_CI = NA_CD + sizeof(float) * NA_MAX_N * KT_SUB * NA_KP;
constexpr size_t NA_FLAGGED = NA_CI + sizeof(int) * NA_MAX_N * KT_SUB * NA_KP;
constexpr size_t NA_TILES = NA_FLAGGED + sizeof(int2) * NA_MAX_N;
constexpr size_t NA_COUNTER = NA_TILES + sizeof(KnnTile) * (NA_MAX_N / KT_QB);
constexpr size_t NA_RMAX = NA_COUNTER + 256;
constexpr size_t NA_PROBS = NA_RMAX + 256;
constexpr size_t NA_STATUS = NA_PROBS + 256;
constexpr size_t NA_BYTES = NA_STATUS + 256;   // about 37.3 MiB

__device__ __align__(256) unsigned char g_knn_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
// Cached device addresses, one per device ordinal.  Host threads making their first
// call at the same time look the address up under one mutex, so the table is never
// written concurrently; later calls read an atomic entry without the lock.
std::atomic<void*> g_knn_noalloc_base[NA_MAX_DEVICES] = {};
std::mutex g_knn_noalloc_mutex;

// Device address of the scratch array on the current device (looked up once).
unsigned char* noalloc_scratch() {
  int dev = 0;
  IA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEVICES) throw Error(IASKIT_ERR_UNSUPPORTED, "device ordinal >= 64");
  void* p = g_knn_noalloc_base[dev].load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> lock(g_knn_noalloc_mutex);
    p = g_knn_noalloc_base[dev].load(std::memory_order_relaxed);
    if (!p) {
      cudaError_t e = cudaGetSymbolAddress(&p, g_knn_noalloc_scratch);
      if (e != cudaSuccess || !p)
        throw Error(IASKIT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_knn_noalloc_base[dev].store(p, std::memory_order_release);
    }
  }
  return static_cast<unsigned char*>(p);
}

void knn_noalloc(const double* X, int N, int d, int kappa, int* knn, cudaStream_t st) {
  unsigned char* base = noalloc_scratch();
  KnnBufs b{};
  b.status = reinterpret_cast<int*>(base + NA_STATUS);
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
