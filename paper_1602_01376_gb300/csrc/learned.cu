// Learned row proposal for skeletonization (not in the paper; it replaces the
// sampling rule of Sec. II-B for the nodes where it proves better).
//
// Per non-root node alpha with n_samp < N - n rows to sample:
//   candidates  at most n_cand / 2 of alpha's kNN candidates (plain sampling order,
//               hits descending, position ascending) plus uniform draws without
//               replacement on the node's LEARN stream, n_cand = min(cand_factor
//               n_samp, N - n) rows in all;
//   features    8 per candidate from the node's column subset (at most 32 evenly spaced
//               ID columns): log(1 + hits) / log(1 + kappa), distance to the subset mean
//               / h, max and mean kernel value to the subset, level / L,
//               log2 n / log2 N, distance / subset radius (capped at 1e3), 0;
//   score       a 3-layer MLP 8 -> 128 -> 128 -> 1 with ReLU, BF16 operands on the
//               tensor cores (mma.sync m16n8k16) and FP32 accumulation;
//   selection   the n_samp best-scored candidates (ties to the lower position),
//               ascending, after an optional Gumbel perturbation of the scores (then a
//               sample without replacement with probabilities ~ exp(score / temp));
//   judge       32 held-out rows on the node's HOLD stream, stratified: half from the
//               node's sibling, half from outside its parent (all from the sibling
//               under the root), each weighted by its stratum's size over its draws;
//               the weighted ID error sum w ||K(h, cols) - K(h, S) P||^2 /
//               sum w ||K(h, cols)||^2 in FP64 of the learned and the plain ID decides,
//               learned kept when not worse.
// Training labels: ridge leverage of each candidate against G = B^T diag(w) B with
// B = K(4096 stratified GRAM-stream rows, cols) and mu = tol^2 trace G,
// log-standardized per node; MSE loss, Adam on FP32 master weights with BF16 copies
// for the kernels.
// Streams: state s0 = splitmix64(splitmix64(seed ^ salt) ^ uid), draw q is
// splitmix64(s0 + q gamma); candidates map j = draw mod (N - n) around the node, the
// stratified draws map into the sibling or around the parent.
#include <cuda_bf16.h>

#include <climits>

#include "kernels.cuh"

namespace iaskit {

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ int stream_pos(uint64_t s0, uint64_t q, int o, int n, int comp) {
  const uint64_t r = splitmix64(s0 + q * 0x9E3779B97F4A7C15ull);
  const int j = (int)(r % (uint64_t)comp);
  return j < o ? j : j + n;
}
__host__ __device__ __forceinline__ uint64_t stream_state(uint64_t seed, uint64_t salt, uint64_t uid) {
  return splitmix64(splitmix64(seed ^ salt) ^ uid);
}

// ------------------------------------------------------------- candidates
// One block per node.  Shared memory: the hash set (4 cap_pow2 ints).
constexpr int LC_THREADS = 256;
__global__ void candidates_kernel(const uint32_t* cand_sorted, const uint64_t* keys_sorted,
                                  const int* node_start, const int* node_cnt, int cnt_bits,
                                  const int* off, const SampleNodeInfo* info,
                                  const LearnNodeInfo* linfo, uint64_t seed, int cap_pow2,
                                  int* cand, float* hits, int* status) {
  extern __shared__ int hset[];
  const int node = blockIdx.x;
  const LearnNodeInfo li = linfo[node];
  if (li.n_cand <= 0) return;
  const SampleNodeInfo inf = info[node];
  const int pb = inf.pb;
  const int o = off[node] - pb, n = off[node + 1] - off[node];
  const int comp = inf.pn - n;
  const int k = min(node_cnt[node], li.n_cand / 2);
  int* out = cand + li.cand_off;
  float* oh = hits + li.cand_off;
  const uint64_t mask = (cnt_bits >= 64) ? ~0ull : ((1ull << cnt_bits) - 1);
  for (int t = threadIdx.x; t < k; t += LC_THREADS) {
    out[t] = (int)cand_sorted[node_start[node] + t];
    oh[t] = (float)(mask - (keys_sorted[node_start[node] + t] & mask));
  }
  const int hsize = 4 * cap_pow2;
  for (int t = threadIdx.x; t < hsize; t += LC_THREADS) hset[t] = -1;
  __syncthreads();
  if (threadIdx.x != 0) return;
  auto insert = [&](int pos) -> bool {
    uint32_t hh = ((uint32_t)pos * 2654435761u) & (uint32_t)(hsize - 1);
    while (true) {
      const int v = hset[hh];
      if (v == pos) return false;
      if (v < 0) {
        hset[hh] = pos;
        return true;
      }
      hh = (hh + 1) & (uint32_t)(hsize - 1);
    }
  };
  for (int t = 0; t < k; ++t) insert(out[t]);
  int have = k;
  const uint64_t s0 = stream_state(seed, LEARN_SALT, (uint64_t)inf.uid);
  const uint64_t limit = 64ull * (uint64_t)comp + 4096ull;
  uint64_t q = 0;
  while (have < li.n_cand) {
    if (q >= limit) {
      atomicOr(status, DEV_OVERFLOW);
      break;
    }
    const int pos = pb + stream_pos(s0, q, o, n, comp);
    if (insert(pos)) {
      out[have] = pos;
      oh[have] = 0.0f;
      ++have;
    }
    ++q;
  }
}

// --------------------------------------------------------------- features
constexpr int LF_THREADS = 256;
constexpr int LF_SUB = 32;
__global__ void features_kernel(const double* Xp, int d, const LearnFeatDesc* descs,
                                uint16_t* feat) {
  extern __shared__ float ys[];  // LF_SUB x d subset, then d for the mean
  __shared__ float s_r;
  const LearnFeatDesc D = descs[blockIdx.y];
  const int k = min(LF_SUB, D.ncols);
  float* mu = ys + LF_SUB * d;
  for (int e = threadIdx.x; e < k * d; e += LF_THREADS) {
    const int j = e / d, q = e % d;
    const int jj = (int)(((int64_t)j * D.ncols) / k);
    const int col = D.colsA ? (jj < D.nA ? D.colsA[jj] : D.colsB[jj - D.nA]) : D.col0 + jj;
    ys[j * d + q] = (float)Xp[(size_t)col * d + q];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < d; q += LF_THREADS) {
    float s = 0.0f;
    for (int j = 0; j < k; ++j) s += ys[j * d + q];
    mu[q] = s / (float)k;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    float r = 0.0f;
    for (int j = threadIdx.x; j < k; j += 32) {
      float s = 0.0f;
      for (int q = 0; q < d; ++q) {
        const float t = ys[j * d + q] - mu[q];
        s = fmaf(t, t, s);
      }
      r = fmaxf(r, sqrtf(s));
    }
    for (int w = 16; w > 0; w >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, w));
    if (threadIdx.x == 0) s_r = fmaxf(r, 1e-30f);
  }
  __syncthreads();
  const float rr = s_r;
  const float sc = (float)D.scale;
  for (int c = blockIdx.x * LF_THREADS + threadIdx.x; c < D.n_cand; c += gridDim.x * LF_THREADS) {
    const int pos = D.cand[c];
    const double* x = Xp + (size_t)pos * d;
    float dm = 0.0f;
    for (int q = 0; q < d; ++q) {
      const float t = (float)x[q] - mu[q];
      dm = fmaf(t, t, dm);
    }
    dm = sqrtf(dm);
    float kmax = 0.0f, ksum = 0.0f;
    for (int j = 0; j < k; ++j) {
      float s = 0.0f;
      for (int q = 0; q < d; ++q) {
        const float t = (float)x[q] - ys[j * d + q];
        s = fmaf(t, t, s);
      }
      const float kv = __expf(s * sc);
      kmax = fmaxf(kmax, kv);
      ksum += kv;
    }
    float f[8];
    f[0] = log1pf(D.hits[c]) * D.inv_log1p_kappa;
    f[1] = dm * D.inv_h;
    f[2] = kmax;
    f[3] = ksum / (float)k;
    f[4] = D.f4;
    f[5] = D.f5;
    f[6] = fminf(dm / rr, 1e3f);
    f[7] = 0.0f;
    uint16_t* o = feat + ((size_t)D.cand_off + c) * 8;
#pragma unroll
    for (int q = 0; q < 8; ++q) o[q] = __bfloat16_as_ushort(__float2bfloat16(f[q]));
  }
}

// ---------------------------------------------------------------------- MLP
// Tensor-core fragment helpers for mma.sync.m16n8k16 (BF16 in, FP32 accumulate).
// Lane l: g = l / 4, t = l % 4.  A (16 x 16, row-major): reg0 = (g, 2t..2t+1),
// reg1 = (g+8, 2t..), reg2 = (g, 2t+8..), reg3 = (g+8, 2t+8..).  B (16 x 8, k x n):
// reg0 = (k = 2t..2t+1, n = g), reg1 = (k = 2t+8.., n = g).  C: c0,c1 = (g, 2t..2t+1),
// c2,c3 = (g+8, 2t..2t+1).  The lower k (or n) index sits in the low half.
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) {
  return (uint32_t)lo | ((uint32_t)hi << 16);
}
__device__ __forceinline__ uint32_t ld32(const uint16_t* p) {  // p 4-byte aligned
  return *reinterpret_cast<const uint32_t*>(p);
}
__device__ __forceinline__ uint16_t f2b(float x) { return __bfloat16_as_ushort(__float2bfloat16(x)); }
__device__ __forceinline__ float b2f(uint16_t x) { return __bfloat162float(__ushort_as_bfloat16(x)); }

constexpr int MT = 64;            // rows per tile (16 per warp)
constexpr int MWARPS = 4;
constexpr int MTHREADS = 32 * MWARPS;
constexpr int WS = MLP_W + 8;     // padded smem row stride (bf16): conflict-free fragment loads

// Shared memory of the forward kernel (bf16 units): W2 [128][WS], W1 [128][8], H1 per
// warp [16][WS]; floats b1, b2, w3.
__global__ void __launch_bounds__(MTHREADS) mlp_forward_kernel(const uint16_t* X, int64_t n,
                                                               MlpDev w, float* y, uint16_t* H1g,
                                                               uint16_t* H2g) {
  extern __shared__ __align__(16) unsigned char smraw[];
  uint16_t* W2s = reinterpret_cast<uint16_t*>(smraw);
  uint16_t* W1s = W2s + MLP_W * WS;
  uint16_t* Hs = W1s + MLP_W * MLP_F;
  float* fb1 = reinterpret_cast<float*>(Hs + MWARPS * 16 * WS);
  float* fb2 = fb1 + MLP_W;
  float* fw3 = fb2 + MLP_W;
  for (int e = threadIdx.x; e < MLP_W * MLP_W; e += MTHREADS)
    W2s[(e / MLP_W) * WS + (e % MLP_W)] = w.W2[e];
  for (int e = threadIdx.x; e < MLP_W * MLP_F; e += MTHREADS) W1s[e] = w.W1[e];
  for (int e = threadIdx.x; e < MLP_W; e += MTHREADS) {
    fb1[e] = w.master[MLP_OFF_B1 + e];
    fb2[e] = w.master[MLP_OFF_B2 + e];
    fw3[e] = b2f(w.w3[e]);
  }
  __syncthreads();
  const float b3 = w.master[MLP_OFF_B3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint16_t* H = Hs + warp * 16 * WS;
  const int64_t ntiles = (n + MT - 1) / MT;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * MT + warp * 16;
    const int64_t ra = r0 + g, rb = r0 + g + 8;
    // layer 1: K = 8 real features (the upper half of k16 is zero)
    uint32_t a[4];
    a[0] = ra < n ? ld32(X + ra * MLP_F + 2 * t) : 0u;
    a[1] = rb < n ? ld32(X + rb * MLP_F + 2 * t) : 0u;
    a[2] = 0u;
    a[3] = 0u;
    __syncwarp();
#pragma unroll 4
    for (int j = 0; j < MLP_W / 8; ++j) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      uint32_t b[2] = {ld32(W1s + (8 * j + g) * MLP_F + 2 * t), 0u};
      mma_bf16(c, a, b);
      const int col = 8 * j + 2 * t;
      const float h0 = fmaxf(c[0] + fb1[col], 0.f), h1 = fmaxf(c[1] + fb1[col + 1], 0.f);
      const float h2 = fmaxf(c[2] + fb1[col], 0.f), h3 = fmaxf(c[3] + fb1[col + 1], 0.f);
      const uint32_t p0 = pack2(f2b(h0), f2b(h1)), p1 = pack2(f2b(h2), f2b(h3));
      *reinterpret_cast<uint32_t*>(H + g * WS + col) = p0;
      *reinterpret_cast<uint32_t*>(H + (g + 8) * WS + col) = p1;
      if (H1g) {
        if (ra < n) *reinterpret_cast<uint32_t*>(H1g + ra * MLP_W + col) = p0;
        if (rb < n) *reinterpret_cast<uint32_t*>(H1g + rb * MLP_W + col) = p1;
      }
    }
    __syncwarp();
    // layer 2: K = 128
    float acc[MLP_W / 8][4];
#pragma unroll
    for (int j = 0; j < MLP_W / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
    for (int k0 = 0; k0 < MLP_W; k0 += 16) {
      uint32_t fa[4];
      fa[0] = ld32(H + g * WS + k0 + 2 * t);
      fa[1] = ld32(H + (g + 8) * WS + k0 + 2 * t);
      fa[2] = ld32(H + g * WS + k0 + 2 * t + 8);
      fa[3] = ld32(H + (g + 8) * WS + k0 + 2 * t + 8);
#pragma unroll
      for (int j = 0; j < MLP_W / 8; ++j) {
        uint32_t fb[2];
        fb[0] = ld32(W2s + (8 * j + g) * WS + k0 + 2 * t);
        fb[1] = ld32(W2s + (8 * j + g) * WS + k0 + 2 * t + 8);
        mma_bf16(acc[j], fa, fb);
      }
    }
    // bias, ReLU, BF16 activations, output layer in FP32
    float ya = 0.f, yb = 0.f;
#pragma unroll
    for (int j = 0; j < MLP_W / 8; ++j) {
      const int col = 8 * j + 2 * t;
      const uint16_t q0 = f2b(fmaxf(acc[j][0] + fb2[col], 0.f));
      const uint16_t q1 = f2b(fmaxf(acc[j][1] + fb2[col + 1], 0.f));
      const uint16_t q2 = f2b(fmaxf(acc[j][2] + fb2[col], 0.f));
      const uint16_t q3 = f2b(fmaxf(acc[j][3] + fb2[col + 1], 0.f));
      ya = fmaf(b2f(q0), fw3[col], fmaf(b2f(q1), fw3[col + 1], ya));
      yb = fmaf(b2f(q2), fw3[col], fmaf(b2f(q3), fw3[col + 1], yb));
      if (H2g) {
        if (ra < n) *reinterpret_cast<uint32_t*>(H2g + ra * MLP_W + col) = pack2(q0, q1);
        if (rb < n) *reinterpret_cast<uint32_t*>(H2g + rb * MLP_W + col) = pack2(q2, q3);
      }
    }
    ya += __shfl_xor_sync(0xffffffffu, ya, 1);
    ya += __shfl_xor_sync(0xffffffffu, ya, 2);
    yb += __shfl_xor_sync(0xffffffffu, yb, 1);
    yb += __shfl_xor_sync(0xffffffffu, yb, 2);
    if (t == 0) {
      if (ra < n) y[ra] = ya + b3;
      if (rb < n) y[rb] = yb + b3;
    }
    __syncwarp();
  }
}

// Backward pass of the mean squared error over one 64-row tile per block; gradients
// are accumulated into grad (FP32, zeroed by the Adam step) with atomics.
// Shared memory (bf16): W2T [128][WS], H1 [64][WS], dA2 [64][WS], dA1 [64][WS],
// X [64][8]; floats: w3 [128], per-block partial sums.
__global__ void __launch_bounds__(MTHREADS) mlp_backward_kernel(const uint16_t* X, const uint16_t* H1g,
                                                                const uint16_t* H2g, const float* y,
                                                                const float* tgt, int64_t n,
                                                                float inv_batch, MlpDev w,
                                                                float* grad, float* loss) {
  extern __shared__ __align__(16) unsigned char smraw[];
  uint16_t* W2T = reinterpret_cast<uint16_t*>(smraw);
  uint16_t* H1s = W2T + MLP_W * WS;
  uint16_t* dA2 = H1s + MT * WS;
  uint16_t* dA1 = dA2 + MT * WS;
  uint16_t* Xs = dA1 + MT * WS;
  float* fw3 = reinterpret_cast<float*>(Xs + MT * MLP_F);
  float* gw3 = fw3 + MLP_W;   // partial sums of this block
  float* gb2 = gw3 + MLP_W;
  float* gb1 = gb2 + MLP_W;
  float* misc = gb1 + MLP_W;  // [0] sum dy, [1] loss
  for (int e = threadIdx.x; e < MLP_W * MLP_W; e += MTHREADS)
    W2T[(e / MLP_W) * WS + (e % MLP_W)] = w.W2T[e];
  for (int e = threadIdx.x; e < MLP_W; e += MTHREADS) {
    fw3[e] = b2f(w.w3[e]);
    gw3[e] = gb2[e] = gb1[e] = 0.f;
  }
  if (threadIdx.x < 2) misc[threadIdx.x] = 0.f;
  const int64_t r0 = (int64_t)blockIdx.x * MT;
  for (int e = threadIdx.x; e < MT * MLP_W; e += MTHREADS) {
    const int r = e / MLP_W, c = e % MLP_W;
    H1s[r * WS + c] = (r0 + r < n) ? H1g[(r0 + r) * MLP_W + c] : (uint16_t)0;
  }
  for (int e = threadIdx.x; e < MT * MLP_F; e += MTHREADS) {
    const int r = e / MLP_F;
    Xs[e] = (r0 + r < n) ? X[r0 * MLP_F + e] : (uint16_t)0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // dy and dA2 = dy w3 (H2 > 0): warp w owns rows 16w .. 16w+15, lanes stride columns
  for (int rr = 0; rr < 16; ++rr) {
    const int r = warp * 16 + rr;
    const int64_t gr = r0 + r;
    float dy = 0.f;
    if (gr < n) {
      const float e = y[gr] - tgt[gr];
      dy = 2.f * e * inv_batch;
      if (lane == 0) {
        atomicAdd(&misc[0], dy);
        atomicAdd(&misc[1], e * e * inv_batch);
      }
    }
    for (int c = lane; c < MLP_W; c += 32) {
      const float h2 = gr < n ? b2f(H2g[gr * MLP_W + c]) : 0.f;
      const float v = h2 > 0.f ? dy * fw3[c] : 0.f;
      dA2[r * WS + c] = f2b(v);
      atomicAdd(&gw3[c], dy * h2);
      atomicAdd(&gb2[c], v);
    }
  }
  __syncthreads();
  // dH1 = dA2 W2 (K = 128), then dA1 = dH1 (H1 > 0)
  {
    const uint16_t* A = dA2 + warp * 16 * WS;
    float acc[MLP_W / 8][4];
#pragma unroll
    for (int j = 0; j < MLP_W / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
    for (int k0 = 0; k0 < MLP_W; k0 += 16) {
      uint32_t fa[4];
      fa[0] = ld32(A + g * WS + k0 + 2 * t);
      fa[1] = ld32(A + (g + 8) * WS + k0 + 2 * t);
      fa[2] = ld32(A + g * WS + k0 + 2 * t + 8);
      fa[3] = ld32(A + (g + 8) * WS + k0 + 2 * t + 8);
#pragma unroll
      for (int j = 0; j < MLP_W / 8; ++j) {
        uint32_t fb[2];
        fb[0] = ld32(W2T + (8 * j + g) * WS + k0 + 2 * t);
        fb[1] = ld32(W2T + (8 * j + g) * WS + k0 + 2 * t + 8);
        mma_bf16(acc[j], fa, fb);
      }
    }
    const int ra = warp * 16 + g, rb = ra + 8;
#pragma unroll
    for (int j = 0; j < MLP_W / 8; ++j) {
      const int col = 8 * j + 2 * t;
      const float m0 = b2f(H1s[ra * WS + col]) > 0.f ? acc[j][0] : 0.f;
      const float m1 = b2f(H1s[ra * WS + col + 1]) > 0.f ? acc[j][1] : 0.f;
      const float m2 = b2f(H1s[rb * WS + col]) > 0.f ? acc[j][2] : 0.f;
      const float m3 = b2f(H1s[rb * WS + col + 1]) > 0.f ? acc[j][3] : 0.f;
      *reinterpret_cast<uint32_t*>(dA1 + ra * WS + col) = pack2(f2b(m0), f2b(m1));
      *reinterpret_cast<uint32_t*>(dA1 + rb * WS + col) = pack2(f2b(m2), f2b(m3));
      atomicAdd(&gb1[col], m0 + m2);
      atomicAdd(&gb1[col + 1], m1 + m3);
    }
  }
  __syncthreads();
  // gW2[j][i] = sum_r dA2[r][j] H1[r][i]: M = 128 (j), N = 128 (i), K = 64 rows.
  // Warp w owns j in [32w, 32w + 32) as two 16-row m-tiles.
  for (int mt = 0; mt < 2; ++mt) {
    const int j0 = warp * 32 + mt * 16;
    float acc[MLP_W / 8][4];
#pragma unroll
    for (int jn = 0; jn < MLP_W / 8; ++jn) acc[jn][0] = acc[jn][1] = acc[jn][2] = acc[jn][3] = 0.f;
#pragma unroll
    for (int k0 = 0; k0 < MT; k0 += 16) {
      uint32_t fa[4];  // A(m = j, k = r) = dA2[r][j]
      fa[0] = pack2(dA2[(k0 + 2 * t) * WS + j0 + g], dA2[(k0 + 2 * t + 1) * WS + j0 + g]);
      fa[1] = pack2(dA2[(k0 + 2 * t) * WS + j0 + g + 8], dA2[(k0 + 2 * t + 1) * WS + j0 + g + 8]);
      fa[2] = pack2(dA2[(k0 + 2 * t + 8) * WS + j0 + g], dA2[(k0 + 2 * t + 9) * WS + j0 + g]);
      fa[3] = pack2(dA2[(k0 + 2 * t + 8) * WS + j0 + g + 8], dA2[(k0 + 2 * t + 9) * WS + j0 + g + 8]);
#pragma unroll
      for (int jn = 0; jn < MLP_W / 8; ++jn) {
        const int i = 8 * jn + g;  // B(k = r, n = i) = H1[r][i]
        uint32_t fb[2];
        fb[0] = pack2(H1s[(k0 + 2 * t) * WS + i], H1s[(k0 + 2 * t + 1) * WS + i]);
        fb[1] = pack2(H1s[(k0 + 2 * t + 8) * WS + i], H1s[(k0 + 2 * t + 9) * WS + i]);
        mma_bf16(acc[jn], fa, fb);
      }
    }
#pragma unroll
    for (int jn = 0; jn < MLP_W / 8; ++jn) {
      const int i = 8 * jn + 2 * t;
      float* G = grad + MLP_OFF_W2;
      atomicAdd(&G[(j0 + g) * MLP_W + i], acc[jn][0]);
      atomicAdd(&G[(j0 + g) * MLP_W + i + 1], acc[jn][1]);
      atomicAdd(&G[(j0 + g + 8) * MLP_W + i], acc[jn][2]);
      atomicAdd(&G[(j0 + g + 8) * MLP_W + i + 1], acc[jn][3]);
    }
  }
  // gW1[j][f] = sum_r dA1[r][j] X[r][f]: M = 128, N = 8, K = 64
  for (int mt = 0; mt < 2; ++mt) {
    const int j0 = warp * 32 + mt * 16;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k0 = 0; k0 < MT; k0 += 16) {
      uint32_t fa[4];
      fa[0] = pack2(dA1[(k0 + 2 * t) * WS + j0 + g], dA1[(k0 + 2 * t + 1) * WS + j0 + g]);
      fa[1] = pack2(dA1[(k0 + 2 * t) * WS + j0 + g + 8], dA1[(k0 + 2 * t + 1) * WS + j0 + g + 8]);
      fa[2] = pack2(dA1[(k0 + 2 * t + 8) * WS + j0 + g], dA1[(k0 + 2 * t + 9) * WS + j0 + g]);
      fa[3] = pack2(dA1[(k0 + 2 * t + 8) * WS + j0 + g + 8], dA1[(k0 + 2 * t + 9) * WS + j0 + g + 8]);
      uint32_t fb[2];
      fb[0] = pack2(Xs[(k0 + 2 * t) * MLP_F + g], Xs[(k0 + 2 * t + 1) * MLP_F + g]);
      fb[1] = pack2(Xs[(k0 + 2 * t + 8) * MLP_F + g], Xs[(k0 + 2 * t + 9) * MLP_F + g]);
      mma_bf16(acc, fa, fb);
    }
    float* G = grad + MLP_OFF_W1;
    const int f = 2 * t;
    atomicAdd(&G[(j0 + g) * MLP_F + f], acc[0]);
    atomicAdd(&G[(j0 + g) * MLP_F + f + 1], acc[1]);
    atomicAdd(&G[(j0 + g + 8) * MLP_F + f], acc[2]);
    atomicAdd(&G[(j0 + g + 8) * MLP_F + f + 1], acc[3]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < MLP_W; e += MTHREADS) {
    atomicAdd(&grad[MLP_OFF_W3 + e], gw3[e]);
    atomicAdd(&grad[MLP_OFF_B2 + e], gb2[e]);
    atomicAdd(&grad[MLP_OFF_B1 + e], gb1[e]);
  }
  if (threadIdx.x == 0) {
    atomicAdd(&grad[MLP_OFF_B3], misc[0]);
    atomicAdd(loss, misc[1]);
  }
}

// Adam with bias correction on the FP32 master weights; refreshes the BF16 copies
// (W1, W2, W2^T, w3) and clears the gradient.
__global__ void mlp_adam_kernel(MlpDev w, float* grad, float* m, float* v, float lr, float beta1,
                                float beta2, float eps, float c1, float c2) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < MLP_NPARAM; e += gridDim.x * blockDim.x) {
    const float gr = grad[e];
    const float mm = beta1 * m[e] + (1.f - beta1) * gr;
    const float vv = beta2 * v[e] + (1.f - beta2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    grad[e] = 0.f;
    const float p = w.master[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    w.master[e] = p;
    const uint16_t pb = f2b(p);
    if (e < MLP_OFF_B1) {
      w.W1[e] = pb;
    } else if (e >= MLP_OFF_W2 && e < MLP_OFF_B2) {
      const int k = e - MLP_OFF_W2, j = k / MLP_W, i = k % MLP_W;
      w.W2[k] = pb;
      w.W2T[i * MLP_W + j] = pb;
    } else if (e >= MLP_OFF_W3 && e < MLP_OFF_B3) {
      w.w3[e - MLP_OFF_W3] = pb;
    }
  }
}

__global__ void mlp_copies_kernel(MlpDev w) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < MLP_NPARAM; e += gridDim.x * blockDim.x) {
    const uint16_t pb = f2b(w.master[e]);
    if (e < MLP_OFF_B1) {
      w.W1[e] = pb;
    } else if (e >= MLP_OFF_W2 && e < MLP_OFF_B2) {
      const int k = e - MLP_OFF_W2, j = k / MLP_W, i = k % MLP_W;
      w.W2[k] = pb;
      w.W2T[i * MLP_W + j] = pb;
    } else if (e >= MLP_OFF_W3 && e < MLP_OFF_B3) {
      w.w3[e - MLP_OFF_W3] = pb;
    }
  }
}

// ------------------------------------------------------------- selection
// One block per node: keys (score descending, position ascending) sorted bitonically,
// the first n_samp positions sorted ascending again.
constexpr int LS_THREADS = 256;
__device__ __forceinline__ uint32_t score_key(float s) {  // larger score -> smaller key
  uint32_t b = __float_as_uint(s == 0.f ? 0.f : s);
  b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // ascending order of s
  return ~b;
}
__global__ void select_kernel(const float* score, const int* cand, const LearnNodeInfo* linfo,
                              const SampleNodeInfo* info, int cap_pow2, int* samp) {
  extern __shared__ unsigned long long keys[];
  const LearnNodeInfo li = linfo[blockIdx.x];
  if (li.n_cand <= 0) return;
  for (int t = threadIdx.x; t < cap_pow2; t += LS_THREADS) {
    if (t < li.n_cand) {
      float s = score[li.cand_off + t];
      if (!(s == s)) s = -INFINITY;  // NaN scores rank last
      keys[t] = ((unsigned long long)score_key(s) << 32) | (uint32_t)cand[li.cand_off + t];
    } else {
      keys[t] = ~0ull;
    }
  }
  __syncthreads();
  auto bitonic = [&](int len) {
    for (int k = 2; k <= len; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < len; t += LS_THREADS) {
          const int p = t ^ j;
          if (p > t) {
            const bool up = (t & k) == 0;
            const unsigned long long a = keys[t], b = keys[p];
            if ((a > b) == up) {
              keys[t] = b;
              keys[p] = a;
            }
          }
        }
        __syncthreads();
      }
  };
  bitonic(cap_pow2);
  int sp = 1;
  while (sp < li.n_samp) sp <<= 1;
  for (int t = threadIdx.x; t < sp; t += LS_THREADS)
    keys[t] = t < li.n_samp ? (unsigned long long)(uint32_t)keys[t] : ~0ull;
  __syncthreads();
  bitonic(sp);
  int* out = samp + info[blockIdx.x].samp_off;
  for (int t = threadIdx.x; t < li.n_samp; t += LS_THREADS) out[t] = (int)(uint32_t)keys[t];
}

__global__ void perturb_kernel(float* score, const LearnNodeInfo* linfo, const SampleNodeInfo* info,
                               uint64_t seed, double temp) {
  const LearnNodeInfo li = linfo[blockIdx.y];
  if (li.n_cand <= 0) return;
  const uint64_t s0 = stream_state(seed, GUMBEL_SALT, (uint64_t)info[blockIdx.y].uid);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < li.n_cand; c += gridDim.x * blockDim.x) {
    const uint64_t r = splitmix64(s0 + (uint64_t)c * 0x9E3779B97F4A7C15ull);
    const double u = ((double)(r >> 11) + 0.5) * 0x1.0p-53;
    const double g = -log(-log(u));
    score[li.cand_off + c] = (float)((double)score[li.cand_off + c] + temp * g);
  }
}

// -------------------------------------------------------------- streams
__global__ void stream_rows_kernel(const StreamDesc* descs, int count, uint64_t seed, uint64_t salt,
                                   int* out) {
  const StreamDesc D = descs[blockIdx.y];
  const uint64_t s0 = stream_state(seed, salt, (uint64_t)D.uid);
  const int far = D.pn - D.par_n;
  const int cs = far == 0 ? count : count / 2;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
    const uint64_t r = splitmix64(s0 + (uint64_t)q * 0x9E3779B97F4A7C15ull);
    int pos;
    if (q < cs) {
      pos = D.sib_o + (int)(r % (uint64_t)D.sib_n);
    } else {
      const int j = (int)(r % (uint64_t)far);
      pos = j < D.par_o ? j : j + D.par_n;
    }
    out[(size_t)D.out_off + q] = D.pb + pos;
  }
}

// -------------------------------------------------------------- judge
// One block per descriptor: err = sum over held-out rows h and columns j of
// (K(h, col_j) - sum_k K(h, skel_k) P[k, j])^2, den = sum K(h, col_j)^2, in FP64.
constexpr int JG_THREADS = 256;
constexpr int JG_ROWS = 8;
__global__ void judge_kernel(const double* Xp, int d, const JudgeDesc* descs, int nh, double* out) {
  extern __shared__ double ks[];  // JG_ROWS x s
  __shared__ double red[2][JG_THREADS / 32];
  const JudgeDesc D = descs[blockIdx.x];
  double num = 0.0, den = 0.0;
  for (int h0 = 0; h0 < nh; h0 += JG_ROWS) {
    const int nr = min(JG_ROWS, nh - h0);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * D.s; e += JG_THREADS) {
      const int r = e / D.s, k = e % D.s;
      const double* x = Xp + (size_t)D.H[h0 + r] * d;
      const double* z = Xp + (size_t)D.skel[k] * d;
      double s = 0.0;
      for (int q = 0; q < d; ++q) {
        const double t = x[q] - z[q];
        s = fma(t, t, s);
      }
      ks[r * D.s + k] = exp(s * D.scale);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * D.ncols; e += JG_THREADS) {
      const int r = e / D.ncols, j = e % D.ncols;
      const int col = D.colsA ? (j < D.nA ? D.colsA[j] : D.colsB[j - D.nA]) : D.col0 + j;
      const double* x = Xp + (size_t)D.H[h0 + r] * d;
      const double* z = Xp + (size_t)col * d;
      double s = 0.0;
      for (int q = 0; q < d; ++q) {
        const double t = x[q] - z[q];
        s = fma(t, t, s);
      }
      const double a = exp(s * D.scale);
      double p = 0.0;
      const double* Pj = D.P + (size_t)j * D.s;
      for (int k = 0; k < D.s; ++k) p = fma(ks[r * D.s + k], Pj[k], p);
      const double ee = a - p;
      const double wt = h0 + r < D.nh_s ? D.w_s : D.w_r;
      num = fma(wt * ee, ee, num);
      den = fma(wt * a, a, den);
    }
  }
  num = warp_sum(num);
  den = warp_sum(den);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = num;
    red[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < JG_THREADS / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    out[2 * blockIdx.x] = a;
    out[2 * blockIdx.x + 1] = b;
  }
}

// -------------------------------------------------------------- labels
__global__ void gather_cols_kernel(const ColsDesc* descs, int* out) {
  const ColsDesc D = descs[blockIdx.x];
  for (int j = threadIdx.x; j < D.ncols; j += blockDim.x)
    out[D.out_off + j] = D.colsA ? (j < D.nA ? D.colsA[j] : D.colsB[j - D.nA]) : D.col0 + j;
}
// G += mu I with mu = tol2 * trace(G), one block per matrix
__global__ void add_ridge_kernel(const RidgeDesc* descs, double tol2) {
  __shared__ double red[32];
  const RidgeDesc D = descs[blockIdx.x];
  double s = 0.0;
  for (int i = threadIdx.x; i < D.n; i += blockDim.x) s += D.G[(size_t)i * D.n + i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  const double mu = tol2 * red[0];
  __syncthreads();
  for (int i = threadIdx.x; i < D.n; i += blockDim.x) D.G[(size_t)i * D.n + i] += mu;
}
// lev_c = sum_i Bc[i, c] Xs[i, c]; target = standardized log lev over the node
__global__ void leverage_kernel(const LevDesc* descs, double* lev_all, float* target) {
  __shared__ double red[2][32];
  const LevDesc D = descs[blockIdx.x];
  double s1 = 0.0, s2 = 0.0;
  for (int c = threadIdx.x; c < D.n_cand; c += blockDim.x) {
    const double* b = D.Bc + (size_t)c * D.nc;
    const double* x = D.Xs + (size_t)c * D.nc;
    double l = 0.0;
    for (int i = 0; i < D.nc; ++i) l = fma(b[i], x[i], l);
    lev_all[D.out_off + c] = l;
    const double z = log(fmax(l, 1e-300));
    s1 += z;
    s2 += z * z;
  }
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s1;
    red[1][threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    red[0][0] = a;
    red[1][0] = b;
  }
  __syncthreads();
  const double mean = red[0][0] / D.n_cand;
  const double var = fmax(red[1][0] / D.n_cand - mean * mean, 0.0);
  const double sd = sqrt(var);
  for (int c = threadIdx.x; c < D.n_cand; c += blockDim.x) {
    const double z = log(fmax(lev_all[D.out_off + c], 1e-300));
    target[D.out_off + c] = sd > 1e-12 ? (float)((z - mean) / sd) : 0.f;
  }
}

__global__ void scale_rows_kernel(const RowScaleDesc* descs) {
  const RowScaleDesc D = descs[blockIdx.y];
  const int64_t n = (int64_t)D.rows * D.cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % D.rows), c = (int)(e / D.rows);
    D.B[(size_t)c * D.ld + r] *= r < D.split ? D.w0 : D.w1;
  }
}

size_t fwd_smem() {
  return (size_t)(MLP_W * WS + MLP_W * MLP_F + MWARPS * 16 * WS) * 2 + 3 * MLP_W * 4;
}
size_t bwd_smem() {
  return (size_t)(MLP_W * WS + 3 * MT * WS + MT * MLP_F) * 2 + (4 * MLP_W + 2) * 4;
}

}  // namespace

void learned_candidates(const uint32_t* cand_sorted, const uint64_t* keys_sorted, const int* node_start,
                        const int* node_cnt, int cnt_bits, const int* off, const SampleNodeInfo* info,
                        const LearnNodeInfo* linfo, int nn, uint64_t seed, int max_cand, int* cand,
                        float* hits, int* status, cudaStream_t st) {
  if (nn <= 0 || max_cand <= 0) return;
  int cap = 1;
  while (cap < max_cand) cap <<= 1;
  const size_t smem = (size_t)4 * cap * sizeof(int);
  if (smem > 200 * 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "learned candidate budget too large");
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(candidates_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope _ps(PK_LEARN, st);
  candidates_kernel<<<nn, LC_THREADS, smem, st>>>(cand_sorted, keys_sorted, node_start, node_cnt, cnt_bits,
                                                  off, info, linfo, seed, cap, cand, hits, status);
  IA_LAUNCH_CHECK();
}

void learned_features(const double* Xp, int d, const LearnFeatDesc* descs, int nd, int max_cand,
                      uint16_t* feat, cudaStream_t st) {
  if (nd <= 0 || max_cand <= 0) return;
  const size_t smem = (size_t)(LF_SUB + 1) * d * sizeof(float);
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope _ps(PK_LEARN, st);
  dim3 grid(std::min<unsigned>(ceil_div(max_cand, LF_THREADS), 64), nd);
  features_kernel<<<grid, LF_THREADS, smem, st>>>(Xp, d, descs, feat);
  IA_LAUNCH_CHECK();
}

void mlp_forward(const uint16_t* X, int64_t n, const MlpDev& w, float* y, uint16_t* H1, uint16_t* H2,
                 cudaStream_t st) {
  if (n <= 0) return;
  const size_t smem = fwd_smem();
  IA_CUDA(cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope _ps(PK_MLP, st);
  const int64_t tiles = (n + MT - 1) / MT;
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, 152 * 4);
  mlp_forward_kernel<<<grid, MTHREADS, smem, st>>>(X, n, w, y, H1, H2);
  IA_LAUNCH_CHECK();
}

void mlp_backward(const uint16_t* X, const uint16_t* H1, const uint16_t* H2, const float* y,
                  const float* t, int64_t n, double inv_batch, const MlpDev& w, float* grad,
                  float* loss, cudaStream_t st) {
  if (n <= 0) return;
  const size_t smem = bwd_smem();
  IA_CUDA(cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope _ps(PK_MLP, st);
  const unsigned grid = (unsigned)((n + MT - 1) / MT);
  mlp_backward_kernel<<<grid, MTHREADS, smem, st>>>(X, H1, H2, y, t, n, (float)inv_batch, w, grad, loss);
  IA_LAUNCH_CHECK();
}

void mlp_adam(const MlpDev& w, float* grad, float* m, float* v, int step, double lr, double beta1,
              double beta2, double eps, cudaStream_t st) {
  ProfScope _ps(PK_MLP, st);
  const float c1 = (float)(1.0 - std::pow(beta1, step)), c2 = (float)(1.0 - std::pow(beta2, step));
  mlp_adam_kernel<<<ceil_div(MLP_NPARAM, 256), 256, 0, st>>>(w, grad, m, v, (float)lr, (float)beta1,
                                                             (float)beta2, (float)eps, c1, c2);
  IA_LAUNCH_CHECK();
}

void mlp_refresh_copies(const MlpDev& w, cudaStream_t st) {
  ProfScope _ps(PK_MLP, st);
  mlp_copies_kernel<<<ceil_div(MLP_NPARAM, 256), 256, 0, st>>>(w);
  IA_LAUNCH_CHECK();
}

void perturb_scores(float* score, const LearnNodeInfo* linfo, const SampleNodeInfo* info, int nn,
                    int max_cand, uint64_t seed, double temp, cudaStream_t st) {
  if (nn <= 0 || max_cand <= 0 || temp == 0.0) return;
  ProfScope _ps(PK_LEARN, st);
  perturb_kernel<<<dim3(std::min<unsigned>(ceil_div(max_cand, 256), 16), nn), 256, 0, st>>>(score, linfo, info,
                                                                                            seed, temp);
  IA_LAUNCH_CHECK();
}

void learned_select(const float* score, const int* cand, const LearnNodeInfo* linfo,
                    const SampleNodeInfo* info, int nn, int max_cand, int* samp, cudaStream_t st) {
  if (nn <= 0 || max_cand <= 0) return;
  int cap = 1;
  while (cap < max_cand) cap <<= 1;
  const size_t smem = (size_t)cap * sizeof(unsigned long long);
  if (smem > 200 * 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "learned candidate budget too large");
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope _ps(PK_LEARN, st);
  select_kernel<<<nn, LS_THREADS, smem, st>>>(score, cand, linfo, info, cap, samp);
  IA_LAUNCH_CHECK();
}

void stream_rows(const StreamDesc* descs, int nd, int count, uint64_t seed, uint64_t salt, int* out,
                 cudaStream_t st) {
  if (nd <= 0 || count <= 0) return;
  ProfScope _ps(PK_LEARN, st);
  dim3 grid(std::min<unsigned>(ceil_div(count, 256), 16), nd);
  stream_rows_kernel<<<grid, 256, 0, st>>>(descs, count, seed, salt, out);
  IA_LAUNCH_CHECK();
}

void id_judge(const double* Xp, int d, const JudgeDesc* descs, int nd, int nh, int max_s, double* out,
              cudaStream_t st) {
  if (nd <= 0) return;
  const size_t smem = (size_t)JG_ROWS * std::max(max_s, 1) * sizeof(double);
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(judge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope _ps(PK_JUDGE, st);
  judge_kernel<<<nd, JG_THREADS, smem, st>>>(Xp, d, descs, nh, out);
  IA_LAUNCH_CHECK();
}

void scale_rows(const RowScaleDesc* descs, int nd, cudaStream_t st) {
  if (nd <= 0) return;
  ProfScope _ps(PK_LEARN, st);
  scale_rows_kernel<<<dim3(64, nd), 256, 0, st>>>(descs);
  IA_LAUNCH_CHECK();
}

void gather_cols(const ColsDesc* descs, int nd, int* out, cudaStream_t st) {
  if (nd <= 0) return;
  ProfScope _ps(PK_LEARN, st);
  gather_cols_kernel<<<nd, 256, 0, st>>>(descs, out);
  IA_LAUNCH_CHECK();
}

void add_ridge(const RidgeDesc* descs, int nd, double tol2, cudaStream_t st) {
  if (nd <= 0) return;
  ProfScope _ps(PK_LEARN, st);
  add_ridge_kernel<<<nd, 256, 0, st>>>(descs, tol2);
  IA_LAUNCH_CHECK();
}

void leverage_targets(const LevDesc* descs, int nd, double* lev, float* target, cudaStream_t st) {
  if (nd <= 0) return;
  ProfScope _ps(PK_LEARN, st);
  leverage_kernel<<<nd, 256, 0, st>>>(descs, lev, target);
  IA_LAUNCH_CHECK();
}

}  // namespace iaskit

namespace iaskit {
namespace {
__global__ void gather_train_kernel(const uint16_t* feat, const float* tgt, const int* idx, int n,
                                    uint16_t* of, float* ot) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = idx[i];
  reinterpret_cast<uint4*>(of)[i] = reinterpret_cast<const uint4*>(feat)[r];
  ot[i] = tgt[r];
}
}  // namespace

void gather_train(const uint16_t* feat, const float* tgt, const int* idx, int n, uint16_t* of, float* ot,
                  cudaStream_t st) {
  if (n <= 0) return;
  ProfScope _ps(PK_MLP, st);
  gather_train_kernel<<<ceil_div(n, 256), 256, 0, st>>>(feat, tgt, idx, n, of, ot);
  IA_LAUNCH_CHECK();
}

}  // namespace iaskit
