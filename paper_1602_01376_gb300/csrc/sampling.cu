// Row sampling for skeletonization (Sec. II-B: nearest-neighbour information
// guides the sampling of K_{[1:N] alpha}).
//
// For node alpha of level l owning permuted positions [o, o + n):
//   1. candidates are the kNN entries (as positions) of alpha's points that fall
//      outside alpha; hits(c) counts their multiplicity;
//   2. n_samp = min(samp_cap, N - n); the first n_samp distinct candidates in the
//      order (hits descending, position ascending) are kept;
//   3. a shortfall is filled uniformly without replacement from the complement of
//      alpha with the node's SplitMix64 stream: state s0 = splitmix64(splitmix64(seed)
//      ^ uid), uid = 2^l + i, draw q is splitmix64(s0 + q * gamma); j = draw mod (N - n)
//      maps to position j (j < o) or j + n; positions already taken are skipped;
//      when n_samp = N - n the sample is the whole complement;
//   4. the sample is returned in ascending position order.
// Several independent problems are sampled together: a step's node list covers
// all points; nodes of problems that have no node at this step only pass through.
// Positions, complements and streams are per problem, so every node gets exactly
// the sample it would get alone.
// Device plan per step: one radix sort of (node, candidate) keys over all N*kappa
// entries gives the hit counts as run lengths; a second stable radix sort by
// (node, hits descending) puts each node's best candidates first (the first sort
// left equal hits in ascending position); one block per node then fills and sorts.
#include <climits>

#include "kernels.cuh"
#include "prims.cuh"

namespace iaskit {

namespace {

__device__ __forceinline__ int node_of(const int* off, int nnodes, int p) {
  int lo = 0, hi = nnodes - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

int bit_length(uint64_t v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

__global__ void knn_pos_kernel(const int* knn, const int* perm, const int* iperm, int N, int kappa,
                               int* knn_pos) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)N * kappa) return;
  int p = (int)(t / kappa), k = (int)(t % kappa);
  knn_pos[t] = iperm[knn[(size_t)perm[p] * kappa + k]];
}

__global__ void cand_keys_kernel(const int* knn_pos, int N, int kappa, const int* off,
                                 const SampleNodeInfo* info, int nnodes, int pos_bits,
                                 uint64_t sentinel, uint64_t* keys) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)N * kappa) return;
  int p = (int)(t / kappa);
  int node = node_of(off, nnodes, p);
  int c = knn_pos[t];
  bool outside = info[node].active && (c < off[node] || c >= off[node + 1]);
  keys[t] = outside ? (((uint64_t)node << pos_bits) | (uint64_t)c) : sentinel;
}

__global__ void run_heads_kernel(const uint64_t* keys, size_t n, uint64_t sentinel, int* heads) {
  size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  uint64_t k = keys[q];
  heads[q] = (k != sentinel && (q == 0 || keys[q - 1] != k)) ? 1 : 0;
}

__global__ void runs_kernel(const uint64_t* keys, size_t n, uint64_t sentinel, const int* heads,
                            const int* idx, int* run_start, int* run_end, uint64_t* run_key) {
  size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  uint64_t k = keys[q];
  if (k == sentinel) return;
  int r = idx[q] + heads[q] - 1;
  if (heads[q]) {
    run_start[r] = (int)q;
    run_key[r] = k;
  }
  if (q + 1 == n || keys[q + 1] != k) run_end[r] = (int)q + 1;
}

__global__ void rank_keys_kernel(const int* run_start, const int* run_end, const uint64_t* run_key,
                                 int nruns, int pos_bits, int cnt_bits, uint64_t* keys2,
                                 uint32_t* vals2, int* node_cnt) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = r < nruns;
  uint64_t node = ~0ull;
  if (in) {
    const uint64_t k = run_key[r];
    node = k >> pos_bits;
    const uint32_t c = (uint32_t)(k & ((1ull << pos_bits) - 1));
    const uint64_t cnt = (uint64_t)(run_end[r] - run_start[r]);
    const uint64_t inv = ((1ull << cnt_bits) - 1) - cnt;
    keys2[r] = (node << cnt_bits) | inv;
    vals2[r] = c;
  }
  // runs are sorted by node: the lanes of one node add their count once
  const unsigned same = __match_any_sync(0xffffffffu, node);
  if (in && (threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&node_cnt[node], __popc(same));
}

// One block per node.  Shared memory: cap_pow2 ints for the sample and a hash set
// of 4 * cap_pow2 ints.
constexpr int SEL_THREADS = 256;
__global__ void select_fill_kernel(const uint32_t* cand_sorted, const int* node_start,
                                   const int* node_cnt, const int* off,
                                   const SampleNodeInfo* info, int samp_cap, uint64_t seed,
                                   int cap_pow2, int* samp, int* status) {
  extern __shared__ int sh[];
  int* arr = sh;
  int* hset = sh + cap_pow2;
  const int hsize = 4 * cap_pow2;
  const int node = blockIdx.x;
  const SampleNodeInfo inf = info[node];
  if (!inf.active) return;
  const int pb = inf.pb;                              // first point of the node's problem
  const int o = off[node] - pb, n = off[node + 1] - off[node];   // o: offset inside the problem
  const int comp = inf.pn - n;
  const int ns = min(samp_cap, comp);
  int* out = samp + inf.samp_off;
  if (ns <= 0) return;
  if (ns == comp) {  // the whole complement, already ascending
    for (int t = threadIdx.x; t < comp; t += SEL_THREADS) out[t] = pb + (t < o ? t : t + n);
    return;
  }
  const int nc = min(ns, node_cnt[node]);
  const uint32_t* cand = cand_sorted + node_start[node];
  for (int t = threadIdx.x; t < cap_pow2; t += SEL_THREADS) arr[t] = t < nc ? (int)cand[t] : INT_MAX;
  for (int t = threadIdx.x; t < hsize; t += SEL_THREADS) hset[t] = -1;
  __syncthreads();
  if (threadIdx.x == 0 && nc < ns) {
    auto insert = [&](int pos) -> bool {  // true if newly inserted
      uint32_t hh = ((uint32_t)pos * 2654435761u) & (uint32_t)(hsize - 1);
      while (true) {
        int v = hset[hh];
        if (v == pos) return false;
        if (v < 0) {
          hset[hh] = pos;
          return true;
        }
        hh = (hh + 1) & (uint32_t)(hsize - 1);
      }
    };
    for (int t = 0; t < nc; ++t) insert(arr[t]);
    int have = nc;
    const uint64_t uid = (uint64_t)inf.uid;
    const uint64_t s0 = splitmix64(splitmix64(seed) ^ uid);
    const uint64_t limit = 64ull * (uint64_t)comp + 4096ull;
    uint64_t q = 0;
    while (have < ns) {
      if (q >= limit) {
        atomicOr(status, DEV_OVERFLOW);
        break;
      }
      uint64_t r = splitmix64(s0 + q * 0x9E3779B97F4A7C15ull);
      int j = (int)(r % (uint64_t)comp);
      int pos = pb + (j < o ? j : j + n);
      if (insert(pos)) arr[have++] = pos;
      ++q;
    }
  }
  __syncthreads();
  // bitonic sort of arr[0 .. cap_pow2) ascending (INT_MAX padding sorts last)
  for (int k = 2; k <= cap_pow2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < cap_pow2; t += SEL_THREADS) {
        int partner = t ^ j;
        if (partner > t) {
          bool up = (t & k) == 0;
          int a = arr[t], b = arr[partner];
          if ((a > b) == up) {
            arr[t] = b;
            arr[partner] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < ns; t += SEL_THREADS) out[t] = arr[t];
}

}  // namespace

void knn_to_positions(const int* knn, const int* perm, const int* iperm, int N, int kappa,
                      int* knn_pos, cudaStream_t st) {
  ProfScope _ps(PK_SAMPLE, st);
  size_t n = (size_t)N * kappa;
  knn_pos_kernel<<<ceil_div(n, 256), 256, 0, st>>>(knn, perm, iperm, N, kappa, knn_pos);
  IA_LAUNCH_CHECK();
}

void sample_level(const int* knn_pos, int N, int kappa, const int* off_dev,
                  const SampleNodeInfo* info_dev, const std::vector<int>& off_host,
                  const std::vector<SampleNodeInfo>& info_host, int samp_cap, uint64_t seed,
                  int* samp, int* dev_status, SampleScratch& s, cudaStream_t st) {
  ProfScope _ps(PK_SAMPLE, st);
  const int nn = (int)info_host.size();
  const size_t n = (size_t)N * kappa;
  int node_bits = 0;
  while ((1 << node_bits) < nn) ++node_bits;
  const int pos_bits = bit_length((uint64_t)N);   // 2^pos_bits > N: the sentinel is no position
  const int key_bits = node_bits + pos_bits;
  if (key_bits > 62) throw Error(IASKIT_ERR_UNSUPPORTED, "sampling key exceeds 62 bits");
  const uint64_t sentinel = (1ull << key_bits) - 1;
  uint64_t* keys = s.keys.ensure_n<uint64_t>(n);
  cand_keys_kernel<<<ceil_div(n, 256), 256, 0, st>>>(knn_pos, N, kappa, off_dev, info_dev, nn,
                                                     pos_bits, sentinel, keys);
  IA_LAUNCH_CHECK();
  radix_sort_u64(keys, nullptr, n, key_bits, s.alt_keys, s.alt_vals, s.hist, s.scan_tmp, st);
  int* heads = s.flags.ensure_n<int>(n);
  int* idx = s.idx.ensure_n<int>(n);
  run_heads_kernel<<<ceil_div(n, 256), 256, 0, st>>>(keys, n, sentinel, heads);
  IA_LAUNCH_CHECK();
  exclusive_scan_i32(heads, idx, n, s.scan_tmp, st);
  int last_idx = 0, last_head = 0;
  d2h(&last_idx, idx + n - 1, 1, st);
  d2h(&last_head, heads + n - 1, 1, st);
  IA_CUDA(cudaStreamSynchronize(st));
  const int nruns = last_idx + last_head;
  int* run_start = s.run_start.ensure_n<int>(nruns + 1);
  int* run_end = s.run_end.ensure_n<int>(nruns + 1);
  uint64_t* run_key = s.run_key.ensure_n<uint64_t>(nruns + 1);
  int* node_cnt = s.node_cnt.ensure_n<int>(nn + 1);
  int* node_start = s.node_start.ensure_n<int>(nn + 1);
  IA_CUDA(cudaMemsetAsync(node_cnt, 0, (nn + 1) * sizeof(int), st));
  uint64_t* keys2 = s.keys2.ensure_n<uint64_t>(nruns + 1);
  uint32_t* vals2 = s.vals2.ensure_n<uint32_t>(nruns + 1);
  const int cnt_bits = pos_bits;  // a candidate is hit at most once per point of the node
  if (nruns > 0) {
    runs_kernel<<<ceil_div(n, 256), 256, 0, st>>>(keys, n, sentinel, heads, idx, run_start,
                                                  run_end, run_key);
    IA_LAUNCH_CHECK();
    rank_keys_kernel<<<ceil_div(nruns, 256), 256, 0, st>>>(run_start, run_end, run_key, nruns,
                                                           pos_bits, cnt_bits, keys2, vals2,
                                                           node_cnt);
    IA_LAUNCH_CHECK();
    radix_sort_u64(keys2, vals2, nruns, node_bits + cnt_bits, s.alt_keys, s.alt_vals, s.hist,
                   s.scan_tmp, st);
  }
  exclusive_scan_i32(node_cnt, node_start, nn, s.scan_tmp, st);
  int maxns = 0;
  for (int i = 0; i < nn; ++i)
    if (info_host[i].active)
      maxns = std::max(maxns, std::min(samp_cap, info_host[i].pn - (off_host[i + 1] - off_host[i])));
  int cap_pow2 = 1;
  while (cap_pow2 < maxns) cap_pow2 <<= 1;
  const size_t smem = (size_t)5 * cap_pow2 * sizeof(int);
  if (smem > 200 * 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "sample size too large");
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(select_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  select_fill_kernel<<<nn, SEL_THREADS, smem, st>>>(vals2, node_start, node_cnt, off_dev, info_dev,
                                                    samp_cap, seed, cap_pow2, samp, dev_status);
  IA_LAUNCH_CHECK();
}

}  // namespace iaskit
