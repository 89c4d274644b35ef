// Exclusive scan and stable radix sort (see prims.cuh).
#include "prims.cuh"

namespace iaskit {

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-wide exclusive scan of SCAN_TILE consecutive elements; writes the block
// total to block_sums[blockIdx.x] when block_sums is not null.
__global__ void scan_tile_kernel(const int* in, int* out, size_t n, int* block_sums) {
  __shared__ int warp_tot[SCAN_THREADS / 32];
  const size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS];
  int local = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    size_t i = base + k;
    v[k] = (i < n) ? in[i] : 0;
    local += v[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int t = warp_tot[lane];
    int s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += u;
    }
    warp_tot[lane] = s - t;  // exclusive prefix of warp totals
    if (lane == 31 && block_sums) block_sums[blockIdx.x] = s;
  }
  __syncthreads();
  int run = warp_tot[warp] + incl - local;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    size_t i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

__global__ void scan_add_kernel(int* out, size_t n, const int* block_offsets) {
  size_t i = (size_t)blockIdx.x * SCAN_TILE + threadIdx.x;
  int add = block_offsets[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k, i += SCAN_THREADS)
    if (i < n) out[i] += add;
}

void scan_rec(const int* in, int* out, size_t n, int* tmp, size_t tmp_len, cudaStream_t st) {
  if (n == 0) return;
  unsigned nb = ceil_div(n, SCAN_TILE);
  if (nb == 1) {
    scan_tile_kernel<<<1, SCAN_THREADS, 0, st>>>(in, out, n, nullptr);
    IA_LAUNCH_CHECK();
    return;
  }
  if (tmp_len < nb) throw Error(IASKIT_ERR_CUDA, "scan scratch too small");
  int* sums = tmp;
  scan_tile_kernel<<<nb, SCAN_THREADS, 0, st>>>(in, out, n, sums);
  IA_LAUNCH_CHECK();
  scan_rec(sums, sums, nb, tmp + nb, tmp_len - nb, st);
  scan_add_kernel<<<nb, SCAN_THREADS, 0, st>>>(out, n, sums);
  IA_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;

__global__ void radix_hist_kernel(const uint64_t* keys, size_t n, int shift, int* hist,
                                  int ntiles) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const size_t base = (size_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    size_t i = base + (size_t)r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Keys of a tile are taken round by round, thread order inside a round, so the
// rank of a key among equal digits follows the input order: the sort is stable.
__global__ void radix_scatter_kernel(const uint64_t* kin, const uint32_t* vin, uint64_t* kout,
                                     uint32_t* vout, size_t n, int shift, const int* offsets,
                                     int ntiles) {
  __shared__ int wcnt[RS_THREADS / 32][256];
  __shared__ int base[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = offsets[(size_t)tid * ntiles + blockIdx.x];
  const unsigned lt_mask = (1u << lane) - 1u;
  const size_t tile0 = (size_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; ++r) {
#pragma unroll
    for (int w = 0; w < RS_THREADS / 32; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const size_t i = tile0 + (size_t)r * RS_THREADS + tid;
    const bool valid = i < n;
    uint64_t key = valid ? kin[i] : 0;
    const int digit = valid ? (int)((key >> shift) & 255u) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const int rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
    __syncthreads();
    {
      int acc = 0;
#pragma unroll
      for (int w = 0; w < RS_THREADS / 32; ++w) {
        int c = wcnt[w][tid];
        wcnt[w][tid] = base[tid] + acc;
        acc += c;
      }
      base[tid] += acc;
    }
    __syncthreads();
    if (valid) {
      int pos = wcnt[warp][digit] + rank;
      kout[pos] = key;
      if (vin) vout[pos] = vin[i];
    }
    __syncthreads();
  }
}

}  // namespace

void exclusive_scan_i32(const int* in, int* out, size_t n, DevBuf& tmp, cudaStream_t st) {
  if (n == 0) return;
  size_t need = 0, m = n;
  while (m > (size_t)SCAN_TILE) {
    m = ceil_div(m, SCAN_TILE);
    need += m;
  }
  need += 1;
  int* t = tmp.ensure_n<int>(need);
  scan_rec(in, out, n, t, need, st);
}

void radix_sort_u64(uint64_t* keys, uint32_t* vals, size_t n, int nbits, DevBuf& alt_keys,
                    DevBuf& alt_vals, DevBuf& hist, DevBuf& scan_tmp, cudaStream_t st) {
  if (n <= 1 || nbits <= 0) return;
  if (n > (size_t)0x7fffffff) throw Error(IASKIT_ERR_UNSUPPORTED, "radix sort of > 2^31 keys");
  const int ntiles = (int)ceil_div(n, RS_TILE);
  uint64_t* k0 = keys;
  uint64_t* k1 = alt_keys.ensure_n<uint64_t>(n);
  uint32_t* v0 = vals;
  uint32_t* v1 = vals ? alt_vals.ensure_n<uint32_t>(n) : nullptr;
  int* h = hist.ensure_n<int>((size_t)256 * ntiles);
  int passes = 0;
  for (int shift = 0; shift < nbits; shift += 8, ++passes) {
    radix_hist_kernel<<<ntiles, RS_THREADS, 0, st>>>(k0, n, shift, h, ntiles);
    IA_LAUNCH_CHECK();
    exclusive_scan_i32(h, h, (size_t)256 * ntiles, scan_tmp, st);
    radix_scatter_kernel<<<ntiles, RS_THREADS, 0, st>>>(k0, v0, k1, v1, n, shift, h, ntiles);
    IA_LAUNCH_CHECK();
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  if (passes & 1) {
    IA_CUDA(cudaMemcpyAsync(keys, k0, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    if (vals) IA_CUDA(cudaMemcpyAsync(vals, v0, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
  }
}

}  // namespace iaskit
