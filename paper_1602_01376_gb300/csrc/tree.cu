// Tree permutation (Sec. II-A, with the ball tree replaced by a median split).
//
// Level l -> l+1, for every node of level l at once:
//   1. per node and coordinate, min and max over the node's points (orderable
//      64-bit keys, shared-memory reduction, one global atomic per block);
//   2. split coordinate c = argmax (max - min), ties to the lowest coordinate;
//   3. rank the points of each node by (x_c, original index): a stable radix sort
//      by x_c followed by a stable radix sort by node; inside a node the input is in
//      ascending original index, so equal x_c stay in index order;
//   4. flag the first floor(n/2) ranks as "left", and stably partition every node's
//      range by that flag (prefix sum of the flags), so both children keep their
//      points in ascending original index.
// Several independent problems are built together: a level's node list covers all
// points; the nodes of a problem whose tree is already complete are passed through
// unsplit (all their points flagged "left", so the partition leaves them in place).
#include "kernels.cuh"
#include "prims.cuh"

namespace iaskit {

namespace {

__device__ __forceinline__ int node_of(const int* off, int nnodes, int p) {
  int lo = 0, hi = nnodes - 1;  // largest i with off[i] <= p
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

constexpr int MM_WARPS = 8;
constexpr int MM_ROWS_PER_BLOCK = 1024;

// Grid: one block per (node-aligned) chunk of positions.  Dynamic shared memory:
// 2 * MM_WARPS * d uint64 (per-warp min and max keys).
__global__ void minmax_kernel(const double* X, const int* perm, int d, const int* chunk_node,
                              const int* chunk_start, const int* chunk_end, uint64_t* node_min,
                              uint64_t* node_max) {
  extern __shared__ uint64_t sm[];
  uint64_t* smin = sm;
  uint64_t* smax = sm + MM_WARPS * d;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = lane; k < d; k += 32) {
    smin[warp * d + k] = ~0ull;
    smax[warp * d + k] = 0ull;
  }
  __syncwarp();
  const int node = chunk_node[blockIdx.x];
  const int s = chunk_start[blockIdx.x], e = chunk_end[blockIdx.x];
  for (int p = s + warp; p < e; p += MM_WARPS) {
    const double* row = X + (size_t)perm[p] * d;
    for (int k = lane; k < d; k += 32) {
      uint64_t key = orderable_key(row[k]);
      uint64_t* mn = &smin[warp * d + k];
      uint64_t* mx = &smax[warp * d + k];
      if (key < *mn) *mn = key;
      if (key > *mx) *mx = key;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    uint64_t mn = ~0ull, mx = 0ull;
    for (int w = 0; w < MM_WARPS; ++w) {
      mn = min(mn, smin[w * d + k]);
      mx = max(mx, smax[w * d + k]);
    }
    atomicMin((unsigned long long*)&node_min[(size_t)node * d + k], (unsigned long long)mn);
    atomicMax((unsigned long long*)&node_max[(size_t)node * d + k], (unsigned long long)mx);
  }
}

__global__ void init_minmax_kernel(uint64_t* mn, uint64_t* mx, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    mn[i] = ~0ull;
    mx[i] = 0ull;
  }
}

__global__ void choose_dim_kernel(const uint64_t* node_min, const uint64_t* node_max, int nnodes,
                                  int d, int* dims) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnodes) return;
  int best = 0;
  double bs = -1.0;
  for (int k = 0; k < d; ++k) {
    double spread = key_to_double(node_max[(size_t)i * d + k]) -
                    key_to_double(node_min[(size_t)i * d + k]);
    if (spread > bs) {  // strict: ties keep the lowest coordinate
      bs = spread;
      best = k;
    }
  }
  dims[i] = best;
}

__global__ void coord_keys_kernel(const double* X, const int* perm, int N, int d, const int* off,
                                  int nnodes, const int* dims, uint64_t* keys, uint32_t* vals) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  int node = node_of(off, nnodes, p);
  keys[p] = orderable_key(X[(size_t)perm[p] * d + dims[node]]);
  vals[p] = (uint32_t)p;
}

__global__ void node_keys_kernel(const uint32_t* vals, int N, const int* off, int nnodes,
                                 uint64_t* keys) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  keys[q] = (uint64_t)node_of(off, nnodes, (int)vals[q]);
}

__global__ void left_flags_kernel(const uint64_t* node_keys, const uint32_t* vals, int N,
                                  const int* off, const int* kleft, int* flags) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  int node = (int)node_keys[q];
  int o = off[node];
  flags[vals[q]] = (q - o) < kleft[node] ? 1 : 0;
}

__global__ void partition_kernel(const int* perm, const int* flags, const int* pre, int N,
                                 const int* off, const int* kleft, int nnodes, int* perm_out) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  int node = node_of(off, nnodes, p);
  int o = off[node];
  int nl = pre[p] - pre[o];  // left-flagged positions in [o, p)
  int dest = flags[p] ? o + nl : o + kleft[node] + (p - o - nl);
  perm_out[dest] = perm[p];
}

__global__ void iota_kernel(int* a, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

__global__ void permute_points_kernel(const double* X, const int* perm, int N, int d, int* iperm,
                                      double* Xp) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)N * d) return;
  int p = (int)(t / d), k = (int)(t % d);
  int src = perm[p];
  Xp[t] = X[(size_t)src * d + k];
  if (k == 0) iperm[src] = p;
}

int bit_length(uint64_t v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

}  // namespace

void build_tree(const double* X, int N, int d, const std::vector<TreeLevel>& levels, int* perm,
                TreeScratch& s, cudaStream_t st) {
  ProfScope _ps(PK_TREE, st);
  const int T = 256;
  iota_kernel<<<ceil_div(N, T), T, 0, st>>>(perm, N);
  IA_LAUNCH_CHECK();
  if (levels.empty()) return;
  uint64_t* keys = s.keys.ensure_n<uint64_t>(N);
  uint32_t* vals = s.vals.ensure_n<uint32_t>(N);
  int* flags = s.flags.ensure_n<int>(N);
  int* pre = s.pre.ensure_n<int>(N);
  int* perm2 = s.perm2.ensure_n<int>(N);
  size_t max_nodes = 1;
  for (const TreeLevel& lv : levels) max_nodes = std::max(max_nodes, lv.kleft.size());
  uint64_t* mm = s.minmax.ensure_n<uint64_t>((size_t)2 * max_nodes * d);
  int* dims = s.dims.ensure_n<int>(max_nodes);
  for (const TreeLevel& lv : levels) {
    const int nn = (int)lv.kleft.size();
    const std::vector<int>& off = lv.off;
    // chunk list: ranges of at most MM_ROWS_PER_BLOCK positions of the split nodes
    std::vector<int> cn, cs, ce;
    for (int i = 0; i < nn; ++i) {
      if (!lv.split[i]) continue;
      for (int a = off[i]; a < off[i + 1]; a += MM_ROWS_PER_BLOCK) {
        cn.push_back(i);
        cs.push_back(a);
        ce.push_back(std::min(off[i + 1], a + MM_ROWS_PER_BLOCK));
      }
    }
    const int nch = (int)cn.size();
    std::vector<int> host(2 * (size_t)nn + 1 + 3 * (size_t)nch);
    std::copy(off.begin(), off.end(), host.begin());
    std::copy(lv.kleft.begin(), lv.kleft.end(), host.begin() + nn + 1);
    std::copy(cn.begin(), cn.end(), host.begin() + 2 * nn + 1);
    std::copy(cs.begin(), cs.end(), host.begin() + 2 * nn + 1 + nch);
    std::copy(ce.begin(), ce.end(), host.begin() + 2 * nn + 1 + 2 * nch);
    int* dev = s.offs.ensure_n<int>(host.size());
    h2d(dev, host.data(), host.size(), st);
    const int* doff = dev;
    const int* dkl = dev + nn + 1;
    const int* dcn = dkl + nn;
    const int* dcs = dcn + nch;
    const int* dce = dcs + nch;
    uint64_t* nmin = mm;
    uint64_t* nmax = mm + (size_t)nn * d;
    init_minmax_kernel<<<ceil_div((size_t)nn * d, T), T, 0, st>>>(nmin, nmax, nn * d);
    IA_LAUNCH_CHECK();
    if (nch > 0) {
      minmax_kernel<<<nch, MM_WARPS * 32, 2 * MM_WARPS * d * sizeof(uint64_t), st>>>(
          X, perm, d, dcn, dcs, dce, nmin, nmax);
      IA_LAUNCH_CHECK();
    }
    choose_dim_kernel<<<ceil_div(nn, T), T, 0, st>>>(nmin, nmax, nn, d, dims);
    IA_LAUNCH_CHECK();
    coord_keys_kernel<<<ceil_div(N, T), T, 0, st>>>(X, perm, N, d, doff, nn, dims, keys, vals);
    IA_LAUNCH_CHECK();
    radix_sort_u64(keys, vals, N, 64, s.alt_keys, s.alt_vals, s.hist, s.scan_tmp, st);
    if (nn > 1) {
      node_keys_kernel<<<ceil_div(N, T), T, 0, st>>>(vals, N, doff, nn, keys);
      IA_LAUNCH_CHECK();
      radix_sort_u64(keys, vals, N, bit_length((uint64_t)(nn - 1)), s.alt_keys, s.alt_vals, s.hist,
                     s.scan_tmp, st);
    } else {
      IA_CUDA(cudaMemsetAsync(keys, 0, (size_t)N * sizeof(uint64_t), st));
    }
    left_flags_kernel<<<ceil_div(N, T), T, 0, st>>>(keys, vals, N, doff, dkl, flags);
    IA_LAUNCH_CHECK();
    exclusive_scan_i32(flags, pre, N, s.scan_tmp, st);
    partition_kernel<<<ceil_div(N, T), T, 0, st>>>(perm, flags, pre, N, doff, dkl, nn, perm2);
    IA_LAUNCH_CHECK();
    IA_CUDA(cudaMemcpyAsync(perm, perm2, (size_t)N * sizeof(int), cudaMemcpyDeviceToDevice, st));
    // the host vectors above are consumed by the copies before they go out of scope
    IA_CUDA(cudaStreamSynchronize(st));
  }
}

void permute_points(const double* X, const int* perm, int N, int d, int* iperm, double* Xp,
                    cudaStream_t st) {
  ProfScope _ps(PK_TREE, st);
  const size_t n = (size_t)N * d;
  permute_points_kernel<<<ceil_div(n, 256), 256, 0, st>>>(X, perm, N, d, iperm, Xp);
  IA_LAUNCH_CHECK();
}

}  // namespace iaskit
