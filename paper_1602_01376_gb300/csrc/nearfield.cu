// Near-field correction S of the kNN-separated operator lambda I + K~ + S (eq. askit,
// Sec. II-B).  ASKIT's second separation rule calls a target i separated from a node
// alpha only when none of i's nearest neighbours lies in alpha; the hierarchical matrix
// of eq. (offdiag-askit) is kept, and for every node alpha that the Evaluate step
// reaches for i under the first rule (the sibling of each ancestor of i's leaf) and that
// holds a neighbour of i, the skeleton evaluation K_{i a~} w~_a is replaced by the exact
// K_{i a} w_a.  The operator apply adds that difference after its Evaluate step.
//
// The pairs (target, node) are grouped by node: near_masks marks, per target, the levels
// of its list whose node holds a neighbour (the level at which each neighbour's
// root-to-leaf path leaves the target's; node sizes follow the tree's median split:
// left = size / 2), and the host collects, per node alpha, the targets that need it
// (all of them in the sibling of alpha).  The sums then run as tiles: 64 targets of one
// node's list against 64 of its columns at a time (the node's points, then its
// skeletons with the opposite sign), both staged in shared memory so that every column
// serves 64 targets, FP64 kernel values in the Gram form |x|^2 + |y|^2 - 2 x.y (as
// kernel_blocks), the tile kept in shared memory for the products with the weights.
// A node's columns are split into chunks (the caller's items), each writing its
// partial sums; near_reduce adds a list's chunks in a fixed order, so the result does
// not depend on scheduling.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

IA_KERNEL_SPEC_TU(kspec_set_near)

namespace iaskit {

namespace {

constexpr int NF_T = 64;        // targets per tile and columns per shared-memory step
constexpr int NF_THREADS = 256;
constexpr int NF_RMAX = 64;     // right-hand sides per launch (16 per thread group)

__global__ void near_mask_kernel(const int* knn_pos, int kappa, const int* pid, const NearProb* probs, int Ntot,
                                 unsigned* masks) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Ntot) return;
  const NearProb P = probs[pid[p]];
  unsigned mask = 0;
  for (int t = 0; t < kappa && P.L > 0; ++t) {
    const int q = knn_pos[(size_t)p * kappa + t];
    int off = P.pbase, size = P.N;
    for (int l = 0; l < P.L; ++l) {
      const int half = size / 2;
      const bool pl = p < off + half, ql = q < off + half;
      if (pl != ql) {  // the level-(l+1) node of p's list holds q
        mask |= 1u << (l + 1);
        break;
      }
      if (pl) {
        size = half;
      } else {
        off += half;
        size -= half;
      }
    }
  }
  masks[p] = mask;
}

// One block per item: targets r0 .. r0 + 63 of a node's list against the item's
// columns; part[item.part + t + r 64] = sign * sum_j K(x_t, x_j) y_j,r.
__global__ void __launch_bounds__(NF_THREADS) near_tile_kernel(const double* Xp, const double* xn, int d, int nrhs,
                                                               const NearItem* items) {
  extern __shared__ double nf_sh[];
  double* xt = nf_sh;                          // [d][NF_T] targets
  double* xc = xt + (size_t)d * NF_T;          // [d][NF_T] columns
  double* Ks = xc + (size_t)d * NF_T;          // [NF_T][NF_T + 1] kernel tile
  double* ws = Ks + NF_T * (NF_T + 1);         // [NF_T][nrhs] weights
  __shared__ double nt_s[NF_T], nc_s[NF_T];
  __shared__ int pos_t[NF_T], pos_c[NF_T];
  const NearItem I = items[blockIdx.x];
  const int tid = threadIdx.x;
  const int nt = min(NF_T, I.n - I.r0);
  if (tid < NF_T) {
    const int p = tid < nt ? I.tgt[I.r0 + tid] : I.tgt[I.r0];
    pos_t[tid] = p;
    nt_s[tid] = xn[p];
  }
  __syncthreads();
  for (int e = tid; e < NF_T * d; e += NF_THREADS) {
    const int t = e / d, k = e % d;
    xt[(size_t)k * NF_T + t] = Xp[(size_t)pos_t[t] * d + k];
  }
  // products: thread (t, q) owns target t and the right-hand sides q, q + 4, ...
  const int mt = tid % NF_T, mq = tid / NF_T;
  double acc[NF_RMAX / 4];
#pragma unroll
  for (int i = 0; i < NF_RMAX / 4; ++i) acc[i] = 0.0;
  const int tx = tid % 16, ty = tid / 16;  // kernel tile: 4 targets x 4 columns per thread
  for (int j0 = 0; j0 < I.ncols; j0 += NF_T) {
    const int nc = min(NF_T, I.ncols - j0);
    __syncthreads();  // the previous step's readers are done
    if (tid < NF_T) {
      const int j = min(j0 + tid, I.ncols - 1);
      const int c = I.cols ? I.cols[j] : I.col0 + j;
      pos_c[tid] = c;
      nc_s[tid] = xn[c];
    }
    __syncthreads();
    for (int e = tid; e < NF_T * d; e += NF_THREADS) {
      const int j = e / d, k = e % d;
      xc[(size_t)k * NF_T + j] = Xp[(size_t)pos_c[j] * d + k];
    }
    for (int e = tid; e < NF_T * nrhs; e += NF_THREADS) {
      const int j = e % NF_T, r = e / NF_T;
      ws[(size_t)j * nrhs + r] = j < nc ? I.y[(size_t)(j0 + j) + (size_t)r * I.ldy] : 0.0;
    }
    __syncthreads();
    double dot[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) dot[a][b] = 0.0;
    for (int k = 0; k < d; ++k) {
      double a4[4], b4[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        a4[a] = xt[(size_t)k * NF_T + tx + 16 * a];
        b4[a] = xc[(size_t)k * NF_T + ty + 16 * a];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) dot[a][b] = fma(a4[a], b4[b], dot[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int t = tx + 16 * a, j = ty + 16 * b;
        const double d2 = fmax((nt_s[t] + nc_s[j]) - 2.0 * dot[a][b], 0.0);
        Ks[t * (NF_T + 1) + j] = (t < nt && j < nc) ? kspec_value(g_kspec, dot[a][b], d2, I.scale) : 0.0;
      }
    __syncthreads();
    for (int j = 0; j < nc; ++j) {
      const double kv = Ks[mt * (NF_T + 1) + j];
      const double* wj = ws + (size_t)j * nrhs;
#pragma unroll
      for (int i = 0; i < NF_RMAX / 4; ++i) {
        const int r = mq + 4 * i;
        if (r < nrhs) acc[i] = fma(kv, wj[r], acc[i]);
      }
    }
  }
  if (mt < nt)
#pragma unroll
    for (int i = 0; i < NF_RMAX / 4; ++i) {
      const int r = mq + 4 * i;
      if (r < nrhs) I.part[(size_t)mt + (size_t)r * NF_T] = I.sign * acc[i];
    }
}

// U[tgt[t] - pbase + r ldu] += sum over the list's chunks, in order, of the partials of
// target t (tile t / 64); one grid row per list.
__global__ void near_reduce_kernel(const NearReduce* lists, int nrhs, double* U) {
  const NearReduce R = lists[blockIdx.y];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < R.n * nrhs; e += gridDim.x * blockDim.x) {
    const int t = e % R.n, r = e / R.n;
    const double* p = R.part + (size_t)(t / NF_T) * R.nchunks * NF_T * nrhs + (t % NF_T) + (size_t)r * NF_T;
    double s = 0.0;
    for (int c = 0; c < R.nchunks; ++c) s += p[(size_t)c * NF_T * nrhs];
    U[R.ubase + (size_t)(R.tgt[t] - R.pbase) + (size_t)r * R.ldu] += s;
  }
}

}  // namespace

void near_masks(const int* knn_pos, int kappa, const int* pid, const NearProb* probs, int Ntot, unsigned* masks,
                cudaStream_t st) {
  if (Ntot <= 0) return;
  ProfScope _ps(PK_NEAR, st);
  near_mask_kernel<<<ceil_div((size_t)Ntot, 256), 256, 0, st>>>(knn_pos, kappa, pid, probs, Ntot, masks);
  IA_LAUNCH_CHECK();
}

int near_tile_rows() { return NF_T; }
int near_max_rhs() { return NF_RMAX; }

void near_tiles(const double* Xp, const double* xn, int d, int nrhs, const NearItem* items_dev, int nitems,
                const NearReduce* lists_dev, int nlists, int max_list, double* U, cudaStream_t st) {
  if (nitems <= 0) return;
  if (nrhs < 1 || nrhs > NF_RMAX) throw Error(IASKIT_ERR_ARG, "near field: nrhs above 64 per launch");
  const size_t smem = sizeof(double) * ((size_t)2 * d * NF_T + NF_T * (NF_T + 1) + (size_t)NF_T * nrhs);
  if (smem > 220 * 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "dimension too large for the near-field kernel");
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(near_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope _ps(PK_NEAR, st);
  near_tile_kernel<<<nitems, NF_THREADS, smem, st>>>(Xp, xn, d, nrhs, items_dev);
  IA_LAUNCH_CHECK();
  for (int l0 = 0; l0 < nlists; l0 += 65535) {
    dim3 grid(std::min<unsigned>(ceil_div((size_t)max_list * nrhs, 256), 4096), (unsigned)std::min(65535, nlists - l0));
    near_reduce_kernel<<<grid, 256, 0, st>>>(lists_dev + l0, nrhs, U);
    IA_LAUNCH_CHECK();
  }
}

}  // namespace iaskit
