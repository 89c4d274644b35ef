// Near-field correction S of the kNN-separated operator lambda I + K~ + S (eq. askit,
// Sec. II-B).  ASKIT's second separation rule calls a target i separated from a node
// alpha only when none of i's nearest neighbours lies in alpha; the hierarchical matrix
// of eq. (offdiag-askit) is kept, and for every node alpha that the Evaluate step
// reaches for i under the first rule (the sibling of each ancestor of i's leaf) and that
// holds a neighbour of i, the skeleton evaluation K_{i a~} w~_a is replaced by the exact
// K_{i a} w_a.  The operator apply adds that difference after its Evaluate step.
//
// One warp per target position.  The levels of the target's list that hold a neighbour
// come from the first split at which each neighbour's root-to-leaf path leaves the
// target's (node sizes follow the tree's median split: left = size / 2); the warp then
// sums, per such node, the exact row over the node's points minus the skeleton row over
// its w~, lanes striding over the points, and lane 0 adds the sums to the target's row.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

namespace iaskit {

namespace {

constexpr int NF_WARPS = 8;  // warps (targets in flight) per block
constexpr int NF_CB = 8;     // right-hand sides per pass over a node

__device__ __forceinline__ double nf_kernel(const double* xs, const double* xj, int d, double scale) {
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    const double t = xs[k] - xj[k];
    s = fma(t, t, s);
  }
  return exp(s * scale);
}

__global__ void __launch_bounds__(NF_WARPS * 32)
    near_field_kernel(const double* Xp, int d, const int* knn_pos, int kappa, const int* pid,
                      const NearProb* probs, const NearNode* nodes, const int* skel, int s_max,
                      const double* W, const double* WT, double* U, int nrhs, int Ntot) {
  extern __shared__ double nf_x[];  // NF_WARPS x d: each warp's target coordinates
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* xs = nf_x + (size_t)wib * d;
  for (int p = blockIdx.x * NF_WARPS + wib; p < Ntot; p += gridDim.x * NF_WARPS) {
    const NearProb P = probs[pid[p]];
    if (P.L == 0) continue;
    // bit l: the level-l node of p's list holds a neighbour of p
    unsigned mask = 0;
    for (int t = lane; t < kappa; t += 32) {
      const int q = knn_pos[(size_t)p * kappa + t];
      int off = P.pbase, size = P.N;
      for (int l = 0; l < P.L; ++l) {
        const int half = size / 2;
        const bool pl = p < off + half, ql = q < off + half;
        if (pl != ql) {
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
    mask = __reduce_or_sync(0xffffffffu, mask);
    if (mask == 0) continue;
    __syncwarp();
    for (int k = lane; k < d; k += 32) xs[k] = Xp[(size_t)p * d + k];
    __syncwarp();
    const size_t blk = (size_t)P.pbase * nrhs + (size_t)(p - P.pbase);  // row p of its block
    while (mask) {
      const int l = __ffs(mask) - 1;
      mask &= mask - 1;
      // the level-l node of the list: p's path for l - 1 splits, then the other side
      int off = P.pbase, size = P.N, uid = 1;
      for (int ll = 0; ll < l; ++ll) {
        const int half = size / 2;
        const bool pl = p < off + half;
        const bool left = (ll < l - 1) ? pl : !pl;
        if (left) {
          size = half;
          uid = 2 * uid;
        } else {
          off += half;
          size -= half;
          uid = 2 * uid + 1;
        }
      }
      const int g = P.nbase + uid;
      const NearNode A = nodes[g];
      const int* sk = skel + (size_t)g * s_max;
      for (int c0 = 0; c0 < nrhs; c0 += NF_CB) {
        const int nc = min(NF_CB, nrhs - c0);
        double acc[NF_CB];
#pragma unroll
        for (int c = 0; c < NF_CB; ++c) acc[c] = 0.0;
        for (int j = off + lane; j < off + size; j += 32) {  // exact: K(x_p, X_alpha) w_alpha
          const double kv = nf_kernel(xs, Xp + (size_t)j * d, d, P.scale);
          const double* wj = W + (size_t)P.pbase * nrhs + (size_t)(j - P.pbase) + (size_t)c0 * P.N;
#pragma unroll
          for (int c = 0; c < NF_CB; ++c)
            if (c < nc) acc[c] = fma(kv, wj[(size_t)c * P.N], acc[c]);
        }
        for (int k = lane; k < A.s; k += 32) {  // minus the skeleton row: K(x_p, X_skel) w~
          const double kv = nf_kernel(xs, Xp + (size_t)sk[k] * d, d, P.scale);
          const double* wt = WT + A.wt_off + k + (size_t)c0 * A.ld;
#pragma unroll
          for (int c = 0; c < NF_CB; ++c)
            if (c < nc) acc[c] = fma(-kv, wt[(size_t)c * A.ld], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < NF_CB; ++c)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        if (lane == 0)
          for (int c = 0; c < nc; ++c) U[blk + (size_t)(c0 + c) * P.N] += acc[c];
      }
    }
  }
}

}  // namespace

void near_field(const double* Xp, int d, const int* knn_pos, int kappa, const int* pid, const NearProb* probs,
                const NearNode* nodes, const int* skel, int s_max, const double* W, const double* WT, double* U,
                int nrhs, int Ntot, cudaStream_t st) {
  if (Ntot <= 0 || kappa <= 0 || nrhs <= 0) return;
  const size_t smem = (size_t)NF_WARPS * d * sizeof(double);
  if (smem > 200 * 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "dimension too large for the near-field kernel");
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(near_field_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope _ps(PK_NEAR, st);
  const int blocks = (int)std::min<int64_t>((Ntot + NF_WARPS - 1) / NF_WARPS, 152 * 16);
  near_field_kernel<<<blocks, NF_WARPS * 32, smem, st>>>(Xp, d, knn_pos, kappa, pid, probs, nodes, skel, s_max,
                                                          W, WT, U, nrhs, Ntot);
  IA_LAUNCH_CHECK();
}

}  // namespace iaskit
