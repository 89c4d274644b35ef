// Exact kernel sums at test points, K(x_test, X) w (Sec. III, "Kernel regression for
// binary classification": a test point x gets the label sign(K(x, X) w), K(x, X) the
// exact kernel row over all training points X).  The same sums at training points
// give the exact K w that the sampled error eps_M of eq. (error) compares with K~ w.
//
// One thread per test point; the training points stream through shared memory in
// tiles of PR_TILE.  Every kernel value is evaluated in FP64 in the Gram form
// |x|^2 + |y|^2 - 2 x.y with the training points' precomputed squared norms (the
// form of kernel_blocks: its cancellation error, about 2^-52 (|x|^2 + |y|^2), moves a
// kernel value by a relative 2^-52 (|x|^2 + |y|^2) / (2 h^2)).  The training points
// are split into chunks so that the grid fills the GPU when there are few test
// points; each chunk writes its partial sums and a second kernel adds the chunks in
// order, so the result does not depend on scheduling.
#include "kernels.cuh"

IA_KERNEL_SPEC_TU(kspec_set_predict)

namespace iaskit {

namespace {

constexpr int PR_THREADS = 128;  // test points per block
constexpr int PR_TILE = 64;      // training points per shared-memory tile
constexpr int PR_R = 4;          // right-hand-side columns per pass

// part[c][r][i] = sum over training points j of chunk c of K(t_i, x_j) w[j][r]
// (training points in permuted order j, weights read through perm from the
// problem's original order).
__global__ void __launch_bounds__(PR_THREADS) predict_partial_kernel(
    const double* T, int M, const double* Xp, const double* xn, const int* perm, int pbase, int N, int d,
    double scale, const double* w, int ldw, int nrhs, int chunk, double* part) {
  extern __shared__ double pr_sh[];
  double* xs = pr_sh;                        // [PR_TILE][d]
  double* xcn = xs + (size_t)PR_TILE * d;    // [PR_TILE]
  double* ws = xcn + PR_TILE;                // [PR_R][PR_TILE]
  const int i = blockIdx.x * PR_THREADS + threadIdx.x;
  const bool active = i < M;
  const double* t = T + (size_t)(active ? i : 0) * d;
  double tn = 0.0;
  for (int q = 0; q < d; ++q) tn = fma(t[q], t[q], tn);
  const int j0 = blockIdx.y * chunk, j1 = min(N, j0 + chunk);
  for (int c0 = 0; c0 < nrhs; c0 += PR_R) {
    const int nr = min(PR_R, nrhs - c0);
    double acc[PR_R];
#pragma unroll
    for (int c = 0; c < PR_R; ++c) acc[c] = 0.0;
    for (int k0 = j0; k0 < j1; k0 += PR_TILE) {
      const int nt = min(PR_TILE, j1 - k0);
      __syncthreads();
      for (int e = threadIdx.x; e < nt * d; e += PR_THREADS) {
        const int kk = e / d, q = e % d;
        xs[(size_t)kk * d + q] = Xp[(size_t)(pbase + k0 + kk) * d + q];
      }
      for (int kk = threadIdx.x; kk < nt; kk += PR_THREADS) {
        xcn[kk] = xn[pbase + k0 + kk];
        const int orig = perm[pbase + k0 + kk] - pbase;  // the problem's original index
        for (int c = 0; c < PR_R; ++c) ws[c * PR_TILE + kk] = c < nr ? w[(size_t)orig + (size_t)(c0 + c) * ldw] : 0.0;
      }
      __syncthreads();
      if (!active) continue;
      for (int kk = 0; kk < nt; ++kk) {
        double dot = 0.0;
        for (int q = 0; q < d; ++q) dot = fma(t[q], xs[(size_t)kk * d + q], dot);
        const double d2 = fmax((tn + xcn[kk]) - 2.0 * dot, 0.0);
        const double kv = kspec_value(g_kspec, dot, d2, scale);
#pragma unroll
        for (int c = 0; c < PR_R; ++c) acc[c] = fma(kv, ws[c * PR_TILE + kk], acc[c]);
      }
    }
    if (active)
      for (int c = 0; c < nr; ++c) part[((size_t)blockIdx.y * nrhs + c0 + c) * M + i] = acc[c];
  }
}

// out[r][i] (ld ldo) = sum over chunks c in order of part[c][r][i]
__global__ void predict_reduce_kernel(const double* part, int M, int nrhs, int nchunk, double* out, int ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * nrhs) return;
  const int i = (int)(e % M), r = (int)(e / M);
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[((size_t)c * nrhs + r) * M + i];
  out[(size_t)i + (size_t)r * ldo] = s;
}

}  // namespace

size_t predict_scratch_doubles(int M, int N, int nrhs) {
  int chunk = 0, nchunk = 0;
  predict_chunks(M, N, chunk, nchunk);
  return (size_t)nchunk * nrhs * M;
}

void predict_chunks(int M, int N, int& chunk, int& nchunk) {
  // about 4 blocks per SM on 152 SMs, chunks of at least 1024 training points
  const int mblocks = (int)ceil_div((size_t)std::max(M, 1), PR_THREADS);
  const int want = std::max(1, (4 * 152 + mblocks - 1) / mblocks);
  const int most = (int)ceil_div((size_t)std::max(N, 1), 1024);
  nchunk = std::max(1, std::min(want, most));
  chunk = (int)ceil_div((size_t)N, (size_t)nchunk);
  chunk = (chunk + PR_TILE - 1) / PR_TILE * PR_TILE;
  nchunk = (int)ceil_div((size_t)N, (size_t)chunk);
}

void kernel_predict(const double* T, int M, const double* Xp, const double* xnorm, const int* perm, int pbase,
                    int N, int d, double scale, const double* w, int ldw, int nrhs, double* part, double* out,
                    int ldo, cudaStream_t st) {
  if (M <= 0 || nrhs <= 0) return;
  int chunk = 0, nchunk = 0;
  predict_chunks(M, N, chunk, nchunk);
  const size_t smem = sizeof(double) * ((size_t)PR_TILE * d + PR_TILE + (size_t)PR_R * PR_TILE);
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(predict_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope _ps(PK_PREDICT, st);
  prof().flops[PK_PREDICT] += (double)M * N * (2.0 * d + 2.0 * nrhs);
  dim3 grid(ceil_div((size_t)M, PR_THREADS), (unsigned)nchunk);
  predict_partial_kernel<<<grid, PR_THREADS, smem, st>>>(T, M, Xp, xnorm, perm, pbase, N, d, scale, w, ldw, nrhs,
                                                          chunk, part);
  IA_LAUNCH_CHECK();
  const int64_t tot = (int64_t)M * nrhs;
  predict_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, M, nrhs, nchunk, out, ldo);
  IA_LAUNCH_CHECK();
}

}  // namespace iaskit
