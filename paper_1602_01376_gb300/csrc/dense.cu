// Batched dense kernels of the factorization, templated on the scalar type T
// (double: plain FP64 path; float: mixed-precision form).
//
//  * kernel_blocks   Gaussian kernel blocks from coordinates (Sec. I, eq. gaussian):
//                    sampled blocks K(samples, columns), leaf blocks lambda I + K_aa
//                    and the U blocks K_{l r~}, K_{r l~} (eq. uv-askit).
//  * cpqr_id         column-pivoted Householder QR of a sampled block; the
//                    interpolative decomposition T = R11^{-1} R12 (Sec. II-B; GEQP3 and
//                    GELS in Sec. II-C) is then trsm_upper_batched.  Trailing column norms are recomputed from the
//                    updated block at every step, accumulated in FP64; pivot ties go to
//                    the lowest column.
//  * getrf / getrs   LU with partial pivoting (ties to the lowest row) and the
//                    corresponding solve (GETRF / GETRS of Alg. "Factorize"/"Solve"),
//                    both blocked by 32 so that most of the work is a register-tiled
//                    product.
//  * gemm_grouped    C <- alpha A B + beta C over many independent small problems, the
//                    products of eqs. innerid and blocksmw.
// In FP64 these kernels are bound by the FP64 pipe (2 FMA per clock per SM on this
// part); they keep it fed with many independent blocks.
#include <cfloat>
#include <type_traits>
#include <climits>

#include <cooperative_groups.h>

#include "kernels.cuh"
#include "pair.cuh"
#include "tc.cuh"

IA_KERNEL_SPEC_TU(kspec_set_dense)

namespace iaskit {

namespace {

template <typename T>
__device__ __forceinline__ T kexp(T x);
template <>
__device__ __forceinline__ double kexp<double>(double x) { return exp(x); }
template <>
__device__ __forceinline__ float kexp<float>(float x) { return expf(x); }

// ------------------------------------------------------------ kernel blocks
// One block per 64 x 64 tile of one descriptor.  The tile's row and column points are
// staged in shared memory (transposed, [coordinate][point]) and every thread forms a
// 4 x 4 register tile of entries.  FP64 blocks use the Gram form
// |x|^2 + |y|^2 - 2 x.y with the squared norms precomputed (one FMA per coordinate;
// the cancellation error, about 2^-52 (|x|^2 + |y|^2), moves a kernel value by a
// relative 2^-52 (|x|^2 + |y|^2) / (2 h^2)); FP32 blocks keep the difference form,
// whose error is relative to the distance itself.
constexpr int KB_T = 64;        // tile edge
constexpr int KB_THREADS = 256; // 16 x 16 threads, 4 x 4 entries each
template <typename T>
__global__ void __launch_bounds__(KB_THREADS) kernel_blocks_kernel(const double* Xp, const double* xn, int d,
                                                                   const KDescT<T>* descs) {
  extern __shared__ __align__(16) unsigned char kb_sh[];
  T* Xr = reinterpret_cast<T*>(kb_sh);         // [d][KB_T]
  T* Xc = Xr + (size_t)d * KB_T;               // [d][KB_T]
  __shared__ double nr_s[KB_T], nc_s[KB_T];
  __shared__ int ri_s[KB_T], ci_s[KB_T];
  const KDescT<T> D = descs[blockIdx.y];
  const bool poly = g_kspec.poly != 0;
  const int tr = (D.nrows + KB_T - 1) / KB_T, tcn = (D.ncols + KB_T - 1) / KB_T;
  const int tid = threadIdx.x;
  for (int tile = blockIdx.x; tile < tr * tcn; tile += gridDim.x) {
  const int i0 = (tile % tr) * KB_T, j0 = (tile / tr) * KB_T;
  __syncthreads();  // the previous tile's readers are done with the staging buffers
  if (tid < KB_T) {
    const int i = min(i0 + tid, D.nrows - 1);
    const int r = D.rows ? D.rows[i] : D.row0 + i;
    ri_s[tid] = r;
    nr_s[tid] = xn ? xn[r] : 0.0;
  } else if (tid < 2 * KB_T) {
    const int j = min(j0 + tid - KB_T, D.ncols - 1);
    const int c = D.colsA ? (j < D.nA ? D.colsA[j] : D.colsB[j - D.nA]) : D.col0 + j;
    ci_s[tid - KB_T] = c;
    nc_s[tid - KB_T] = xn ? xn[c] : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < KB_T * d; e += KB_THREADS) {
    const int p = e / d, k = e % d;
    Xr[(size_t)k * KB_T + p] = (T)Xp[(size_t)ri_s[p] * d + k];
    Xc[(size_t)k * KB_T + p] = (T)Xp[(size_t)ci_s[p] * d + k];
  }
  __syncthreads();
  const int tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  for (int k = 0; k < d; ++k) {
    T xr[4], xc[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      xr[a] = Xr[(size_t)k * KB_T + tx + 16 * a];
      xc[a] = Xc[(size_t)k * KB_T + ty + 16 * a];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (std::is_same<T, double>::value || poly) {
          acc[a][b] = fma(xr[a], xc[b], acc[a][b]);  // the dot product (Gram form)
        } else {
          const T t = xr[a] - xc[b];
          acc[a][b] = fma(t, t, acc[a][b]);
        }
      }
  }
  const T scale = (T)D.scale;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int li = tx + 16 * a, lj = ty + 16 * b;
      const int i = i0 + li, j = j0 + lj;
      if (i >= D.nrows || j >= D.ncols) continue;
      T v;
      if (poly) {
        v = kspec_pow<T>(fma(acc[a][b], scale, (T)g_kspec.c), g_kspec.p);
      } else {
        T d2 = acc[a][b];
        if (std::is_same<T, double>::value) d2 = fmax((nr_s[li] + nc_s[lj]) - 2.0 * acc[a][b], 0.0);
        v = kexp<T>(d2 * scale);
      }
      if (ri_s[li] == ci_s[lj]) v += (T)D.diag;
      D.out[(size_t)i + (size_t)j * D.ld] = v;
    }
  }
}

// Kernel blocks on FP32 pairs (the operator blocks of the mixed form): coordinates
// as pairs (Xpair = split Xp), the squared distance in the difference form with every
// coordinate difference, square and partial sum kept as a pair (error relative to the
// distance itself, no cancellation), then exp as a pair (fp2::exp_neg) and the
// diagonal shift; the result is written as pairs (hi, lo).
__global__ void __launch_bounds__(KB_THREADS) kernel_blocks_pair_kernel(const float2* Xpair, int d,
                                                                        const KDescT<float2>* descs) {
  extern __shared__ __align__(16) unsigned char kb_sh[];
  float2* Xr = reinterpret_cast<float2*>(kb_sh);  // [d][KB_T]
  float2* Xc = Xr + (size_t)d * KB_T;              // [d][KB_T]
  __shared__ int ri_s[KB_T], ci_s[KB_T];
  const KDescT<float2> D = descs[blockIdx.y];
  const bool poly = g_kspec.poly != 0;
  const fp2::pair scale = fp2::from_double(D.scale), diag = fp2::from_double(D.diag);
  const int tr = (D.nrows + KB_T - 1) / KB_T, tcn = (D.ncols + KB_T - 1) / KB_T;
  const int tid = threadIdx.x;
  for (int tile = blockIdx.x; tile < tr * tcn; tile += gridDim.x) {
    const int i0 = (tile % tr) * KB_T, j0 = (tile / tr) * KB_T;
    __syncthreads();  // the previous tile's readers are done with the staging buffers
    if (tid < KB_T) {
      const int i = min(i0 + tid, D.nrows - 1);
      ri_s[tid] = D.rows ? D.rows[i] : D.row0 + i;
    } else if (tid < 2 * KB_T) {
      const int j = min(j0 + tid - KB_T, D.ncols - 1);
      ci_s[tid - KB_T] = D.colsA ? (j < D.nA ? D.colsA[j] : D.colsB[j - D.nA]) : D.col0 + j;
    }
    __syncthreads();
    for (int e = tid; e < KB_T * d; e += KB_THREADS) {
      const int p = e / d, k = e % d;
      Xr[(size_t)k * KB_T + p] = Xpair[(size_t)ri_s[p] * d + k];
      Xc[(size_t)k * KB_T + p] = Xpair[(size_t)ci_s[p] * d + k];
    }
    __syncthreads();
    const int tx = tid % 16, ty = tid / 16;
    float sh[4][4], sl[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) sh[a][b] = sl[a][b] = 0.0f;
    for (int k = 0; k < d; ++k) {
      float2 xr[4], xc[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        xr[a] = Xr[(size_t)k * KB_T + tx + 16 * a];
        xc[a] = Xc[(size_t)k * KB_T + ty + 16 * a];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (poly) {  // the dot product as a pair: (sh, sl) += x_r x_c
            const fp2::pair pr = fp2::mul(fp2::pair{xr[a].x, xr[a].y}, fp2::pair{xc[b].x, xc[b].y});
            const fp2::pair s2 = fp2::add(fp2::pair{sh[a][b], sl[a][b]}, pr);
            sh[a][b] = s2.h;
            sl[a][b] = s2.l;
            continue;
          }
          // t = x_r - x_c as th + tl, then (sh, sl) += t^2.  th is often the exact
          // difference of the high parts and tl (the low parts' difference) is then
          // not small against it: t^2 = th^2 + 2 th tl + tl^2 keeps all three terms.
          float th, te;
          fp2::two_sum(xr[a].x, -xc[b].x, th, te);
          const float tl = __fadd_rn(te, __fsub_rn(xr[a].y, xc[b].y));
          const float p = __fmul_rn(th, th);
          float q = fmaf(th, th, -p);
          q = fmaf(tl, tl, q);
          q = fmaf(__fadd_rn(th, th), tl, q);
          float s2, e2;
          fp2::two_sum(sh[a][b], p, s2, e2);
          sl[a][b] = __fadd_rn(sl[a][b], __fadd_rn(e2, q));
          sh[a][b] = s2;
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int li = tx + 16 * a, lj = ty + 16 * b;
        const int i = i0 + li, j = j0 + lj;
        if (i >= D.nrows || j >= D.ncols) continue;
        const fp2::pair d2 = fp2::renorm(sh[a][b], sl[a][b]);
        fp2::pair v;
        if (poly) {
          const fp2::pair t = fp2::add(fp2::mul(d2, scale), fp2::from_double(g_kspec.c));
          v = t;
          for (int e = 1; e < g_kspec.p; ++e) v = fp2::mul(v, t);
        } else {
          v = fp2::exp_neg(fp2::mul(d2, scale));
        }
        if (ri_s[li] == ci_s[lj]) v = fp2::add(v, diag);
        D.out[(size_t)i + (size_t)j * D.ld] = make_float2(v.h, v.l);
      }
  }
}

__global__ void row_norms_kernel(const double* Xp, int N, int d, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = 0.0;
  for (int k = 0; k < d; ++k) s = fma(Xp[(size_t)i * d + k], Xp[(size_t)i * d + k], s);
  out[i] = s;
}

// ----------------------------------------------------------------- CPQR / ID
constexpr int QR_THREADS = 512;
constexpr int QR_WARPS = QR_THREADS / 32;
constexpr int QR_RPL = 16;  // rows per lane held in registers (columns of up to 512 rows)

// (v, idx) over the block, in the value's own type: larger value wins, equal values go
// to the lower index.  FP32 magnitudes compare exactly as their FP64 images would (the
// conversion is exact and monotone), without FP64 instructions.
template <typename V>
__device__ __forceinline__ void warp_argmax_t(V& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const V v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    if (v2 > v || (v2 == v && i2 < i)) {
      v = v2;
      i = i2;
    }
  }
}
template <typename V>
__device__ void block_argmax_t(V& v, int& idx, V* rv, int* ri) {
  warp_argmax_t(v, idx);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    rv[warp] = v;
    ri[warp] = idx;
  }
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? rv[lane] : (V)-1;
    idx = lane < (int)(blockDim.x >> 5) ? ri[lane] : INT_MAX;
    warp_argmax_t(v, idx);
    if (lane == 0) {
      rv[0] = v;
      ri[0] = idx;
    }
  }
  __syncthreads();
  v = rv[0];
  idx = ri[0];
}

__device__ void block_argmax(double& v, int& idx, double* rv, int* ri) {
  warp_argmax(v, idx);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    rv[warp] = v;
    ri[warp] = idx;
  }
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? rv[lane] : -1.0;
    idx = lane < (int)(blockDim.x >> 5) ? ri[lane] : INT_MAX;
    warp_argmax(v, idx);
    if (lane == 0) {
      rv[0] = v;
      ri[0] = idx;
    }
  }
  __syncthreads();
  v = rv[0];
  idx = ri[0];
}

__device__ double block_sum(double v, double* rv) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) rv[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < QR_WARPS ? rv[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) rv[0] = v;
  }
  __syncthreads();
  v = rv[0];
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One block per node, FP64 (the FP32 form is cpqr_f32_kernel / cpqr_cluster_kernel).
// Dynamic shared memory: norms (ncols doubles), v (nrows T), piv (ncols ints).
template <typename T>
__global__ void __launch_bounds__(QR_THREADS) cpqr_kernel(const CpqrDescT<T>* descs, int s_max,
                                                          double tol) {
  extern __shared__ double shq[];
  __shared__ double rv[QR_WARPS];
  __shared__ int ri[QR_WARPS];
  const CpqrDescT<T> D = descs[blockIdx.x];
  T* A = D.A;
  const int ld = D.ld, nr = D.nrows, nc = D.ncols;
  double* norms = shq;
  T* v = reinterpret_cast<T*>(shq + nc);
  int* piv = reinterpret_cast<int*>(shq + nc + nr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < nc; j += QR_WARPS) {
    T part = 0;
    for (int i = lane; i < nr; i += 32) {
      T a = A[(size_t)i + (size_t)j * ld];
      part = fma(a, a, part);
    }
    double s = warp_sum((double)part);
    if (lane == 0) {
      norms[j] = s;
      piv[j] = j;
    }
  }
  __syncthreads();
  const int cap = min(s_max, min(nc, nr));
  double nu0 = 0.0;
  int s = 0;
  for (int k = 0; k < cap; ++k) {
    double best = -1.0;
    int bi = INT_MAX;
    for (int j = k + threadIdx.x; j < nc; j += QR_THREADS) argmax_merge(best, bi, norms[j], j);
    block_argmax(best, bi, rv, ri);
    const double nu = sqrt(best);
    if (k == 0) {
      nu0 = nu;
    } else if (nu == 0.0 || (tol > 0.0 && nu <= tol * nu0)) {
      break;
    }
    const int p = bi;
    if (p != k) {
      for (int i = threadIdx.x; i < nr; i += QR_THREADS) {
        T t = A[(size_t)i + (size_t)k * ld];
        A[(size_t)i + (size_t)k * ld] = A[(size_t)i + (size_t)p * ld];
        A[(size_t)i + (size_t)p * ld] = t;
      }
      if (threadIdx.x == 0) {
        double tn = norms[k];
        norms[k] = norms[p];
        norms[p] = tn;
        int tp = piv[k];
        piv[k] = piv[p];
        piv[p] = tp;
      }
    }
    __syncthreads();
    for (int i = k + threadIdx.x; i < nr; i += QR_THREADS) v[i - k] = A[(size_t)i + (size_t)k * ld];
    __syncthreads();
    const double x0 = (double)v[0];
    const double alpha = x0 >= 0.0 ? -nu : nu;
    double part = 0.0;
    for (int i = 1 + threadIdx.x; i < nr - k; i += QR_THREADS) {
      double vi = (double)v[i];
      part = fma(vi, vi, part);
    }
    const double v0 = x0 - alpha;
    const double vv = block_sum(part, rv) + v0 * v0;
    if (threadIdx.x == 0) v[0] = (T)v0;
    __syncthreads();
    const T beta = vv > 0.0 ? (T)(2.0 / vv) : (T)0;
    {
    for (int j = k + 1 + warp; j < nc; j += QR_WARPS) {
      T* col = A + (size_t)j * ld;
      T dot = 0;
      {
        for (int i = k + lane; i < nr; i += 32) dot = fma(v[i - k], col[i], dot);
        dot = warp_sum_t<T>(dot);
        const T f = beta * dot;
        T part = 0;
        for (int i = k + lane; i < nr; i += 32) {
          T a = col[i] - f * v[i - k];
          col[i] = a;
          if (i > k) part = fma(a, a, part);
        }
        const double nrm = warp_sum((double)part);
        if (lane == 0) norms[j] = nrm;
      }
    }
    }
    for (int i = k + threadIdx.x; i < nr; i += QR_THREADS)
      A[(size_t)i + (size_t)k * ld] = (i == k) ? (T)alpha : (T)0;
    s = k + 1;
    __syncthreads();
  }
  // T = R11^{-1} R12 follows in trsm_upper_batched (blocked, many blocks per node)
  for (int j = threadIdx.x; j < nc; j += QR_THREADS) D.piv[j] = piv[j];
  if (threadIdx.x == 0) *D.rank = s;
}

// ------------------------------------------------ FP32 CPQR
// Column norms of the FP32 ID are combined across lanes as FP32 pairs (hi + lo, about
// 48 significant bits, fp2 arithmetic) rather than in FP64: this part issues two FP64
// FMAs per clock per SM, and FP64 butterflies over every column made up most of a
// step.  Pairs are kept normalized and compared lexicographically (hi, then lo);
// nu = |column|, alpha and beta are formed once per step by one thread in FP64.
__device__ __forceinline__ bool pair_gt(float2 a, float2 b) { return a.x > b.x || (a.x == b.x && a.y > b.y); }
__device__ __forceinline__ bool pair_eq(float2 a, float2 b) { return a.x == b.x && a.y == b.y; }
// (h, l) <- sum over the warp; every lane gets the same pair (two-sum is exact, so the
// butterfly is symmetric).
__device__ __forceinline__ void pair_warp_sum(float& h, float& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
    float sm, e;
    fp2::two_sum(h, h2, sm, e);
    e = __fadd_rn(e, __fadd_rn(l, l2));
    fp2::fast_two_sum(sm, e, h, l);
  }
}
// Sum of 32 FP32 values x[0], x[stride], ... in order, as a pair (two-sum chain).
__device__ __forceinline__ float2 pair_sum32(const float* x, int stride) {
  float h = 0.0f, l = 0.0f;
#pragma unroll 8
  for (int i = 0; i < 32; ++i) {
    float sm, e;
    fp2::two_sum(h, x[i * stride], sm, e);
    h = sm;
    l = __fadd_rn(l, e);
  }
  float rh, rl;
  fp2::fast_two_sum(h, l, rh, rl);
  return make_float2(rh, rl);
}
// Per warp: the lane partials of up to QP_SLOTS columns (slot-major, padded rows), so
// that lane s combines slot s's 32 partials in one sequential pair sum instead of a
// butterfly per column.
constexpr int QP_SLOTS = 64, QP_LD = 33;

// (best, idx) over the warp: larger pair wins, equal pairs go to the lower index.
__device__ __forceinline__ void pair_warp_argmax(float2& v, int& idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float2 v2;
    v2.x = __shfl_xor_sync(0xffffffffu, v.x, o);
    v2.y = __shfl_xor_sync(0xffffffffu, v.y, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (pair_gt(v2, v) || (pair_eq(v2, v) && i2 < idx)) {
      v = v2;
      idx = i2;
    }
  }
}
// Householder step from the pivot column: x0 its entry on the diagonal, vvp the pair sum
// of the squares below it, nu its norm: alpha = -sign(x0) nu, v0 = x0 - alpha,
// beta = 2 / (v0^2 + vvp) (FP64, one thread).
__device__ __forceinline__ void householder_f32(float x0f, float2 vvp, double nu, float& alpha, float& v0f,
                                                float& beta) {
  const double x0 = (double)x0f;
  const double a = x0 >= 0.0 ? -nu : nu;
  const double v0 = x0 - a;
  const double vv = ((double)vvp.x + (double)vvp.y) + v0 * v0;
  alpha = (float)a;
  v0f = (float)v0;
  beta = vv > 0.0 ? (float)(2.0 / vv) : 0.0f;
}

// One block per node, A in global memory.  Dynamic shared memory: norms (ncols pairs),
// v (nrows floats), piv (ncols ints), laid out like cpqr_kernel's.
__global__ void __launch_bounds__(QR_THREADS) cpqr_f32_kernel(const CpqrDescT<float>* descs, int s_max,
                                                              double tol) {
  extern __shared__ double shq[];
  __shared__ float2 rvp[QR_WARPS];
  __shared__ int ri[QR_WARPS];
  __shared__ double nu_s;
  __shared__ int stop_s, p_s;
  __shared__ float alpha_s, beta_s;
  const CpqrDescT<float> D = descs[blockIdx.x];
  float* A = D.A;
  const int ld = D.ld, nr = D.nrows, nc = D.ncols;
  float2* norms = reinterpret_cast<float2*>(shq);
  float* v = reinterpret_cast<float*>(shq + nc);
  int* piv = reinterpret_cast<int*>(shq + nc + nr);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // per-warp lane partials of the column norms (after piv, 16-byte aligned)
  float* psum = reinterpret_cast<float*>(shq + nc + nr + (nc + 1) / 2 + 1) + (size_t)warp * QP_SLOTS * QP_LD;
  for (int j = warp; j < nc; j += QR_WARPS) {
    float part = 0.0f;
    for (int i = lane; i < nr; i += 32) {
      const float a = A[(size_t)i + (size_t)j * ld];
      part = fmaf(a, a, part);
    }
    float h = part, l = 0.0f;
    pair_warp_sum(h, l);
    if (lane == 0) {
      norms[j] = make_float2(h, l);
      piv[j] = j;
    }
  }
  __syncthreads();
  const int cap = min(s_max, min(nc, nr));
  double nu0 = 0.0;  // thread 0
  int s = 0;
  for (int k = 0; k < cap; ++k) {
    float2 best = make_float2(-1.0f, 0.0f);
    int bi = INT_MAX;
    for (int j = k + tid; j < nc; j += QR_THREADS) {
      const float2 nv = norms[j];
      if (pair_gt(nv, best) || (pair_eq(nv, best) && j < bi)) {
        best = nv;
        bi = j;
      }
    }
    pair_warp_argmax(best, bi);
    if (lane == 0) {
      rvp[warp] = best;
      ri[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
      best = lane < QR_WARPS ? rvp[lane] : make_float2(-1.0f, 0.0f);
      bi = lane < QR_WARPS ? ri[lane] : INT_MAX;
      pair_warp_argmax(best, bi);
      if (lane == 0) {
        const double nu = sqrt(fmax((double)best.x + (double)best.y, 0.0));
        int stop = 0;
        if (k == 0) nu0 = nu;
        else stop = (nu == 0.0 || (tol > 0.0 && nu <= tol * nu0)) ? 1 : 0;
        nu_s = nu;
        stop_s = stop;
        p_s = bi;
      }
    }
    __syncthreads();
    if (stop_s) break;
    const int p = p_s;
    if (p != k) {
      for (int i = tid; i < nr; i += QR_THREADS) {
        const float t = A[(size_t)i + (size_t)k * ld];
        A[(size_t)i + (size_t)k * ld] = A[(size_t)i + (size_t)p * ld];
        A[(size_t)i + (size_t)p * ld] = t;
      }
      if (tid == 0) {
        const float2 tn = norms[k];
        norms[k] = norms[p];
        norms[p] = tn;
        const int tp = piv[k];
        piv[k] = piv[p];
        piv[p] = tp;
      }
    }
    __syncthreads();
    float ph = 0.0f, pl = 0.0f;  // sum of v_i^2 below the diagonal, as a pair
    for (int i = k + tid; i < nr; i += QR_THREADS) {
      const float vi = A[(size_t)i + (size_t)k * ld];
      v[i - k] = vi;
      if (i > k) {
        const float sq = __fmul_rn(vi, vi);
        const float se = fmaf(vi, vi, -sq);
        float sm, e;
        fp2::two_sum(ph, sq, sm, e);
        fp2::fast_two_sum(sm, __fadd_rn(pl, __fadd_rn(e, se)), ph, pl);
      }
    }
    pair_warp_sum(ph, pl);
    if (lane == 0) rvp[warp] = make_float2(ph, pl);
    __syncthreads();
    if (warp == 0) {
      ph = lane < QR_WARPS ? rvp[lane].x : 0.0f;
      pl = lane < QR_WARPS ? rvp[lane].y : 0.0f;
      pair_warp_sum(ph, pl);
      if (lane == 0) {
        float al, v0, be;
        householder_f32(v[0], make_float2(ph, pl), nu_s, al, v0, be);
        alpha_s = al;
        beta_s = be;
        v[0] = v0;
      }
    }
    __syncthreads();
    const float beta = beta_s;
    const int tcount = (nr - k + 31) / 32;  // rows per lane of the trailing column
    if (tcount <= QR_RPL) {
      // a warp keeps CW columns in registers between the dot products and the updates,
      // so that their loads and reductions overlap
      constexpr int CW = 4;
      for (int j = k + 1 + CW * warp; j < nc; j += CW * QR_WARPS) {
        float* cp[CW];
        bool has[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          has[c] = j + c < nc;
          cp[c] = A + (size_t)(has[c] ? j + c : j) * ld;
        }
        float x[CW][QR_RPL];
#pragma unroll
        for (int t = 0; t < QR_RPL; ++t) {
          const int i = k + lane + 32 * t;
          const bool in = t < tcount && i < nr;
#pragma unroll
          for (int c = 0; c < CW; ++c) x[c][t] = in ? cp[c][i] : 0.0f;
        }
        float dt[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) dt[c] = 0.0f;
#pragma unroll
        for (int t = 0; t < QR_RPL; ++t) {
          const int i = k + lane + 32 * t;
          const float vi = (t < tcount && i < nr) ? v[i - k] : 0.0f;
#pragma unroll
          for (int c = 0; c < CW; ++c) dt[c] = fmaf(vi, x[c][t], dt[c]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int c = 0; c < CW; ++c) dt[c] += __shfl_xor_sync(0xffffffffu, dt[c], o);
        float pn[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) pn[c] = 0.0f;
#pragma unroll
        for (int t = 0; t < QR_RPL; ++t) {
          const int i = k + lane + 32 * t;
          if (t < tcount && i < nr) {
            const float vi = v[i - k];
#pragma unroll
            for (int c = 0; c < CW; ++c) {
              const float a = x[c][t] - (beta * dt[c]) * vi;
              if (has[c]) cp[c][i] = a;
              if (i > k) pn[c] = fmaf(a, a, pn[c]);
            }
          }
        }
        const int slot0 = ((j - (k + 1 + CW * warp)) / (CW * QR_WARPS)) * CW;
#pragma unroll
        for (int c = 0; c < CW; ++c) psum[(size_t)(slot0 + c) * QP_LD + lane] = pn[c];
      }
      // every column of this warp: its norm from the 32 lane partials, lane s for slot s
      __syncwarp();
      const int ncol_w = nc - (k + 1 + CW * warp);
      const int nslot = ncol_w > 0 ? ((ncol_w + CW * QR_WARPS - 1) / (CW * QR_WARPS)) * CW : 0;
      for (int sl = lane; sl < nslot; sl += 32) {
        const int col = k + 1 + CW * warp + (sl / CW) * (CW * QR_WARPS) + sl % CW;
        if (col < nc) norms[col] = pair_sum32(psum + (size_t)sl * QP_LD, 1);
      }
    } else {
      for (int j = k + 1 + warp; j < nc; j += QR_WARPS) {
        float* col = A + (size_t)j * ld;
        float dot = 0.0f;
        for (int i = k + lane; i < nr; i += 32) dot = fmaf(v[i - k], col[i], dot);
        dot = warp_sum_t<float>(dot);
        const float f = beta * dot;
        float part = 0.0f;
        for (int i = k + lane; i < nr; i += 32) {
          const float a = col[i] - f * v[i - k];
          col[i] = a;
          if (i > k) part = fmaf(a, a, part);
        }
        float l = 0.0f;
        pair_warp_sum(part, l);
        if (lane == 0) norms[j] = make_float2(part, l);
      }
    }
    const float alpha = alpha_s;
    for (int i = k + tid; i < nr; i += QR_THREADS) A[(size_t)i + (size_t)k * ld] = (i == k) ? alpha : 0.0f;
    s = k + 1;
    __syncthreads();
  }
  for (int j = tid; j < nc; j += QR_THREADS) D.piv[j] = piv[j];
  if (tid == 0) *D.rank = s;
}

// ------------------------------------------------ CPQR on a thread-block cluster
// The same column-pivoted Householder QR (FP32 values, FP64 column norms, ties to the
// lowest column) for one node spread over a cluster of CS blocks: block r keeps the
// physical columns [64 r, 64 r + 64) in registers (4 columns per warp, 16 rows per
// lane, up to 512 rows), so the trailing matrix is never re-read from memory.  Columns
// do not move; a logical <-> physical map (the same in every block) records the swaps.
// Each block publishes its best remaining column (norm, logical index and the column
// itself) in a double-buffered slot; one cluster barrier per step; then every block
// reads the CS candidates through distributed shared memory, takes the same pivot,
// copies the winning column, forms the same Householder vector and updates its own
// columns.  All blocks take the same decisions, so they pass the same barriers.
namespace cg = cooperative_groups;
constexpr int QC_COLS = 64, QC_THREADS = 512, QC_RPL = 16;
constexpr int QC_MAX_ROWS = 32 * QC_RPL;

// Shared state of one block of a cluster CPQR (see cpqr_cluster_kernel).
struct QcShared {
  float ccol[2][QC_MAX_ROWS];  // this block's candidate column, per step parity
  float2 cval[2];              // its squared norm as a pair (-1: none)
  int cidx[2];                 // its logical index
  float vloc[QC_MAX_ROWS];     // Householder vector of the step
  float2 norm_s[QC_COLS];      // squared norms of this block's columns (-1: pivoted or absent)
  int phys_of[QC_COLS * 8], log_of[QC_COLS * 8];
  double nu;
  float alpha, beta;
  int best_j, cand_q, stop;
  float psum[QC_THREADS / 32][4][32];  // per warp: lane partials of its 4 columns' norms
};

__global__ void __launch_bounds__(QC_THREADS, 1) cpqr_cluster_kernel(const CpqrDescT<float>* descs, int s_max,
                                                                     double tol) {
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const CpqrDescT<float> D = descs[blockIdx.x / CS];
  __shared__ QcShared S;
  float* vloc = S.vloc;
  float2* norm_s = S.norm_s;
  int* phys_of = S.phys_of;
  int* log_of = S.log_of;
  float* A = D.A;
  const int ld = D.ld, nr = D.nrows, nc = D.ncols;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int jw = rank * QC_COLS + warp * 4;  // physical column of (warp, c = 0)
  const float2 NONE = make_float2(-1.0f, 0.0f);
  float x[4][QC_RPL];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int t = 0; t < QC_RPL; ++t) {
      const int i = lane + 32 * t, j = jw + c;
      x[c][t] = (j < nc && i < nr) ? A[(size_t)i + (size_t)j * ld] : 0.0f;
    }
  for (int j = tid; j < nc; j += QC_THREADS) {
    phys_of[j] = j;
    log_of[j] = j;
  }
  {
    float h[4] = {0.0f, 0.0f, 0.0f, 0.0f}, l[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int t = 0; t < QC_RPL; ++t)
#pragma unroll
      for (int c = 0; c < 4; ++c) h[c] = fmaf(x[c][t], x[c][t], h[c]);
#pragma unroll
    for (int c = 0; c < 4; ++c) pair_warp_sum(h[c], l[c]);
    if (lane == 0)
#pragma unroll
      for (int c = 0; c < 4; ++c) norm_s[warp * 4 + c] = jw + c < nc ? make_float2(h[c], l[c]) : NONE;
  }
  const int cap = min(s_max, min(nc, nr));
  double nu0 = 0.0;  // thread 0
  int s = 0;
  for (int k = 0; k < cap; ++k) {
    const int b = k & 1;
    // publish this block's best remaining column (norm, logical index, values) in slot b
    __syncthreads();  // norms and maps are current
    if (warp == 0) {
      float2 bv = NONE;
      int bj = INT_MAX, bq = -1;
      for (int q = lane; q < QC_COLS; q += 32) {
        const int j = rank * QC_COLS + q;
        if (j < nc && norm_s[q].x >= 0.0f) {
          const int lj = log_of[j];
          if (pair_gt(norm_s[q], bv) || (pair_eq(norm_s[q], bv) && lj < bj)) {
            bv = norm_s[q];
            bj = lj;
            bq = q;
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        float2 v2;
        v2.x = __shfl_xor_sync(0xffffffffu, bv.x, o);
        v2.y = __shfl_xor_sync(0xffffffffu, bv.y, o);
        const int j2 = __shfl_xor_sync(0xffffffffu, bj, o), q2 = __shfl_xor_sync(0xffffffffu, bq, o);
        if (pair_gt(v2, bv) || (pair_eq(v2, bv) && j2 < bj)) {
          bv = v2;
          bj = j2;
          bq = q2;
        }
      }
      if (lane == 0) {
        S.cval[b] = bv;
        S.cidx[b] = bj;
        S.cand_q = bq;
      }
    }
    __syncthreads();
    {
      const int q = S.cand_q;
      if (q >= 0 && warp == q / 4) {
        const int qc = q % 4;
#pragma unroll
        for (int t = 0; t < QC_RPL; ++t) {  // selects, not an indexed register array
          const float v = qc == 0 ? x[0][t] : qc == 1 ? x[1][t] : qc == 2 ? x[2][t] : x[3][t];
          const int i = lane + 32 * t;
          if (i < nr) S.ccol[b][i] = v;
        }
      }
    }
    cl.sync();  // every block's candidate for step k is published
    if (warp == 0) {
      float2 bv = NONE;
      int bj = INT_MAX;
      if (lane < CS) {
        bv = *cl.map_shared_rank(&S.cval[b], lane);
        bj = *cl.map_shared_rank(&S.cidx[b], lane);
      }
      pair_warp_argmax(bv, bj);
      if (lane == 0) {
        const double nu = sqrt(fmax((double)bv.x + (double)bv.y, 0.0));
        int stop = bj == INT_MAX ? 1 : 0;  // no column left (not reached: cap <= nc)
        if (k == 0) nu0 = nu;
        else if (nu == 0.0 || (tol > 0.0 && nu <= tol * nu0)) stop = 1;
        S.nu = nu;
        S.best_j = bj;
        S.stop = stop;
      }
    }
    __syncthreads();
    if (S.stop) break;  // every block takes the same decision
    const int p = S.best_j;
    const int P = phys_of[p], owner = P / QC_COLS;
    {
      const float* rc = cl.map_shared_rank(&S.ccol[b][0], owner);
      for (int i = k + tid; i < nr; i += QC_THREADS) vloc[i] = rc[i];
    }
    __syncthreads();
    if (tid == 0 && p != k) {
      const int Pk = phys_of[k];
      phys_of[k] = P;
      phys_of[p] = Pk;
      log_of[P] = k;
      log_of[Pk] = p;
    }
    if (warp == 0) {  // v = (x_k - alpha, x_{k+1}, ...), the same in every block
      float ph = 0.0f, pl = 0.0f;
      for (int i = k + 1 + lane; i < nr; i += 32) {
        const float vi = vloc[i];
        const float sq = __fmul_rn(vi, vi);
        const float se = fmaf(vi, vi, -sq);
        float sm, e;
        fp2::two_sum(ph, sq, sm, e);
        fp2::fast_two_sum(sm, __fadd_rn(pl, __fadd_rn(e, se)), ph, pl);
      }
      pair_warp_sum(ph, pl);
      if (lane == 0) {
        float al, v0, be;
        householder_f32(vloc[k], make_float2(ph, pl), S.nu, al, v0, be);
        S.alpha = al;
        S.beta = be;
        vloc[k] = v0;
      }
    }
    __syncthreads();
    const float beta = S.beta;
    // the pivot column becomes (R entries above, alpha, zeros below)
    if (rank == owner && warp == (P % QC_COLS) / 4) {
      const int pc = P % 4;
      const float al = S.alpha;
#pragma unroll
      for (int c = 0; c < 4; ++c)  // selects on every column: no indexed register array
#pragma unroll
        for (int t = 0; t < QC_RPL; ++t) {
          const int i = lane + 32 * t;
          x[c][t] = (c != pc || i < k) ? x[c][t] : (i == k ? al : 0.0f);
        }
      if (lane == 0) norm_s[P % QC_COLS] = NONE;
    }
    __syncwarp();
    // update this block's remaining columns and their norms over rows > k
    bool live[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) live[c] = jw + c < nc && norm_s[warp * 4 + c].x >= 0.0f;
    if (live[0] || live[1] || live[2] || live[3]) {
      float dt[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int t = 0; t < QC_RPL; ++t) {
        const int i = lane + 32 * t;
        const float vi = (i >= k && i < nr) ? vloc[i] : 0.0f;
#pragma unroll
        for (int c = 0; c < 4; ++c) dt[c] = fmaf(vi, x[c][t], dt[c]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 4; ++c) dt[c] += __shfl_xor_sync(0xffffffffu, dt[c], o);
      float pn[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int t = 0; t < QC_RPL; ++t) {
        const int i = lane + 32 * t;
        if (i >= k && i < nr) {
          const float vi = vloc[i];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float a = x[c][t] - (beta * dt[c]) * vi;
            x[c][t] = live[c] ? a : x[c][t];
            if (i > k) pn[c] = fmaf(a, a, pn[c]);
          }
        }
      }
      // the norms from the 32 lane partials in lane order (as in cpqr_f32_kernel)
#pragma unroll
      for (int c = 0; c < 4; ++c) S.psum[warp][c][lane] = pn[c];
      __syncwarp();
      if (lane < 4 && live[lane]) norm_s[warp * 4 + lane] = pair_sum32(&S.psum[warp][lane][0], 1);
    }
    s = k + 1;
  }
  cl.sync();  // no block reads another's shared memory after this point
  // columns go to their logical positions (every block loaded its columns before)
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int j = jw + c;
    if (j >= nc) continue;
    const int L = log_of[j];
#pragma unroll
    for (int t = 0; t < QC_RPL; ++t) {
      const int i = lane + 32 * t;
      if (i < nr) A[(size_t)i + (size_t)L * ld] = x[c][t];
    }
  }
  if (rank == 0) {
    for (int j = tid; j < nc; j += QC_THREADS) D.piv[j] = phys_of[j];
    if (tid == 0) *D.rank = s;
  }
}

// ------------------------------------------------ FP32 GEMM on the tensor cores
// C = alpha A B + beta C for one 128 x 128 tile of one descriptor per block.  The K
// dimension is walked in chunks of 32: each thread holds the next chunk's values of A
// and B in registers (loaded while the tensor core works on the current chunk), then
// splits them into TF32 hi/lo pairs and stores them K-major into shared memory, and one
// thread issues 3 tcgen05 MMAs per 8 values of K (lo.hi, hi.lo, hi.hi) into a 128 x 128
// FP32 accumulator in TMEM.  One staging buffer per block (64 KB), three blocks per SM,
// so one block's staging overlaps the others' MMAs.  The epilogue reads the tile back
// with tcgen05.ld.  Waits are bounded; a wait that gives up stops the block's work and
// leaves its tile unwritten.
constexpr int GT_M = 128, GT_N = 128, GT_K = 32, GT_THREADS = 256;
constexpr int GT_UNITS = GT_M * GT_K / 4 / GT_THREADS;  // 16-byte units per thread per operand
constexpr long GT_WAIT = 1L << 22;
static_assert(GT_M == GT_N, "A and B tiles share the staging layout");

// Unit u = (row group rg, K group kg, row rr) holds the 4 consecutive K values of one
// row: 16 contiguous bytes of the K-major layout (word offset 4 u), so a quarter warp
// stores 128 contiguous bytes and 8 lanes read 8 consecutive rows of a column of A.
struct GtFrag {
  float a[GT_UNITS][4], b[GT_UNITS][4];
};
__device__ __forceinline__ void gt_load(const GemmDescT<float>& D, int m0, int n0, int k0, GtFrag& f) {
  const float* A = D.A + (size_t)m0 + (size_t)k0 * D.lda;  // A: M x K column-major
  const float* B = D.B + (size_t)k0 + (size_t)n0 * D.ldb;  // B: K x N column-major
  const int ra = D.M - m0, rb = D.N - n0, kk = D.K - k0;
#pragma unroll
  for (int i = 0; i < GT_UNITS; ++i) {
    const int u = threadIdx.x + i * GT_THREADS;
    const int r = (u / (8 * (GT_K / 4))) * 8 + (u & 7), k = ((u >> 3) & (GT_K / 4 - 1)) * 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      f.a[i][j] = (r < ra && k + j < kk) ? A[(size_t)r + (size_t)(k + j) * D.lda] : 0.0f;
      f.b[i][j] = (r < rb && k + j < kk) ? B[(size_t)(k + j) + (size_t)r * D.ldb] : 0.0f;
    }
  }
}
__device__ __forceinline__ void gt_split_store(const float (&v)[4], uint4* hi, uint4* lo) {
  uint4 h, l;
  h.x = tc::to_tf32(v[0]);
  h.y = tc::to_tf32(v[1]);
  h.z = tc::to_tf32(v[2]);
  h.w = tc::to_tf32(v[3]);
  l.x = tc::to_tf32(v[0] - __uint_as_float(h.x));
  l.y = tc::to_tf32(v[1] - __uint_as_float(h.y));
  l.z = tc::to_tf32(v[2] - __uint_as_float(h.z));
  l.w = tc::to_tf32(v[3] - __uint_as_float(h.w));
  *hi = h;
  *lo = l;
}
__device__ __forceinline__ void gt_store(const GtFrag& f, uint32_t* Ah, uint32_t* Al, uint32_t* Bh,
                                         uint32_t* Bl) {
#pragma unroll
  for (int i = 0; i < GT_UNITS; ++i) {
    const int u = threadIdx.x + i * GT_THREADS;
    gt_split_store(f.a[i], reinterpret_cast<uint4*>(Ah) + u, reinterpret_cast<uint4*>(Al) + u);
    gt_split_store(f.b[i], reinterpret_cast<uint4*>(Bh) + u, reinterpret_cast<uint4*>(Bl) + u);
  }
}

__global__ void __launch_bounds__(GT_THREADS, 3) gemm_tc_kernel(const GemmDescT<float>* descs,
                                                                const GemmTile* tiles, int* status) {
  extern __shared__ __align__(1024) unsigned char gt_sh[];
  constexpr int OPW = GT_M * GT_K;  // words of one operand array
  uint32_t* Ah = reinterpret_cast<uint32_t*>(gt_sh);
  uint32_t* Al = Ah + OPW;
  uint32_t* Bh = Al + OPW;
  uint32_t* Bl = Bh + OPW;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Bl + OPW);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  __shared__ int abort_s;
  const GemmTile Tl = tiles[blockIdx.x];
  const GemmDescT<float> D = descs[Tl.desc];
  const int m0 = Tl.tm * GT_M, n0 = Tl.tn * GT_N;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nk = (D.K + GT_K - 1) / GT_K;
  if (warp == 0) tc::tmem_alloc(tslot, GT_N);
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    abort_s = 0;
  }
  GtFrag f;
  if (nk > 0) gt_load(D, m0, n0, 0, f);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = tc::idesc_tf32(GT_M, GT_N);
  constexpr uint32_t SBO = (GT_K / 4) * 128;
  const uint32_t sah = tc::smem_addr(Ah), sal = tc::smem_addr(Al), sbh = tc::smem_addr(Bh),
                 sbl = tc::smem_addr(Bl);
  int inflight = -1;  // chunk whose MMAs have not reported completion
  for (int kc = 0; kc < nk; ++kc) {
    gt_store(f, Ah, Al, Bh, Bl);  // the MMAs of chunk kc - 1 have completed
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < GT_K / 8; ++ks) {
        const uint32_t ko = (uint32_t)ks * 256;
        const uint64_t dah = tc::smem_desc(sah + ko, 128, SBO), dal = tc::smem_desc(sal + ko, 128, SBO);
        const uint64_t dbh = tc::smem_desc(sbh + ko, 128, SBO), dbl = tc::smem_desc(sbl + ko, 128, SBO);
        tc::mma_tf32(tmem, dal, dbh, idesc, kc > 0 || ks > 0);
        tc::mma_tf32(tmem, dah, dbl, idesc, true);
        tc::mma_tf32(tmem, dah, dbh, idesc, true);
      }
      tc::mma_commit(mbar);
    }
    inflight = kc;
    if (kc + 1 < nk) gt_load(D, m0, n0, (kc + 1) * GT_K, f);  // in flight during the MMAs
    if (warp == 0) {
      if (!tc::mbar_wait(mbar, (uint32_t)(kc & 1), GT_WAIT) && lane == 0) {
        atomicOr(status, DEV_TIMEOUT);
        abort_s = 1;
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (abort_s) break;
    inflight = -1;
  }
  if (abort_s) {
    // give the MMAs that did not report completion one more bounded wait before the
    // block releases its TMEM and shared memory
    if (warp == 0 && inflight >= 0) tc::mbar_wait(mbar, (uint32_t)(inflight & 1), GT_WAIT);
  } else {
    // warp w: TMEM lanes 32 (w % 4) .., columns 64 (w / 4) .. + 63
    const int row = m0 + (warp & 3) * 32 + lane;
    const float alpha = (float)D.alpha, beta = (float)D.beta;
#pragma unroll 1
    for (int c0 = (warp >> 2) * 64; c0 < (warp >> 2) * 64 + 64; c0 += 16) {
      float v[16];
      if (nk > 0) {
        tc::tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.0f;
      }
      if (row < D.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (col < D.N) {
            float* cp = D.C + (size_t)row + (size_t)col * D.ldc;
            *cp = beta == 0.0f ? alpha * v[j] : alpha * v[j] + beta * *cp;
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_free(tmem, GT_N);
}

template <typename T>
__global__ void assemble_P_kernel(const PDescT<T>* descs, int ndesc) {
  const PDescT<T> D = descs[blockIdx.y];
  const int64_t total = (int64_t)D.s * D.ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % D.s), jj = (int)(e / D.s);
    const int col = D.piv[jj];
    const double val =
        jj < D.s ? (r == jj ? 1.0 : 0.0) : (double)D.A[(size_t)r + (size_t)jj * D.ld];
    D.P[(size_t)r + (size_t)col * D.s] = val;
    if (r == 0 && jj < D.s)
      D.skel[jj] = D.colsA ? (col < D.nA ? D.colsA[col] : D.colsB[col - D.nA]) : D.col0 + col;
  }
}

// ---------------------------------------------------------------- LU (GETRF)
// Blocked right-looking LU with partial pivoting, one CTA per matrix:
//   for each panel of NB columns: factor the panel column by column (pivot search
//   over the whole remaining column, swaps inside the panel), apply the panel's
//   row swaps to the other columns, U12 = L11^{-1} A12, and A22 -= L21 U12 as a
//   tiled product.  The row swaps touch whole rows, as LAPACK's GETRF stores them.
constexpr int LU_THREADS = 256;
constexpr int LU_NB = 32;
constexpr int LU_MAX_N = 1024;  // largest LU block
constexpr int LU_TM = 64;  // trailing-update tile (rows)
constexpr int LU_TN = 64;  // trailing-update tile (cols)

// After an LU (every thread of the block): per 32 x 32 diagonal block, the inverse of
// L's unit lower block and of U's upper block, and the permutation of the pivots (see
// LuDescT).  A warp inverts one block: lane i holds row i of the block and builds row i
// of the inverse, every step a broadcast of one finished row (32 shuffles) and one
// multiply-add per column.  A zero diagonal of U (reported as singular by the LU)
// leaves an infinite row.
template <typename T>
__device__ void lu_diag_inverses(const LuDescT<T>& D) {
  if constexpr (sizeof(T) == 4) {
    if (!D.dinv) return;
    __shared__ int perm_s[1024];
    const int n = D.n, ld = D.ld, nb = (n + 31) / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T* A = D.A;
    __syncthreads();
    for (int job = warp; job < 2 * nb; job += LU_THREADS / 32) {
      const int blk = job >> 1, upper = job & 1, b0 = 32 * blk, bs = min(32, n - b0);
      T row[32], inv[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        row[k] = (lane < bs && k < bs) ? A[(size_t)(b0 + lane) + (size_t)(b0 + k) * ld] : (T)0;
        inv[k] = (k == lane && lane < bs) ? (T)1 : (T)0;
      }
      if (!upper) {
        // row i of L^-1 = e_i - sum_{k < i} l_ik (row k of L^-1)
#pragma unroll
        for (int k = 0; k < 31; ++k) {
          const T l = row[k];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const T v = __shfl_sync(0xffffffffu, inv[j], k);
            if (lane > k) inv[j] -= l * v;
          }
        }
      } else {
        // row i of U^-1 = (e_i - sum_{k > i} u_ik (row k of U^-1)) / u_ii, from the bottom
#pragma unroll
        for (int k = 31; k >= 0; --k) {
          if (lane == k && k < bs) {
            const T r = (T)1 / row[k];
#pragma unroll
            for (int j = 0; j < 32; ++j) inv[j] *= r;
          }
          const T u = row[k];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const T v = __shfl_sync(0xffffffffu, inv[j], k);
            if (lane < k) inv[j] -= u * v;
          }
        }
      }
      T* out = D.dinv + (size_t)2048 * blk + (size_t)upper * 1024 + (size_t)lane * 32;
#pragma unroll
      for (int j = 0; j < 32; ++j) out[j] = lane < bs ? inv[j] : (T)0;
    }
    // the pivots' row permutation: perm[i] = source row of row i after all interchanges
    for (int i = tid; i < n; i += LU_THREADS) perm_s[i] = i;
    __syncthreads();
    if (tid == 0)
      for (int k = 0; k < n; ++k) {
        const int p = D.ipiv[k];
        if (p != k) {
          const int t = perm_s[k];
          perm_s[k] = perm_s[p];
          perm_s[p] = t;
        }
      }
    __syncthreads();
    int* perm = reinterpret_cast<int*>(D.dinv + (size_t)2048 * nb);
    for (int i = tid; i < n; i += LU_THREADS) perm[i] = perm_s[i];
  }
}

// PSH: the launch gave room for the panel (rows x NB) in shared memory; else it is
// factored in place.  The trailing update's next tile (operands) and this tile's C
// values are loaded into registers while the current tile's products run.
template <typename T, bool PSH>
__global__ void __launch_bounds__(LU_THREADS, sizeof(T) == 4 ? 2 : 1)
    getrf_kernel(const LuDescT<T>* descs, int* status, int pld) {
  __shared__ T rv[LU_THREADS / 32];
  __shared__ int ri[LU_THREADS / 32];
  __shared__ T L11[LU_NB][LU_NB + 1];
  __shared__ T As[LU_NB][LU_TM + 1];
  __shared__ T Bs[LU_NB][LU_TN + 1];
  __shared__ int sw_perm[LU_MAX_N], sw_src[2 * LU_NB], sw_dst[2 * LU_NB];
  __shared__ int sw_m;
  extern __shared__ __align__(16) unsigned char lu_sh[];
  const LuDescT<T> D = descs[blockIdx.x];
  T* A = D.A;
  const int n = D.n, ld = D.ld;
  const int tid = threadIdx.x;
  auto at = [&](int i, int j) -> T& { return A[(size_t)i + (size_t)j * ld]; };
  for (int k0 = 0; k0 < n; k0 += LU_NB) {
    const int nb = min(LU_NB, n - k0);
    // 1. panel factorization: rows k0.. of the panel's columns, in shared memory when
    //    the launch gave room for them (PSH), else in place
    T* pb = PSH ? reinterpret_cast<T*>(lu_sh) : A + (size_t)k0 * ld;
    const int pl = PSH ? pld : ld, roff = PSH ? k0 : 0;
    auto pn = [&](int i, int c) -> T& { return pb[(size_t)(i - roff) + (size_t)c * pl]; };
    if (PSH) {
      for (int e = tid; e < (n - k0) * nb; e += LU_THREADS) {
        const int i = k0 + e % (n - k0), c = e / (n - k0);
        pn(i, c) = at(i, k0 + c);
      }
      __syncthreads();
    }
    for (int j = 0; j < nb; ++j) {
      const int k = k0 + j;
      T best = (T)-1;  // partial pivoting on |a_ik| in T (ties to the lowest row)
      int bi = INT_MAX;
      for (int i = k + tid; i < n; i += LU_THREADS) {
        const T a = fabs(pn(i, j));
        if (a > best || (a == best && i < bi)) {
          best = a;
          bi = i;
        }
      }
      // the warps' candidates, then every thread combines them (one barrier)
      warp_argmax_t(best, bi);
      if ((tid & 31) == 0) {
        rv[tid >> 5] = best;
        ri[tid >> 5] = bi;
      }
      __syncthreads();
      best = rv[0];
      bi = ri[0];
#pragma unroll
      for (int w = 1; w < LU_THREADS / 32; ++w) {
        const T v2 = rv[w];
        const int i2 = ri[w];
        if (v2 > best || (v2 == best && i2 < bi)) {
          best = v2;
          bi = i2;
        }
      }
      const int p = bi;
      if (tid == 0) D.ipiv[k] = p;
      if (p != k && tid < nb) {
        T t = pn(k, tid);
        pn(k, tid) = pn(p, tid);
        pn(p, tid) = t;
      }
      __syncthreads();
      const T piv = pn(k, j);
      if (piv == (T)0) {
        if (tid == 0) atomicOr(status, DEV_SINGULAR);
        continue;
      }
      // scaling and rank-1 update of the panel's remaining columns: a thread per row,
      // the pivot row's entries in registers, each row's entries loaded before any of
      // them is stored
      T prow[LU_NB];
#pragma unroll
      for (int c = 0; c < LU_NB; ++c) prow[c] = (c > j && c < nb) ? pn(k, c) : (T)0;
      for (int i = k + 1 + tid; i < n; i += LU_THREADS) {
        T row[LU_NB];
#pragma unroll
        for (int c = 0; c < LU_NB; ++c) row[c] = (c > j && c < nb) ? pn(i, c) : (T)0;
        const T l = pn(i, j) / piv;
        pn(i, j) = l;
#pragma unroll
        for (int c = 0; c < LU_NB; ++c)
          if (c > j && c < nb) pn(i, c) = row[c] - l * prow[c];
      }
      __syncthreads();
    }
    if (PSH) {
      for (int e = tid; e < (n - k0) * nb; e += LU_THREADS) {
        const int i = k0 + e % (n - k0), c = e / (n - k0);
        at(i, k0 + c) = pn(i, c);
      }
      __syncthreads();
    }
    // 2. the panel's row interchanges on the columns outside the panel, as one
    //    permutation: row i receives old row sw_perm[i - k0]; the (at most 2 nb) rows
    //    that move are listed, then every warp moves them column by column with all of
    //    a column group's loads issued before its stores
    for (int i = k0 + tid; i < n; i += LU_THREADS) sw_perm[i - k0] = i;
    if (tid == 0) sw_m = 0;
    __syncthreads();
    if (tid == 0)
      for (int j = 0; j < nb; ++j) {
        const int p = D.ipiv[k0 + j];
        if (p != k0 + j) {
          const int t = sw_perm[j];
          sw_perm[j] = sw_perm[p - k0];
          sw_perm[p - k0] = t;
        }
      }
    __syncthreads();
    for (int i = k0 + tid; i < n; i += LU_THREADS)
      if (sw_perm[i - k0] != i) {
        const int q = atomicAdd(&sw_m, 1);
        sw_src[q] = sw_perm[i - k0];
        sw_dst[q] = i;
      }
    __syncthreads();
    {
      const int m = sw_m, nout = n - nb, lane = tid & 31, warp = tid >> 5;
      for (int x0 = warp * 4; x0 < nout && m > 0; x0 += 4 * (LU_THREADS / 32)) {
        T v[2][4];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int t = lane + 32 * q, x = x0 + u;
            const int c = x < k0 ? x : x + nb;
            v[q][u] = (t < m && x < nout) ? at(sw_src[t], c) : (T)0;
          }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int t = lane + 32 * q, x = x0 + u;
            const int c = x < k0 ? x : x + nb;
            if (t < m && x < nout) at(sw_dst[t], c) = v[q][u];
          }
      }
    }
    __syncthreads();
    const int c0 = k0 + nb;
    if (c0 >= n) break;
    // 3. U12 = L11^{-1} A12 (unit lower), one thread per column
    for (int t = tid; t < nb * nb; t += LU_THREADS) L11[t % nb][t / nb] = at(k0 + t % nb, k0 + t / nb);
    __syncthreads();
    for (int c = c0 + tid; c < n; c += LU_THREADS) {
      T x[LU_NB];
#pragma unroll
      for (int r = 0; r < LU_NB; ++r) x[r] = r < nb ? at(k0 + r, c) : (T)0;
#pragma unroll
      for (int r = 1; r < LU_NB; ++r) {
        T acc = x[r];
#pragma unroll
        for (int q = 0; q < LU_NB; ++q)
          if (q < r) acc -= L11[r][q] * x[q];
        x[r] = acc;
      }
#pragma unroll
      for (int r = 0; r < LU_NB; ++r)
        if (r < nb) at(k0 + r, c) = x[r];
    }
    __syncthreads();
    // 4. A22 -= L21 U12, tiles of LU_TM x LU_TN, 4 x 4 per thread; tile t + 1's operands
    //    are in flight during tile t's products
    const int m2 = n - c0;
    const int tx = tid & 15, ty = tid >> 4;
    const int ntm = (m2 + LU_TM - 1) / LU_TM, ntiles = ntm * ((m2 + LU_TN - 1) / LU_TN);
    constexpr int AV = LU_NB * LU_TM / LU_THREADS, BV = LU_NB * LU_TN / LU_THREADS;
    T an[AV], bn[BV];
    auto fetch = [&](int t) {
      const int tm = (t % ntm) * LU_TM, tn = (t / ntm) * LU_TN;
#pragma unroll
      for (int u = 0; u < AV; ++u) {
        const int e = tid + u * LU_THREADS, r = e % LU_TM, q = e / LU_TM;
        an[u] = (q < nb && tm + r < m2) ? at(c0 + tm + r, k0 + q) : (T)0;
      }
#pragma unroll
      for (int u = 0; u < BV; ++u) {
        const int e = tid + u * LU_THREADS, q = e % LU_NB, cc = e / LU_NB;
        bn[u] = (q < nb && tn + cc < m2) ? at(k0 + q, c0 + tn + cc) : (T)0;
      }
    };
    if (ntiles > 0) fetch(0);
    for (int t = 0; t < ntiles; ++t) {
      const int tm = (t % ntm) * LU_TM, tn = (t / ntm) * LU_TN;
#pragma unroll
      for (int u = 0; u < AV; ++u) {
        const int e = tid + u * LU_THREADS;
        As[e / LU_TM][e % LU_TM] = an[u];
      }
#pragma unroll
      for (int u = 0; u < BV; ++u) {
        const int e = tid + u * LU_THREADS;
        Bs[e % LU_NB][e / LU_NB] = bn[u];
      }
      __syncthreads();
      if (t + 1 < ntiles) fetch(t + 1);
      T cv[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int r = tm + tx + 16 * a, cc = tn + ty + 16 * b;
          cv[a][b] = (r < m2 && cc < m2) ? at(c0 + r, c0 + cc) : (T)0;
        }
      T acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
#pragma unroll 8
      for (int q = 0; q < LU_NB; ++q) {
        T av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[q][tx + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Bs[q][ty + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int r = tm + tx + 16 * a, cc = tn + ty + 16 * b;
          if (r < m2 && cc < m2) at(c0 + r, c0 + cc) = cv[a][b] - acc[a][b];
        }
      __syncthreads();
    }
  }
}

// One block per factored LU: its dinv area (lu_diag_inverses).
__global__ void __launch_bounds__(LU_THREADS, 1) lu_dinv_kernel(const LuDescT<float>* descs) {
  lu_diag_inverses(descs[blockIdx.x]);
}

// ---------------------------------------------------------------- GETRS
// Grid (chunk of NC right-hand sides, descriptor): the chunks of one matrix are
// neighbours in launch order, so its LU factors are read from L2 after the first.
// The chunk lives in shared memory; rows are processed in blocks of 32: a warp solves the 32 x 32 diagonal
// block for one column with shuffles, then all threads update the rows below
// (forward) or above (backward) with a register-tiled product.
constexpr int RS_THREADS = 256;

// 16-byte vector of T for shared-memory broadcasts
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};

// out[c] = X[row * NC + c] for c < NC: 16-byte loads where the row is 16-byte aligned
template <typename T, int NC>
__device__ __forceinline__ void load_row(const T* X, int row, T (&out)[NC]) {
  if constexpr ((NC * sizeof(T)) % 16 == 0) {
    using V = typename Vec16<T>::type;
    const V* p = reinterpret_cast<const V*>(X + (size_t)row * NC);
#pragma unroll
    for (int q = 0; q < NC / Vec16<T>::n; ++q) {
      const V v = p[q];
      const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
      for (int u = 0; u < Vec16<T>::n; ++u) out[q * Vec16<T>::n + u] = e[u];
    }
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) out[c] = X[(size_t)row * NC + c];
  }
}

// (s, c) += (ah + al)(bh + bl): the product ah bh exactly as p + e (FMA), the cross
// terms and e into the low part, p into the high part by Knuth's two-sum (its rounding
// error into the low part as well).  The explicitly rounded operations keep the
// compiler from contracting the two-sum into FMAs.
__device__ __forceinline__ void pair_mac(float ah, float al, float bh, float bl, float& s, float& c) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  c = __fadd_rn(c, __fadd_rn(err, e));
  s = t;
}

// X_r -= sum_{k < bs} M[r, b0 + k] X_{b0 + k} (one row r, NC columns) with the 32 rows
// X_{b0..} given as FP32 pairs in Xp (row-major, 32 x NC): each FP64 entry of M is split
// into a pair as it is loaded, the products are formed exactly and summed as pairs
// (pair_mac), and the sum is subtracted in FP64.  Only the split and the final
// subtraction use the FP64 pipe: one FP64 operation per entry of M instead of NC FMAs.
template <int NC>
__device__ __forceinline__ void pair_row_update(const double* M, int ld, int r, int b0, int bs,
                                                const float2* Xp, double* X) {
  float s[NC], c[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) s[q] = c[q] = 0.0f;
  for (int k = 0; k < bs; ++k) {
    const double mv = M[(size_t)r + (size_t)(b0 + k) * ld];
    const float mh = __double2float_rn(mv), ml = __double2float_rn(mv - (double)mh);
    const float2* xr = Xp + k * NC;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const float2 x = xr[q];
      pair_mac(mh, ml, x.x, x.y, s[q], c[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) X[(size_t)r * NC + q] -= (double)s[q] + (double)c[q];
}

// The rows b0 .. b0 + bs of X, split into FP32 pairs (rows past bs zero).
template <int NC>
__device__ __forceinline__ void split_rows(const double* X, int b0, int bs, float2* Xp, int tid) {
  for (int e = tid; e < 32 * NC; e += RS_THREADS) {
    const int k = e / NC;
    const double v = k < bs ? X[(size_t)(b0 + k) * NC + (e % NC)] : 0.0;
    const float h = __double2float_rn(v);
    Xp[e] = make_float2(h, __double2float_rn(v - (double)h));
  }
}

// X (n x NC chunk of right-hand sides) lives in shared memory row-major, so that the
// register-tiled updates read a row of X with 16-byte broadcasts.  The 32 x 32
// diagonal blocks are read into registers before their sequential substitution.
// PAIR (FP64 only): the updates below and above each diagonal block run on FP32 pairs
// (pair_row_update); the substitutions through the diagonal blocks stay in FP64.
template <typename T, int NC, bool UPPER_ONLY, bool PAIR>
__global__ void __launch_bounds__(RS_THREADS) getrs_kernel(const LuSolveDescT<T>* descs) {
  static_assert(!PAIR || sizeof(T) == 8, "pair updates take FP64 factors");
  extern __shared__ __align__(16) unsigned char rs_sh[];
  // PAIR: the current block's 32 rows as pairs first, 32 x NC float2
  float2* Xp = reinterpret_cast<float2*>(rs_sh);
  T* X = reinterpret_cast<T*>(rs_sh + (PAIR ? 32 * NC * sizeof(float2) : 0));  // n x NC, X[i * NC + c]
  const LuSolveDescT<T> D = descs[blockIdx.y];
  const int c0 = blockIdx.x * NC;
  if (c0 >= D.ncols) return;
  const int nc = min(NC, D.ncols - c0);
  const int n = D.n;
  const T* LU = D.LU;
  const int ld = D.ldlu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int t = tid; t < n * NC; t += RS_THREADS) {
    const int i = t % n, c = t / n;
    X[(size_t)i * NC + c] = c < nc ? D.B[(size_t)i + (size_t)(c0 + c) * D.ldb] : (T)0;
  }
  __syncthreads();
  if (!UPPER_ONLY && tid < nc) {
    for (int k = 0; k < n; ++k) {
      const int p = D.ipiv[k];
      if (p != k) {
        const T t = X[(size_t)k * NC + tid];
        X[(size_t)k * NC + tid] = X[(size_t)p * NC + tid];
        X[(size_t)p * NC + tid] = t;
      }
    }
  }
  __syncthreads();
  // forward substitution with the unit lower triangle
  for (int b0 = 0; b0 < (UPPER_ONLY ? 0 : n); b0 += 32) {
    const int bs = min(32, n - b0);
    if (warp < nc) {
      if constexpr (sizeof(T) == 4) {
        T l[32];  // row b0 + lane of the diagonal block (FP32: registers to spare)
#pragma unroll
        for (int k = 0; k < 32; ++k)
          l[k] = (lane < bs && k < bs) ? LU[(size_t)(b0 + lane) + (size_t)(b0 + k) * ld] : (T)0;
        for (int c = warp; c < nc; c += RS_THREADS / 32) {
          T x = lane < bs ? X[(size_t)(b0 + lane) * NC + c] : (T)0;
#pragma unroll
          for (int k = 0; k < 31; ++k) {
            const T xk = __shfl_sync(0xffffffffu, x, k);
            if (k < bs - 1 && lane > k && lane < bs) x -= l[k] * xk;
          }
          if (lane < bs) X[(size_t)(b0 + lane) * NC + c] = x;
        }
      } else {
        for (int c = warp; c < nc; c += RS_THREADS / 32) {
          T x = lane < bs ? X[(size_t)(b0 + lane) * NC + c] : (T)0;
          for (int k = 0; k < bs - 1; ++k) {
            const T xk = __shfl_sync(0xffffffffu, x, k);
            if (lane > k && lane < bs) x -= LU[(size_t)(b0 + lane) + (size_t)(b0 + k) * ld] * xk;
          }
          if (lane < bs) X[(size_t)(b0 + lane) * NC + c] = x;
        }
      }
    }
    __syncthreads();
    if constexpr (PAIR) {
      if (b0 + bs < n) {
        split_rows<NC>(reinterpret_cast<const double*>(X), b0, bs, Xp, tid);
        __syncthreads();
        for (int r = b0 + bs + tid; r < n; r += RS_THREADS)
          pair_row_update<NC>(reinterpret_cast<const double*>(LU), ld, r, b0, bs, Xp,
                              reinterpret_cast<double*>(X));
      }
      __syncthreads();
      continue;
    }
    for (int r = b0 + bs + tid; r < n; r += RS_THREADS) {
      T acc[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = 0;
      for (int k = 0; k < bs; ++k) {
        const T lv = LU[(size_t)r + (size_t)(b0 + k) * ld];
        T xv[NC];
        load_row<T, NC>(X, b0 + k, xv);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fma(lv, xv[c], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) X[(size_t)r * NC + c] -= acc[c];
    }
    __syncthreads();
  }
  // backward substitution with the upper triangle
  for (int b1 = n; b1 > 0; b1 -= 32) {
    const int b0 = max(0, b1 - 32), bs = b1 - b0;
    if (warp < nc) {
      if constexpr (sizeof(T) == 4) {
        T u[32];
#pragma unroll
        for (int k = 0; k < 32; ++k)
          u[k] = (lane < bs && k < bs) ? LU[(size_t)(b0 + lane) + (size_t)(b0 + k) * ld] : (T)0;
        for (int c = warp; c < nc; c += RS_THREADS / 32) {
          T x = lane < bs ? X[(size_t)(b0 + lane) * NC + c] : (T)0;
#pragma unroll
          for (int k = 31; k >= 0; --k) {
            if (k < bs) {
              // a zero diagonal entry (rank-deficient R11) gives a zero row in the ID
              if (lane == k) x = (UPPER_ONLY && u[k] == (T)0) ? (T)0 : x / u[k];
              const T xk = __shfl_sync(0xffffffffu, x, k);
              if (lane < k) x -= u[k] * xk;
            }
          }
          if (lane < bs) X[(size_t)(b0 + lane) * NC + c] = x;
        }
      } else {
        // each lane the reciprocal of its own diagonal entry, once per block: one FP64
        // division per warp instead of one per substitution step
        T rinv = (T)0;
        if (lane < bs) {
          const T dk = LU[(size_t)(b0 + lane) + (size_t)(b0 + lane) * ld];
          rinv = (UPPER_ONLY && dk == (T)0) ? (T)0 : (T)1 / dk;
        }
        for (int c = warp; c < nc; c += RS_THREADS / 32) {
          T x = lane < bs ? X[(size_t)(b0 + lane) * NC + c] : (T)0;
          for (int k = bs - 1; k >= 0; --k) {
            if (lane == k) x *= rinv;
            const T xk = __shfl_sync(0xffffffffu, x, k);
            if (lane < k) x -= LU[(size_t)(b0 + lane) + (size_t)(b0 + k) * ld] * xk;
          }
          if (lane < bs) X[(size_t)(b0 + lane) * NC + c] = x;
        }
      }
    }
    __syncthreads();
    if constexpr (PAIR) {
      if (b0 > 0) {
        split_rows<NC>(reinterpret_cast<const double*>(X), b0, bs, Xp, tid);
        __syncthreads();
        for (int r = tid; r < b0; r += RS_THREADS)
          pair_row_update<NC>(reinterpret_cast<const double*>(LU), ld, r, b0, bs, Xp,
                              reinterpret_cast<double*>(X));
      }
      __syncthreads();
      continue;
    }
    for (int r = tid; r < b0; r += RS_THREADS) {
      T acc[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = 0;
      for (int k = 0; k < bs; ++k) {
        const T uv = LU[(size_t)r + (size_t)(b0 + k) * ld];
        T xv[NC];
        load_row<T, NC>(X, b0 + k, xv);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fma(uv, xv[c], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) X[(size_t)r * NC + c] -= acc[c];
    }
    __syncthreads();
  }
  for (int t = tid; t < n * nc; t += RS_THREADS) {
    const int i = t % n, c = t / n;
    D.B[(size_t)i + (size_t)(c0 + c) * D.ldb] = X[(size_t)i * NC + c];
  }
}

// D (16 x 8, FP32) += A (16 x 8) B (8 x 8), TF32 operands, one warp (mma.sync
// m16n8k8; A row-major fragments: rows lane/4 and lane/4 + 8, columns lane%4 and
// lane%4 + 4; B column fragments: rows lane%4 and lane%4 + 4, column lane/4; D: rows
// lane/4 and lane/4 + 8, columns 2 (lane%4) and 2 (lane%4) + 1).
__device__ __forceinline__ void mma_tf32_16x8x8(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// FP32 LU solve with the diagonal blocks' inverses (lu_diag_inverses): rows gathered
// through the pivots' permutation; per 32-row block, X_b <- (L_bb)^-1 X_b as a small
// product (every thread: one row, two columns), then the rows below get
// X_r -= L_rb X_b, two rows per thread with the 16 columns in registers; the same
// upwards with U.  No step is a sequential substitution, and every global load of a
// step is issued before its values are used: the block's 32 L (or U) values of a row
// are loaded together, and the next step's inverse block is fetched during this one.
// INV (GETRI): the right-hand sides are the identity's columns and the result is the
// matrix's inverse.  With P A = L U, A^-1 = U^-1 L^-1 P: chunk c0 solves for the
// identity's columns c0 .. c0 + 15, whose rows above c0 stay zero through the forward
// pass (its first c0 / 32 steps are skipped), and column c of U^-1 L^-1 is column
// perm[c] of A^-1, where the chunk writes it.
constexpr int RI_NC = 16;
constexpr int RI_LD = RI_NC + 4;  // X row stride: consecutive rows in distinct shared-memory banks
template <bool INV>
__global__ void __launch_bounds__(RS_THREADS, 2) getrs_inv_kernel(const LuSolveDescT<float>* descs) {
  extern __shared__ __align__(16) unsigned char ri_sh[];
  float* X = reinterpret_cast<float*>(ri_sh);  // n x RI_NC, row-major, stride RI_LD
  __shared__ __align__(16) float Dv[32][33];
  const LuSolveDescT<float> D = descs[blockIdx.y];
  const int c0 = blockIdx.x * RI_NC;
  if (c0 >= D.ncols) return;
  const int nc = min(RI_NC, D.ncols - c0), n = D.n, ld = D.ldlu, nb = (n + 31) / 32;
  const float* LU = D.LU;
  const int* perm = reinterpret_cast<const int*>(D.dinv + (size_t)2048 * nb);
  const int tid = threadIdx.x;
  for (int t = tid; t < n * RI_NC; t += RS_THREADS) {
    const int i = t % n, c = t / n;
    if constexpr (INV) X[(size_t)i * RI_LD + c] = (c < nc && i == c0 + c) ? 1.0f : 0.0f;
    else X[(size_t)i * RI_LD + c] = c < nc ? D.B[(size_t)perm[i] + (size_t)(c0 + c) * D.ldb] : 0.0f;
  }
  const int s0 = INV ? (c0 >> 5) : 0;          // first forward step with a nonzero row
  const int di = tid >> 3, dc = (tid & 7) * 2;  // diagonal product: row di, columns dc, dc + 1
  constexpr int DV_PER = 1024 / RS_THREADS;     // inverse entries staged per thread
  float dnext[DV_PER];
  auto fetch_inv = [&](int pass, int step) {
    const int blk = pass == 0 ? step : nb - 1 - step;
    const float* inv = D.dinv + (size_t)2048 * blk + (size_t)pass * 1024;
#pragma unroll
    for (int u = 0; u < DV_PER; ++u) dnext[u] = inv[tid + u * RS_THREADS];
  };
  fetch_inv(0, s0);
  for (int pass = 0; pass < 2; ++pass) {  // 0: L downwards, 1: U upwards
    for (int step = pass == 0 ? s0 : 0; step < nb; ++step) {
      const int blk = pass == 0 ? step : nb - 1 - step;
      const int b0 = 32 * blk, bs = min(32, n - b0);
      __syncthreads();  // X rows of the previous step are final; Dv is free
#pragma unroll
      for (int u = 0; u < DV_PER; ++u) {
        const int e = tid + u * RS_THREADS;
        Dv[e >> 5][e & 31] = dnext[u];
      }
      __syncthreads();
      // the next step's inverse block, in flight during this step
      if (step + 1 < nb) fetch_inv(pass, step + 1);
      else if (pass == 0) fetch_inv(1, 0);
      float o0 = 0.0f, o1 = 0.0f;
      if (di < bs) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          if (k < bs) {
            const float a = Dv[di][k];
            const float2 xv = *reinterpret_cast<const float2*>(&X[(size_t)(b0 + k) * RI_LD + dc]);
            o0 = fmaf(a, xv.x, o0);
            o1 = fmaf(a, xv.y, o1);
          }
        }
      }
      __syncthreads();
      if (di < bs) *reinterpret_cast<float2*>(&X[(size_t)(b0 + di) * RI_LD + dc]) = make_float2(o0, o1);
      __syncthreads();
      // rows to update: below the block (L) or above it (U).  X_r -= L_rb X_b as
      // 16 x 16 x 32 products on the tensor cores (mma.sync m16n8k8 TF32, three
      // products per FP32 product: lo.hi + hi.lo + hi.hi), one 16-row group per warp
      // at a time; X_b's fragments are split once per step.
      const int r_lo = pass == 0 ? b0 + bs : 0, r_hi = pass == 0 ? n : b0;
      const int warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
      uint32_t bh[4][2][2], bl[4][2][2];  // [k tile][n tile][reg]
#pragma unroll
      for (int kt = 0; kt < 4; ++kt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int k = kt * 8 + tq + 4 * q;
            const float x = k < bs ? X[(size_t)(b0 + k) * RI_LD + nt * 8 + gq] : 0.0f;
            bh[kt][nt][q] = tc::to_tf32(x);
            bl[kt][nt][q] = tc::to_tf32(x - __uint_as_float(bh[kt][nt][q]));
          }
      // the L (or U) fragments of a row group: rows gq, gq + 8; columns tq, tq + 4
      auto load_frag = [&](int R, float (&f)[4][4]) {
        const int ra = R + gq, rb = R + gq + 8;
        const bool va = ra < r_hi, vb = rb < r_hi;
        const float* la = LU + (size_t)(va ? ra : r_lo) + (size_t)b0 * ld;
        const float* lb = LU + (size_t)(vb ? rb : r_lo) + (size_t)b0 * ld;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
          const int k0 = kt * 8 + tq, k1 = k0 + 4;
          f[kt][0] = (va && k0 < bs) ? la[(size_t)k0 * ld] : 0.0f;
          f[kt][1] = (vb && k0 < bs) ? lb[(size_t)k0 * ld] : 0.0f;
          f[kt][2] = (va && k1 < bs) ? la[(size_t)k1 * ld] : 0.0f;
          f[kt][3] = (vb && k1 < bs) ? lb[(size_t)k1 * ld] : 0.0f;
        }
      };
      constexpr int RSTEP = 16 * (RS_THREADS / 32);
      float av[4][4], an[4][4];  // this row group's fragments, and the next one's (in flight)
      if (r_lo + 16 * warp < r_hi) load_frag(r_lo + 16 * warp, av);
      for (int R0 = r_lo + 16 * warp; R0 < r_hi; R0 += RSTEP) {
        const int ra = R0 + gq, rb = R0 + gq + 8;
        const bool va = ra < r_hi, vb = rb < r_hi;
        if (R0 + RSTEP < r_hi) load_frag(R0 + RSTEP, an);
        float acc[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[nt][q] = 0.0f;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
          uint32_t ah[4], al[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            ah[q] = tc::to_tf32(av[kt][q]);
            al[q] = tc::to_tf32(av[kt][q] - __uint_as_float(ah[q]));
          }
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) {
            mma_tf32_16x8x8(acc[nt], al, bh[kt][nt]);
            mma_tf32_16x8x8(acc[nt], ah, bl[kt][nt]);
            mma_tf32_16x8x8(acc[nt], ah, bh[kt][nt]);
          }
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int c = nt * 8 + 2 * tq;
          if (va) {
            float2* xa = reinterpret_cast<float2*>(&X[(size_t)ra * RI_LD + c]);
            const float2 t = *xa;
            *xa = make_float2(t.x - acc[nt][0], t.y - acc[nt][1]);
          }
          if (vb) {
            float2* xb = reinterpret_cast<float2*>(&X[(size_t)rb * RI_LD + c]);
            const float2 t = *xb;
            *xb = make_float2(t.x - acc[nt][2], t.y - acc[nt][3]);
          }
        }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt)
#pragma unroll
          for (int q = 0; q < 4; ++q) av[kt][q] = an[kt][q];
      }
    }
  }
  __syncthreads();
  for (int t = tid; t < n * nc; t += RS_THREADS) {
    const int i = t % n, c = t / n;
    const int oc = INV ? perm[c0 + c] : c0 + c;
    D.B[(size_t)i + (size_t)oc * D.ldb] = X[(size_t)i * RI_LD + c];
  }
}

// ---------------------------------------------------------------- GEMM
constexpr int GK = 16;   // k step
constexpr int G_THREADS = 256;

// Tile TM x TN, 256 threads, 4 x 4 outputs per thread: (64, 64) for general
// problems, (256, 16) when every problem of the launch has at most 16 columns.
template <typename T, int TM, int TN>
__global__ void __launch_bounds__(G_THREADS) gemm_kernel(const GemmDescT<T>* descs,
                                                         const GemmTile* tiles) {
  constexpr int TX = TM / 4, TY = TN / 4;
  static_assert(TX * TY == G_THREADS, "tile must map to 256 threads");
  __shared__ __align__(16) T As[GK][TM + 4];
  __shared__ __align__(16) T Bs[GK][TN + 4];
  const GemmTile Tl = tiles[blockIdx.x];
  const GemmDescT<T> D = descs[Tl.desc];
  const int m0 = Tl.tm * TM, n0 = Tl.tn * TN;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  // the FP32 64 x 64 tiles (only used without the tensor-core GEMM) keep the plain loop:
  // the test below costs them a register spill
  constexpr bool SKIP = sizeof(T) == 8 || TN <= 32;
  const bool live = !SKIP || (m0 + 4 * tx < D.M && n0 + 4 * ty < D.N);
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  for (int k0 = 0; k0 < D.K; k0 += GK) {
#pragma unroll
    for (int r = 0; r < TM * GK / G_THREADS; ++r) {
      const int e = threadIdx.x + r * G_THREADS;
      const int am = e % TM, ak = e / TM;         // A tile: TM rows x 16 k
      const int gm = m0 + am, gk = k0 + ak;
      As[ak][am] = (gm < D.M && gk < D.K) ? D.A[(size_t)gm + (size_t)gk * D.lda] : (T)0;
    }
#pragma unroll
    for (int r = 0; r < (TN * GK + G_THREADS - 1) / G_THREADS; ++r) {
      const int e = threadIdx.x + r * G_THREADS;
      if (e < TN * GK) {
        const int bk = e % GK, bn = e / GK;       // B tile: 16 k x TN cols
        const int gk2 = k0 + bk, gn = n0 + bn;
        Bs[bk][bn] = (gk2 < D.K && gn < D.N) ? D.B[(size_t)gk2 + (size_t)gn * D.ldb] : (T)0;
      }
    }
    __syncthreads();
    // a thread whose 4 x 4 outputs all lie outside C (a tile wider or taller than the
    // problem: 4 right-hand sides in a 16-column tile) skips the arithmetic
    if (live) {
#pragma unroll
      for (int kk = 0; kk < GK; ++kk) {
        T a[4], b[4];  // rows 4 tx .. 4 tx + 3 and columns 4 ty .. 4 ty + 3: 16-byte loads
        load_row<T, 4>(&As[kk][0], tx, a);
        load_row<T, 4>(&Bs[kk][0], ty, b);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
      }
    }
    __syncthreads();
  }
  const T alpha = (T)D.alpha, beta = (T)D.beta;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gm = m0 + 4 * tx + r, gn = n0 + 4 * ty + c;
      if (gm < D.M && gn < D.N) {
        T* cp = D.C + (size_t)gm + (size_t)gn * D.ldc;
        *cp = D.beta == 0.0 ? alpha * acc[r][c] : alpha * acc[r][c] + beta * *cp;
      }
    }
}

// 512 x 8 tiles exist for FP32 only (the FP64 A tile would exceed static shared memory).
template <typename T>
void gemm_narrow(const GemmDescT<T>* descs_dev, const GemmTile* tiles_dev, int ntiles, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value)
    gemm_kernel<float, 512, 8><<<ntiles, G_THREADS, 0, st>>>(descs_dev, tiles_dev);
  else
    throw Error(IASKIT_ERR_ARG, "512 x 8 tiles are FP32 only");
}

// ---------------------------------------------------------------- small helpers
template <typename T>
__global__ void copy_kernel(const CopyDescT<T>* descs, int ndesc) {
  for (int q = blockIdx.y; q < ndesc; q += gridDim.y) {
    const CopyDescT<T> D = descs[q];
    const int64_t total = (int64_t)D.rows * D.cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int i = (int)(e % D.rows), j = (int)(e / D.rows);
      D.dst[(size_t)i + (size_t)j * D.ldd] = D.src[(size_t)i + (size_t)j * D.lds];
    }
  }
}

template <typename T>
__global__ void form_Z_kernel(const ZDescT<T>* descs, int ndesc) {
  for (int q = blockIdx.y; q < ndesc; q += gridDim.y) {
    const ZDescT<T> D = descs[q];
    const int n = D.sl + D.sr;
    const int64_t total = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int i = (int)(e % n), j = (int)(e / n);
      T v;
      if (i < D.sl && j < D.sl) v = (i == j) ? (T)1 : (T)0;
      else if (i >= D.sl && j >= D.sl) v = (i == j) ? (T)1 : (T)0;
      else if (i < D.sl) v = D.Cl[(size_t)i + (size_t)(j - D.sl) * D.sl];
      else v = D.Cr[(size_t)(i - D.sl) + (size_t)j * D.sr];
      D.Z[(size_t)i + (size_t)j * n] = v;
    }
  }
}

template <typename T>
__global__ void permute_rows_kernel(const T* in, int ldi, T* out, int ldo, const int* perm, int N,
                                    int ncols, bool scatter) {
  const int64_t total = (int64_t)N * ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e % N), c = (int)(e / N);
    if (scatter) out[(size_t)perm[p] + (size_t)c * ldo] = in[(size_t)p + (size_t)c * ldi];
    else out[(size_t)p + (size_t)c * ldo] = in[(size_t)perm[p] + (size_t)c * ldi];
  }
}

__global__ void d2f_kernel(const double* in, float* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void f2d_kernel(const float* in, double* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

// u_rows += K(x_rows, x_cols) y, one thread per target row, up to MV_R right-hand
// sides per pass; the column points are staged in shared memory.
constexpr int MV_THREADS = 128;
constexpr int MV_R = 16;
constexpr int MV_TILE = 32;
__global__ void __launch_bounds__(MV_THREADS) kernel_matvec_kernel(const double* Xp, const double* xn, int d,
                                                                   int nrhs, const KMatvecDesc* descs) {
  extern __shared__ double xs[];  // MV_TILE x d, then the MV_TILE column norms
  double* xcn = xs + MV_TILE * d;
  const KMatvecDesc D = descs[blockIdx.y];
  const double neg_inv_2h2 = D.scale;
  const int i = blockIdx.x * MV_THREADS + threadIdx.x;
  const bool active = i < D.nrows;
  const int row = D.row0 + (active ? i : 0);
  const double* xr = Xp + (size_t)row * d;
  const double xrn = xn[row];
  for (int c0 = 0; c0 < nrhs; c0 += MV_R) {
    const int nr = min(MV_R, nrhs - c0);
    double acc[MV_R];
#pragma unroll
    for (int c = 0; c < MV_R; ++c) acc[c] = 0.0;
    for (int k0 = 0; k0 < D.ncols; k0 += MV_TILE) {
      const int nt = min(MV_TILE, D.ncols - k0);
      __syncthreads();
      for (int e = threadIdx.x; e < nt * d; e += MV_THREADS) {
        const int kk = e / d, q = e % d;
        const int col = D.cols ? D.cols[k0 + kk] : D.col0 + k0 + kk;
        xs[kk * d + q] = Xp[(size_t)col * d + q];
      }
      for (int kk = threadIdx.x; kk < nt; kk += MV_THREADS)
        xcn[kk] = xn[D.cols ? D.cols[k0 + kk] : D.col0 + k0 + kk];
      __syncthreads();
      if (!active) continue;
      for (int kk = 0; kk < nt; ++kk) {
        double dot = 0.0;
        for (int q = 0; q < d; ++q) dot = fma(xr[q], xs[kk * d + q], dot);
        const double d2 = fmax((xrn + xcn[kk]) - 2.0 * dot, 0.0);  // Gram form, as kernel_blocks
        const double kv = kspec_value(g_kspec, dot, d2, neg_inv_2h2);
        const double* yk = D.y + (size_t)(k0 + kk) + (size_t)c0 * D.ldy;
#pragma unroll
        for (int c = 0; c < MV_R; ++c)
          if (c < nr) acc[c] = fma(kv, yk[(size_t)c * D.ldy], acc[c]);
      }
    }
    if (active)
      for (int c = 0; c < nr; ++c) D.u[(size_t)i + (size_t)(c0 + c) * D.ldu] += acc[c];
  }
}

__global__ void check_finite_kernel(const double* x, int64_t n, int* status) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, DEV_BADINPUT);
}

unsigned grid_for(int64_t work, int threads, unsigned cap = 65535u) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  return (unsigned)std::min<int64_t>(b, cap);
}

template <typename T, int NC, bool UPPER_ONLY, bool PAIR>
void launch_getrs(const LuSolveDescT<T>* descs_dev, int ndesc, int max_n, int max_cols,
                  cudaStream_t st) {
  const size_t smem = (size_t)max_n * NC * sizeof(T) + (PAIR ? 32 * NC * sizeof(float2) : 0);
  if (smem > 220 * 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "LU block too large");
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(getrs_kernel<T, NC, UPPER_ONLY, PAIR>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (ndesc > 65535) throw Error(IASKIT_ERR_UNSUPPORTED, "more than 65535 LU solves in one launch");
  dim3 grid(ceil_div(max_cols, NC), ndesc);
  getrs_kernel<T, NC, UPPER_ONLY, PAIR><<<grid, RS_THREADS, smem, st>>>(descs_dev);
  IA_LAUNCH_CHECK();
}

template <typename T, bool UPPER_ONLY, bool PAIR = false>
void solve_dispatch(const LuSolveDescT<T>* descs_dev, int ndesc, int max_n, int max_cols, cudaStream_t st) {
  // chunk width: 16 columns while the chunk stays small enough for 3 blocks per SM
  if (max_cols >= 16 && (size_t)max_n * 16 * sizeof(T) <= 72 * 1024)
    launch_getrs<T, 16, UPPER_ONLY, PAIR>(descs_dev, ndesc, max_n, max_cols, st);
  else if (max_cols >= 8 && (size_t)max_n * 8 * sizeof(T) <= 144 * 1024)
    launch_getrs<T, 8, UPPER_ONLY, PAIR>(descs_dev, ndesc, max_n, max_cols, st);
  else if (max_cols >= 4)
    launch_getrs<T, 4, UPPER_ONLY, PAIR>(descs_dev, ndesc, max_n, max_cols, st);
  else
    launch_getrs<T, 1, UPPER_ONLY, PAIR>(descs_dev, ndesc, max_n, max_cols, st);
}

}  // namespace

template <typename T>
void kernel_blocks(const double* Xp, const double* xnorm, int d, const KDescT<T>* descs_dev, int ndesc,
                   int64_t max_entries, cudaStream_t st) {
  if (ndesc <= 0 || max_entries <= 0) return;
  if (std::is_same<T, double>::value && !xnorm) throw Error(IASKIT_ERR_ARG, "kernel blocks need point norms");
  if (ndesc > 65535) throw Error(IASKIT_ERR_UNSUPPORTED, "more than 65535 kernel blocks in one launch");
  // blocks per descriptor: about its tile count (the kernel strides over the tiles)
  const int64_t max_tiles = std::min<int64_t>(max_entries / (KB_T * KB_T / 2) + 1, 4096);
  const size_t smem = (size_t)2 * KB_T * d * sizeof(T);
  if (smem > 200 * 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "dimension too large for kernel blocks");
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(kernel_blocks_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope _ps(pk_of<T>(PK_KBLOCK), st);
  dim3 grid((unsigned)max_tiles, ndesc);
  kernel_blocks_kernel<T><<<grid, KB_THREADS, smem, st>>>(Xp, xnorm, d, descs_dev);
  IA_LAUNCH_CHECK();
}

void kernel_blocks_pair(const float2* Xpair, int d, const KDescT<float2>* descs_dev, int ndesc,
                        int64_t max_entries, cudaStream_t st) {
  if (ndesc <= 0 || max_entries <= 0) return;
  if (ndesc > 65535) throw Error(IASKIT_ERR_UNSUPPORTED, "more than 65535 kernel blocks in one launch");
  const int64_t max_tiles = std::min<int64_t>(max_entries / (KB_T * KB_T / 2) + 1, 4096);
  const size_t smem = (size_t)2 * KB_T * d * sizeof(float2);
  if (smem > 200 * 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "dimension too large for kernel blocks");
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(kernel_blocks_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope _ps(PK_KBLOCK_PAIR, st);
  dim3 grid((unsigned)max_tiles, ndesc);
  kernel_blocks_pair_kernel<<<grid, KB_THREADS, smem, st>>>(Xpair, d, descs_dev);
  IA_LAUNCH_CHECK();
}

void point_norms(const double* Xp, int N, int d, double* out, cudaStream_t st) {
  if (N <= 0) return;
  ProfScope _ps(PK_MISC, st);
  row_norms_kernel<<<ceil_div(N, 256), 256, 0, st>>>(Xp, N, d, out);
  IA_LAUNCH_CHECK();
}

template <typename T>
void cpqr_id(const CpqrDescT<T>* descs_dev, int ndesc, int max_rows, int max_cols, int s_max,
             double tol, cudaStream_t st, bool cluster) {
  if (ndesc <= 0) return;
  int cs = 1;
  while (cs * QC_COLS < max_cols) cs *= 2;
  // the cluster form pays off while the launch holds few nodes (measured on a 512 x 512
  // ID: one node 1.95 ms on a cluster of 8 against 6.45 ms on one block; at 32 nodes
  // 5.8 against 6.5 ms; at 64 nodes 9.7 against 6.5 ms)
  if (std::is_same<T, float>::value && cluster && max_rows <= QC_MAX_ROWS && max_cols <= 8 * QC_COLS &&
      ndesc * cs <= 256) {
    ProfScope _ps(pk_of<T>(PK_CPQR), st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ndesc * cs));
    cfg.blockDim = dim3(QC_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    IA_CUDA(cudaLaunchKernelEx(&cfg, cpqr_cluster_kernel, reinterpret_cast<const CpqrDescT<float>*>(descs_dev),
                               s_max, tol));
    IA_LAUNCH_CHECK();
    return;
  }
  const size_t smem = (size_t)(2 * max_cols + max_rows) * sizeof(double);
  if (smem > 220 * 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "ID block too large for one CTA");
  ProfScope _ps(pk_of<T>(PK_CPQR), st);
  if (std::is_same<T, float>::value) {
    if (max_cols > QP_SLOTS * QR_WARPS) throw Error(IASKIT_ERR_UNSUPPORTED, "ID block wider than 1024 columns");
    const size_t smem32 = (size_t)(2 * max_cols + max_rows + (max_cols + 1) / 2 + 1) * sizeof(double) +
                          (size_t)QR_WARPS * QP_SLOTS * QP_LD * sizeof(float);
    IA_CUDA(cudaFuncSetAttribute(cpqr_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32));
    cpqr_f32_kernel<<<ndesc, QR_THREADS, smem32, st>>>(reinterpret_cast<const CpqrDescT<float>*>(descs_dev),
                                                      s_max, tol);
  } else {
    if (smem > 48 * 1024)
      IA_CUDA(cudaFuncSetAttribute(cpqr_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cpqr_kernel<double><<<ndesc, QR_THREADS, smem, st>>>(reinterpret_cast<const CpqrDescT<double>*>(descs_dev),
                                                        s_max, tol);
  }
  IA_LAUNCH_CHECK();
}

template <typename T>
void assemble_P(const PDescT<T>* descs_dev, int ndesc, int max_cols, cudaStream_t st) {
  if (ndesc <= 0) return;
  ProfScope _ps(PK_ASSEMBLE_P, st);
  dim3 grid(grid_for((int64_t)max_cols * 64, 256, 1024), ndesc);
  assemble_P_kernel<T><<<grid, 256, 0, st>>>(descs_dev, ndesc);
  IA_LAUNCH_CHECK();
}

template <typename T>
void getrf_batched(const LuDescT<T>* descs_dev, int ndesc, int max_n, int* dev_status,
                   cudaStream_t st, bool inv) {
  if (ndesc <= 0) return;
  if (max_n <= 0) return;  // every block is empty
  if (max_n > LU_MAX_N) throw Error(IASKIT_ERR_UNSUPPORTED, "LU block larger than 1024");
  ProfScope _ps(pk_of<T>(PK_GETRF), st);
  // the panel (rows x 32) in shared memory when it fits next to the static tiles
  const int pld = max_n;
  size_t smem = (size_t)pld * LU_NB * sizeof(T);
  const bool fits = smem <= 160 * 1024;
  if (!fits) smem = 0;
  // (the kernel's static tiles take up to 42 KB: the opt-in is needed for any panel)
  if (fits) {
    IA_CUDA(cudaFuncSetAttribute(getrf_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    getrf_kernel<T, true><<<ndesc, LU_THREADS, smem, st>>>(descs_dev, dev_status, pld);
  } else {
    getrf_kernel<T, false><<<ndesc, LU_THREADS, 0, st>>>(descs_dev, dev_status, 0);
  }
  IA_LAUNCH_CHECK();
  if (std::is_same<T, float>::value && inv) {
    if (max_n > 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "LU block too large for its inverse blocks");
    lu_dinv_kernel<<<ndesc, LU_THREADS, 0, st>>>(reinterpret_cast<const LuDescT<float>*>(descs_dev));
    IA_LAUNCH_CHECK();
  }
}

template <typename T>
void getrs_batched(const LuSolveDescT<T>* descs_dev, int ndesc, int max_n, int max_cols,
                   cudaStream_t st, bool inv, bool pair) {
  if (ndesc <= 0 || max_cols <= 0) return;
  ProfScope _ps(pk_of<T>(PK_GETRS), st);
  if constexpr (std::is_same<T, double>::value) {
    if (pair) {
      solve_dispatch<double, false, true>(descs_dev, ndesc, max_n, max_cols, st);
      return;
    }
  }
  if (std::is_same<T, float>::value && inv) {
    const size_t smem = (size_t)max_n * RI_LD * sizeof(float);
    if (smem > 200 * 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "LU block too large");
    if (smem > 48 * 1024)
      IA_CUDA(cudaFuncSetAttribute(getrs_inv_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (ndesc > 65535) throw Error(IASKIT_ERR_UNSUPPORTED, "more than 65535 LU solves in one launch");
    dim3 grid(ceil_div(max_cols, RI_NC), ndesc);
    getrs_inv_kernel<false><<<grid, RS_THREADS, smem, st>>>(reinterpret_cast<const LuSolveDescT<float>*>(descs_dev));
    IA_LAUNCH_CHECK();
    return;
  }
  solve_dispatch<T, false>(descs_dev, ndesc, max_n, max_cols, st);
}

void getri_batched(const LuSolveDescT<float>* descs_dev, int ndesc, int max_n, cudaStream_t st) {
  if (ndesc <= 0 || max_n <= 0) return;
  ProfScope _ps(PK_GETRI32, st);
  const size_t smem = (size_t)max_n * RI_LD * sizeof(float);
  if (smem > 200 * 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "LU block too large");
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(getrs_inv_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (ndesc > 65535) throw Error(IASKIT_ERR_UNSUPPORTED, "more than 65535 LU inverses in one launch");
  dim3 grid(ceil_div(max_n, RI_NC), ndesc);
  getrs_inv_kernel<true><<<grid, RS_THREADS, smem, st>>>(descs_dev);
  IA_LAUNCH_CHECK();
}

template <typename T>
void trsm_upper_batched(const LuSolveDescT<T>* descs_dev, int ndesc, int max_n, int max_cols,
                        cudaStream_t st) {
  if (ndesc <= 0 || max_cols <= 0 || max_n <= 0) return;
  ProfScope _ps(pk_of<T>(PK_GETRS), st);
  solve_dispatch<T, true>(descs_dev, ndesc, max_n, max_cols, st);
}

template <typename T>
void gemm_grouped(const GemmDescT<T>* descs_dev, const GemmTile* tiles_dev, int ntiles,
                  GemmShape shape, cudaStream_t st, int* dev_status) {
  if (ntiles <= 0) return;
  ProfScope _ps(pk_of<T>(PK_GEMM), st);
  if (shape == GEMM_TC) {
    if (!std::is_same<T, float>::value || !dev_status)
      throw Error(IASKIT_ERR_ARG, "tensor-core tiles are for FP32 products with a status word");
    const size_t smem = (size_t)4 * GT_M * GT_K * sizeof(uint32_t) + 64;
    IA_CUDA(cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    gemm_tc_kernel<<<ntiles, GT_THREADS, smem, st>>>(reinterpret_cast<const GemmDescT<float>*>(descs_dev),
                                                    tiles_dev, dev_status);
    IA_LAUNCH_CHECK();
    return;
  }
  if (!gemm_shape_valid(shape, sizeof(T) == 8)) throw Error(IASKIT_ERR_ARG, "tile shape not available");
  if (shape == GEMM_SKINNY)
    gemm_kernel<T, 256, 16><<<ntiles, G_THREADS, 0, st>>>(descs_dev, tiles_dev);
  else if (shape == GEMM_WIDE)
    gemm_kernel<T, 128, 32><<<ntiles, G_THREADS, 0, st>>>(descs_dev, tiles_dev);
  else if (shape == GEMM_NARROW)
    gemm_narrow<T>(descs_dev, tiles_dev, ntiles, st);
  else
    gemm_kernel<T, 64, 64><<<ntiles, G_THREADS, 0, st>>>(descs_dev, tiles_dev);
  IA_LAUNCH_CHECK();
}

template <typename T>
void copy_batched(const CopyDescT<T>* descs_dev, int ndesc, int64_t max_entries, cudaStream_t st) {
  if (ndesc <= 0) return;
  ProfScope _ps(PK_MISC, st);
  dim3 grid(grid_for(max_entries, 256, 1024), std::min(ndesc, 65535));
  copy_kernel<T><<<grid, 256, 0, st>>>(descs_dev, ndesc);
  IA_LAUNCH_CHECK();
}

template <typename T>
void form_Z(const ZDescT<T>* descs_dev, int ndesc, int64_t max_entries, cudaStream_t st) {
  if (ndesc <= 0) return;
  ProfScope _ps(PK_MISC, st);
  dim3 grid(grid_for(max_entries, 256, 1024), std::min(ndesc, 65535));
  form_Z_kernel<T><<<grid, 256, 0, st>>>(descs_dev, ndesc);
  IA_LAUNCH_CHECK();
}

template <typename T>
void permute_rows(const T* in, int ldi, T* out, int ldo, const int* perm, int N, int ncols,
                  bool scatter, cudaStream_t st) {
  ProfScope _ps(PK_MISC, st);
  permute_rows_kernel<T><<<grid_for((int64_t)N * ncols, 256, 8192), 256, 0, st>>>(
      in, ldi, out, ldo, perm, N, ncols, scatter);
  IA_LAUNCH_CHECK();
}

// ------------------------------------------------ FP64-accurate products on FP32 pairs
__global__ void split_pairs_kernel(const double* in, float2* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = in[i];
    const float hi = __double2float_rn(x);
    out[i] = make_float2(hi, __double2float_rn(x - (double)hi));  // same bytes as in[i] when aliased
  }
}
void split_pairs(const double* in, float2* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ProfScope _ps(PK_MISC, st);
  split_pairs_kernel<<<grid_for(n, 256, 8192), 256, 0, st>>>(in, out, n);
  IA_LAUNCH_CHECK();
}

constexpr int GP_K = 16;
// An A entry as a pair: stored as a pair, or split from FP64 on the way in.
__device__ __forceinline__ float2 a_pair(float2 v) { return v; }
__device__ __forceinline__ float2 a_pair(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}
template <typename DescT, int TM, int TN>
__global__ void __launch_bounds__(G_THREADS) gemm_pair_kernel(const DescT* descs, const GemmTile* tiles) {
  constexpr int TX = TM / 4;
  static_assert(TX * (TN / 4) == G_THREADS, "tile must map to 256 threads");
  __shared__ __align__(16) float Ash[GP_K][TM + 4], Asl[GP_K][TM + 4];
  __shared__ __align__(16) float Bsh[GP_K][TN + 4], Bsl[GP_K][TN + 4];
  const GemmTile Tl = tiles[blockIdx.x];
  const DescT D = descs[Tl.desc];
  const int m0 = Tl.tm * TM, n0 = Tl.tn * TN;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const bool live = m0 + 4 * tx < D.M && n0 + 4 * ty < D.N;  // some output inside C
  float s[4][4], c[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) s[a][b] = c[a][b] = 0.0f;
  for (int k0 = 0; k0 < D.K; k0 += GP_K) {
#pragma unroll
    for (int r = 0; r < TM * GP_K / G_THREADS; ++r) {
      const int e = threadIdx.x + r * G_THREADS;
      const int am = e % TM, ak = e / TM;
      const int gm = m0 + am, gk = k0 + ak;
      const float2 v = (gm < D.M && gk < D.K) ? a_pair(D.A[(size_t)gm + (size_t)gk * D.lda]) : make_float2(0.0f, 0.0f);
      Ash[ak][am] = v.x;
      Asl[ak][am] = v.y;
    }
    static_assert((TN * GP_K) % G_THREADS == 0, "whole B elements per thread");
#pragma unroll
    for (int r = 0; r < TN * GP_K / G_THREADS; ++r) {
      const int e = threadIdx.x + r * G_THREADS;
      const int bk = e % GP_K, bn = e / GP_K;
      const int gk = k0 + bk, gn = n0 + bn;
      const double b = (gk < D.K && gn < D.N) ? D.B[(size_t)gk + (size_t)gn * D.ldb] : 0.0;
      const float bh = __double2float_rn(b);
      Bsh[bk][bn] = bh;
      Bsl[bk][bn] = __double2float_rn(b - (double)bh);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < (live ? GP_K : 0); ++kk) {  // threads with no output inside C skip
      const float4 ah = *reinterpret_cast<const float4*>(&Ash[kk][4 * tx]);
      const float4 al = *reinterpret_cast<const float4*>(&Asl[kk][4 * tx]);
      const float4 bh = *reinterpret_cast<const float4*>(&Bsh[kk][4 * ty]);
      const float4 bl = *reinterpret_cast<const float4*>(&Bsl[kk][4 * ty]);
      const float ahv[4] = {ah.x, ah.y, ah.z, ah.w}, alv[4] = {al.x, al.y, al.z, al.w};
      const float bhv[4] = {bh.x, bh.y, bh.z, bh.w}, blv[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) pair_mac(ahv[r], alv[r], bhv[q], blv[q], s[r][q], c[r][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gm = m0 + 4 * tx + r, gn = n0 + 4 * ty + q;
      if (gm < D.M && gn < D.N) {
        double* cp = D.C + (size_t)gm + (size_t)gn * D.ldc;
        const double v = (double)s[r][q] + (double)c[r][q];
        *cp = D.beta == 0.0 ? D.alpha * v : D.alpha * v + D.beta * *cp;
      }
    }
}

void gemm_pair_grouped(const GemmDescPair* descs_dev, const GemmTile* tiles_dev, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return;
  ProfScope _ps(PK_GEMM_PAIR, st);
  gemm_pair_kernel<GemmDescPair, GEMM_PAIR_TM, GEMM_PAIR_TN><<<ntiles, G_THREADS, 0, st>>>(descs_dev, tiles_dev);
  IA_LAUNCH_CHECK();
}
void gemm_pair64_grouped(const GemmDesc* descs_dev, const GemmTile* tiles_dev, int ntiles, GemmShape shape,
                         cudaStream_t st) {
  if (ntiles <= 0) return;
  ProfScope _ps(PK_GEMM_PAIR, st);
  if (shape == GEMM_SKINNY)
    gemm_pair_kernel<GemmDesc, 256, 16><<<ntiles, G_THREADS, 0, st>>>(descs_dev, tiles_dev);
  else if (shape == GEMM_SQUARE)
    gemm_pair_kernel<GemmDesc, 64, 64><<<ntiles, G_THREADS, 0, st>>>(descs_dev, tiles_dev);
  else
    throw Error(IASKIT_ERR_ARG, "pair products take 256 x 16 or 64 x 64 tiles");
  IA_LAUNCH_CHECK();
}

void convert_d2f(const double* in, float* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ProfScope _ps(PK_MISC, st);
  d2f_kernel<<<grid_for(n, 256, 8192), 256, 0, st>>>(in, out, n);
  IA_LAUNCH_CHECK();
}
void convert_f2d(const float* in, double* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ProfScope _ps(PK_MISC, st);
  f2d_kernel<<<grid_for(n, 256, 8192), 256, 0, st>>>(in, out, n);
  IA_LAUNCH_CHECK();
}

void kernel_matvec(const double* Xp, const double* xnorm, int d, int nrhs, const KMatvecDesc* descs_dev,
                   int ndesc, int max_rows, cudaStream_t st) {
  if (ndesc <= 0 || max_rows <= 0) return;
  const size_t smem = (size_t)MV_TILE * (d + 1) * sizeof(double);
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(kernel_matvec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  ProfScope _ps(PK_MATVEC, st);
  dim3 grid(ceil_div(max_rows, MV_THREADS), ndesc);
  kernel_matvec_kernel<<<grid, MV_THREADS, smem, st>>>(Xp, xnorm, d, nrhs, descs_dev);
  IA_LAUNCH_CHECK();
}

// Each block sums a chunk of one sampled row in FP32 (an estimate needs no more) and
// adds it to out in FP64.
constexpr int RS_CHUNK = 8192;
__global__ void __launch_bounds__(256) kernel_rowsums_kernel(const double* Xp, int d,
                                                              const RowSumDesc* descs, double* out) {
  extern __shared__ float xi[];
  __shared__ float part[8];
  const RowSumDesc D = descs[blockIdx.y];
  const int r = blockIdx.x % KROWSUM_ROWS, chunk = blockIdx.x / KROWSUM_ROWS;
  const int j0 = chunk * RS_CHUNK;
  if (j0 >= D.N) return;
  const int j1 = min(D.N, j0 + RS_CHUNK);
  const int i = D.pbase + (int)(((int64_t)r * D.N) / KROWSUM_ROWS);
  for (int q = threadIdx.x; q < d; q += blockDim.x) xi[q] = (float)Xp[(size_t)i * d + q];
  __syncthreads();
  const float sc = (float)D.scale;
  float acc = 0.0f;
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const double* xj = Xp + (size_t)(D.pbase + j) * d;
    float d2 = 0.0f;
    if (g_kspec.poly) {  // |K| of the polynomial kernel from the dot product
      for (int q = 0; q < d; ++q) d2 = fmaf(xi[q], (float)xj[q], d2);
      acc += fabsf(kspec_pow(fmaf(d2, sc, (float)g_kspec.c), g_kspec.p));
      continue;
    }
    for (int q = 0; q < d; ++q) {
      const float t = xi[q] - (float)xj[q];
      d2 = fmaf(t, t, d2);
    }
    acc += __expf(d2 * sc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < 8; ++w) s += part[w];
    atomicAdd(&out[(size_t)blockIdx.y * KROWSUM_ROWS + r], (double)s);
  }
}

void kernel_rowsums(const double* Xp, int d, const RowSumDesc* descs_dev, int nprob, int max_n,
                    double* out, cudaStream_t st) {
  if (nprob <= 0) return;
  const size_t smem = (size_t)d * sizeof(float);
  ProfScope _ps(PK_MISC, st);
  IA_CUDA(cudaMemsetAsync(out, 0, (size_t)nprob * KROWSUM_ROWS * sizeof(double), st));
  const unsigned chunks = ceil_div(max_n, RS_CHUNK);
  kernel_rowsums_kernel<<<dim3(KROWSUM_ROWS * chunks, nprob), 256, smem, st>>>(Xp, d, descs_dev, out);
  IA_LAUNCH_CHECK();
}

void check_finite(const double* x, int64_t n, int* dev_status, cudaStream_t st) {
  if (n <= 0) return;
  ProfScope _ps(PK_MISC, st);
  check_finite_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(x, n, dev_status);
  IA_LAUNCH_CHECK();
}

#define IASKIT_INSTANTIATE(T)                                                                    \
  template void kernel_blocks<T>(const double*, const double*, int, const KDescT<T>*, int, int64_t,  \
                                 cudaStream_t);                                                  \
  template void cpqr_id<T>(const CpqrDescT<T>*, int, int, int, int, double, cudaStream_t, bool);  \
  template void assemble_P<T>(const PDescT<T>*, int, int, cudaStream_t);                          \
  template void getrf_batched<T>(const LuDescT<T>*, int, int, int*, cudaStream_t, bool);          \
  template void getrs_batched<T>(const LuSolveDescT<T>*, int, int, int, cudaStream_t, bool, bool);      \
  template void trsm_upper_batched<T>(const LuSolveDescT<T>*, int, int, int, cudaStream_t);       \
  template void gemm_grouped<T>(const GemmDescT<T>*, const GemmTile*, int, GemmShape,             \
                                cudaStream_t, int*);                                             \
  template void copy_batched<T>(const CopyDescT<T>*, int, int64_t, cudaStream_t);                 \
  template void form_Z<T>(const ZDescT<T>*, int, int64_t, cudaStream_t);                          \
  template void permute_rows<T>(const T*, int, T*, int, const int*, int, int, bool, cudaStream_t);
IASKIT_INSTANTIATE(double)
IASKIT_INSTANTIATE(float)
#undef IASKIT_INSTANTIATE

}  // namespace iaskit
