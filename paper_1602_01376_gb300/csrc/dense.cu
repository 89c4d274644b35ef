// Batched dense kernels of the factorization (FP64).
//
//  * kernel_blocks   Gaussian kernel blocks from coordinates (Sec. I, eq. gaussian):
//                    sampled blocks K(samples, columns), leaf blocks lambda I + K_aa
//                    and the U blocks K_{l r~}, K_{r l~} (eq. uv-askit).
//  * cpqr_id         column-pivoted Householder QR of a sampled block and the
//                    interpolative decomposition T = R11^{-1} R12 (Sec. II-B; GEQP3 and
//                    GELS in Sec. II-C).  Trailing column norms are recomputed from the
//                    updated block at every step; pivot ties go to the lowest column.
//  * getrf / getrs   LU with partial pivoting (ties to the lowest row) and the
//                    corresponding solve (GETRF / GETRS of Alg. "Factorize"/"Solve").
//  * gemm_grouped    C <- alpha A B + beta C over many independent small problems, the
//                    products of eqs. innerid and blocksmw.
// FP64 runs at about 2 FMA per clock per SM on this part, so these kernels are bound
// by the FP64 pipe; they keep it fed with many independent blocks.
#include <cfloat>
#include <climits>

#include "kernels.cuh"

namespace iaskit {

namespace {

// ------------------------------------------------------------ kernel blocks
__global__ void kernel_blocks_kernel(const double* Xp, int d, double neg_inv_2h2,
                                     const KDesc* descs, int ndesc) {
  for (int q = blockIdx.y; q < ndesc; q += gridDim.y) {
    const KDesc D = descs[q];
    const int64_t total = (int64_t)D.nrows * D.ncols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int i = (int)(e % D.nrows), j = (int)(e / D.nrows);
      const int r = D.rows ? D.rows[i] : D.row0 + i;
      const int c = D.colsA ? (j < D.nA ? D.colsA[j] : D.colsB[j - D.nA]) : D.col0 + j;
      const double* xr = Xp + (size_t)r * d;
      const double* xc = Xp + (size_t)c * d;
      double d2 = 0.0;
      for (int k = 0; k < d; ++k) {
        double t = xr[k] - xc[k];
        d2 = fma(t, t, d2);
      }
      double v = exp(d2 * neg_inv_2h2);
      if (r == c) v += D.diag;
      D.out[(size_t)i + (size_t)j * D.ld] = v;
    }
  }
}

// ----------------------------------------------------------------- CPQR / ID
constexpr int QR_THREADS = 256;
constexpr int QR_WARPS = QR_THREADS / 32;

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
    v = lane < QR_WARPS ? rv[lane] : -1.0;
    idx = lane < QR_WARPS ? ri[lane] : INT_MAX;
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

// One block per node.  Dynamic shared memory: norms (ncols doubles), v (nrows
// doubles), piv (ncols ints).
__global__ void __launch_bounds__(QR_THREADS) cpqr_kernel(const CpqrDesc* descs, int s_max,
                                                          double tol) {
  extern __shared__ double shq[];
  __shared__ double rv[QR_WARPS];
  __shared__ int ri[QR_WARPS];
  const CpqrDesc D = descs[blockIdx.x];
  double* A = D.A;
  const int ld = D.ld, nr = D.nrows, nc = D.ncols;
  double* norms = shq;
  double* v = shq + nc;
  int* piv = (int*)(shq + nc + nr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < nc; j += QR_WARPS) {
    double s = 0.0;
    for (int i = lane; i < nr; i += 32) {
      double a = A[(size_t)i + (size_t)j * ld];
      s = fma(a, a, s);
    }
    s = warp_sum(s);
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
        double t = A[(size_t)i + (size_t)k * ld];
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
    const double x0 = v[0];
    const double alpha = x0 >= 0.0 ? -nu : nu;
    double part = 0.0;
    for (int i = 1 + threadIdx.x; i < nr - k; i += QR_THREADS) part = fma(v[i], v[i], part);
    const double v0 = x0 - alpha;
    const double vv = block_sum(part, rv) + v0 * v0;
    if (threadIdx.x == 0) v[0] = v0;
    __syncthreads();
    const double beta = vv > 0.0 ? 2.0 / vv : 0.0;
    for (int j = k + 1 + warp; j < nc; j += QR_WARPS) {
      double* col = A + (size_t)j * ld;
      double dot = 0.0;
      for (int i = k + lane; i < nr; i += 32) dot = fma(v[i - k], col[i], dot);
      dot = warp_sum(dot);
      const double f = beta * dot;
      double nrm = 0.0;
      for (int i = k + lane; i < nr; i += 32) {
        double a = col[i] - f * v[i - k];
        col[i] = a;
        if (i > k) nrm = fma(a, a, nrm);
      }
      nrm = warp_sum(nrm);
      if (lane == 0) norms[j] = nrm;
    }
    for (int i = k + threadIdx.x; i < nr; i += QR_THREADS)
      A[(size_t)i + (size_t)k * ld] = (i == k) ? alpha : 0.0;
    s = k + 1;
    __syncthreads();
  }
  // T = R11^{-1} R12 in place, column-oriented back substitution; a zero diagonal
  // entry of R11 gives a zero row of T.
  const int nt = nc - s;
  for (int kk = s - 1; kk >= 0 && nt > 0; --kk) {
    const double rkk = A[(size_t)kk + (size_t)kk * ld];
    for (int j = threadIdx.x; j < nt; j += QR_THREADS) {
      double* a = &A[(size_t)kk + (size_t)(s + j) * ld];
      *a = (rkk == 0.0) ? 0.0 : *a / rkk;
    }
    __syncthreads();
    const int64_t items = (int64_t)kk * nt;
    for (int64_t t = threadIdx.x; t < items; t += QR_THREADS) {
      const int i = (int)(t % kk), j = s + (int)(t / kk);
      A[(size_t)i + (size_t)j * ld] -= A[(size_t)i + (size_t)kk * ld] * A[(size_t)kk + (size_t)j * ld];
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < nc; j += QR_THREADS) D.piv[j] = piv[j];
  if (threadIdx.x == 0) *D.rank = s;
}

__global__ void assemble_P_kernel(const PDesc* descs, int ndesc) {
  const PDesc D = descs[blockIdx.y];
  const int64_t total = (int64_t)D.s * D.ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % D.s), jj = (int)(e / D.s);
    const int col = D.piv[jj];
    const double val = jj < D.s ? (r == jj ? 1.0 : 0.0) : D.A[(size_t)r + (size_t)jj * D.ld];
    D.P[(size_t)r + (size_t)col * D.s] = val;
    if (r == 0 && jj < D.s)
      D.skel[jj] = D.colsA ? (col < D.nA ? D.colsA[col] : D.colsB[col - D.nA]) : D.col0 + col;
  }
}

// ---------------------------------------------------------------- LU (GETRF)
constexpr int LU_THREADS = 256;

__global__ void __launch_bounds__(LU_THREADS) getrf_kernel(const LuDesc* descs, int* status) {
  __shared__ double rv[LU_THREADS / 32];
  __shared__ int ri[LU_THREADS / 32];
  const LuDesc D = descs[blockIdx.x];
  double* A = D.A;
  const int n = D.n, ld = D.ld;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = INT_MAX;
    for (int i = k + threadIdx.x; i < n; i += LU_THREADS)
      argmax_merge(best, bi, fabs(A[(size_t)i + (size_t)k * ld]), i);
    warp_argmax(best, bi);
    __syncthreads();
    if (lane == 0) {
      rv[warp] = best;
      ri[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
      best = lane < LU_THREADS / 32 ? rv[lane] : -1.0;
      bi = lane < LU_THREADS / 32 ? ri[lane] : INT_MAX;
      warp_argmax(best, bi);
      if (lane == 0) {
        rv[0] = best;
        ri[0] = bi;
      }
    }
    __syncthreads();
    const int p = ri[0];
    if (threadIdx.x == 0) D.ipiv[k] = p;
    if (p != k)
      for (int j = threadIdx.x; j < n; j += LU_THREADS) {
        double t = A[(size_t)k + (size_t)j * ld];
        A[(size_t)k + (size_t)j * ld] = A[(size_t)p + (size_t)j * ld];
        A[(size_t)p + (size_t)j * ld] = t;
      }
    __syncthreads();
    const double piv = A[(size_t)k + (size_t)k * ld];
    if (piv == 0.0) {
      if (threadIdx.x == 0) atomicOr(status, DEV_SINGULAR);
      continue;
    }
    for (int i = k + 1 + threadIdx.x; i < n; i += LU_THREADS) A[(size_t)i + (size_t)k * ld] /= piv;
    __syncthreads();
    const int m = n - k - 1;
    const int64_t items = (int64_t)m * m;
    for (int64_t t = threadIdx.x; t < items; t += LU_THREADS) {
      const int i = k + 1 + (int)(t % m), j = k + 1 + (int)(t / m);
      A[(size_t)i + (size_t)j * ld] -= A[(size_t)i + (size_t)k * ld] * A[(size_t)k + (size_t)j * ld];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- GETRS
constexpr int RS_THREADS = 256;

// Grid: (descriptor, column chunk).  Dynamic shared memory: n * cc doubles.
__global__ void __launch_bounds__(RS_THREADS) getrs_kernel(const LuSolveDesc* descs, int cc) {
  extern __shared__ double X[];
  const LuSolveDesc D = descs[blockIdx.x];
  const int c0 = blockIdx.y * cc;
  if (c0 >= D.ncols) return;
  const int nc = min(cc, D.ncols - c0);
  const int n = D.n;
  const double* LU = D.LU;
  const int ld = D.ldlu;
  for (int64_t t = threadIdx.x; t < (int64_t)n * nc; t += RS_THREADS) {
    const int i = (int)(t % n), c = (int)(t / n);
    X[(size_t)c * n + i] = D.B[(size_t)i + (size_t)(c0 + c) * D.ldb];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nc; c += RS_THREADS) {
    double* x = X + (size_t)c * n;
    for (int k = 0; k < n; ++k) {
      const int p = D.ipiv[k];
      if (p != k) {
        double t = x[k];
        x[k] = x[p];
        x[p] = t;
      }
    }
  }
  __syncthreads();
  for (int k = 0; k < n - 1; ++k) {  // unit lower triangle
    const int m = n - k - 1;
    for (int t = threadIdx.x; t < m * nc; t += RS_THREADS) {
      const int i = k + 1 + t % m, c = t / m;
      X[(size_t)c * n + i] -= LU[(size_t)i + (size_t)k * ld] * X[(size_t)c * n + k];
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {  // upper triangle
    const double ukk = LU[(size_t)k + (size_t)k * ld];
    for (int c = threadIdx.x; c < nc; c += RS_THREADS) X[(size_t)c * n + k] /= ukk;
    __syncthreads();
    for (int t = threadIdx.x; t < k * nc; t += RS_THREADS) {
      const int i = t % k, c = t / k;
      X[(size_t)c * n + i] -= LU[(size_t)i + (size_t)k * ld] * X[(size_t)c * n + k];
    }
    __syncthreads();
  }
  for (int64_t t = threadIdx.x; t < (int64_t)n * nc; t += RS_THREADS) {
    const int i = (int)(t % n), c = (int)(t / n);
    D.B[(size_t)i + (size_t)(c0 + c) * D.ldb] = X[(size_t)c * n + i];
  }
}

// ---------------------------------------------------------------- GEMM
constexpr int GT = 64;   // tile
constexpr int GK = 16;   // k step
constexpr int G_THREADS = 256;

__global__ void __launch_bounds__(G_THREADS) gemm_kernel(const GemmDesc* descs,
                                                         const GemmTile* tiles) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const GemmTile T = tiles[blockIdx.x];
  const GemmDesc D = descs[T.desc];
  const int m0 = T.tm * GT, n0 = T.tn * GT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < D.K; k0 += GK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = threadIdx.x + r * G_THREADS;  // 0 .. 1023
      const int am = e % GT, ak = e / GT;         // A tile: 64 rows x 16 k
      const int gm = m0 + am, gk = k0 + ak;
      As[ak][am] = (gm < D.M && gk < D.K) ? D.A[(size_t)gm + (size_t)gk * D.lda] : 0.0;
      const int bk = e % GK, bn = e / GK;         // B tile: 16 k x 64 cols
      const int gk2 = k0 + bk, gn = n0 + bn;
      Bs[bk][bn] = (gk2 < D.K && gn < D.N) ? D.B[(size_t)gk2 + (size_t)gn * D.ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        a[r] = As[kk][tx + 16 * r];
        b[r] = Bs[kk][ty + 16 * r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gm = m0 + tx + 16 * r, gn = n0 + ty + 16 * c;
      if (gm < D.M && gn < D.N) {
        double* cp = D.C + (size_t)gm + (size_t)gn * D.ldc;
        *cp = D.beta == 0.0 ? D.alpha * acc[r][c] : D.alpha * acc[r][c] + D.beta * *cp;
      }
    }
}

// ---------------------------------------------------------------- small helpers
__global__ void copy_kernel(const CopyDesc* descs, int ndesc) {
  for (int q = blockIdx.y; q < ndesc; q += gridDim.y) {
    const CopyDesc D = descs[q];
    const int64_t total = (int64_t)D.rows * D.cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int i = (int)(e % D.rows), j = (int)(e / D.rows);
      D.dst[(size_t)i + (size_t)j * D.ldd] = D.src[(size_t)i + (size_t)j * D.lds];
    }
  }
}

__global__ void form_Z_kernel(const ZDesc* descs, int ndesc) {
  for (int q = blockIdx.y; q < ndesc; q += gridDim.y) {
    const ZDesc D = descs[q];
    const int n = D.sl + D.sr;
    const int64_t total = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int i = (int)(e % n), j = (int)(e / n);
      double v;
      if (i < D.sl && j < D.sl) v = (i == j) ? 1.0 : 0.0;
      else if (i >= D.sl && j >= D.sl) v = (i == j) ? 1.0 : 0.0;
      else if (i < D.sl) v = D.Cl[(size_t)i + (size_t)(j - D.sl) * D.sl];
      else v = D.Cr[(size_t)(i - D.sl) + (size_t)j * D.sr];
      D.Z[(size_t)i + (size_t)j * n] = v;
    }
  }
}

__global__ void permute_rows_kernel(const double* in, int ldi, double* out, int ldo,
                                    const int* perm, int N, int ncols, bool scatter) {
  const int64_t total = (int64_t)N * ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e % N), c = (int)(e / N);
    if (scatter) out[(size_t)perm[p] + (size_t)c * ldo] = in[(size_t)p + (size_t)c * ldi];
    else out[(size_t)p + (size_t)c * ldo] = in[(size_t)perm[p] + (size_t)c * ldi];
  }
}

// u_rows += K(x_rows, x_cols) y, one thread per target row, up to MV_R right-hand
// sides per pass; the column points are staged in shared memory.
constexpr int MV_THREADS = 128;
constexpr int MV_R = 16;
constexpr int MV_TILE = 32;
__global__ void __launch_bounds__(MV_THREADS) kernel_matvec_kernel(const double* Xp, int d,
                                                                   double neg_inv_2h2, int nrhs,
                                                                   const KMatvecDesc* descs) {
  extern __shared__ double xs[];  // MV_TILE x d
  const KMatvecDesc D = descs[blockIdx.y];
  const int i = blockIdx.x * MV_THREADS + threadIdx.x;
  const bool active = i < D.nrows;
  const int row = D.row0 + (active ? i : 0);
  const double* xr = Xp + (size_t)row * d;
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
      __syncthreads();
      if (!active) continue;
      for (int kk = 0; kk < nt; ++kk) {
        double d2 = 0.0;
        for (int q = 0; q < d; ++q) {
          double t = xr[q] - xs[kk * d + q];
          d2 = fma(t, t, d2);
        }
        const double kv = exp(d2 * neg_inv_2h2);
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

}  // namespace

void kernel_blocks(const double* Xp, int d, double h, const KDesc* descs_dev, int ndesc,
                   int64_t max_entries, cudaStream_t st) {
  if (ndesc <= 0) return;
  dim3 grid(grid_for(max_entries, 256, 4096), std::min(ndesc, 65535));
  ProfScope _ps(PK_KBLOCK, st);
  kernel_blocks_kernel<<<grid, 256, 0, st>>>(Xp, d, -1.0 / (2.0 * h * h), descs_dev, ndesc);
  IA_LAUNCH_CHECK();
}

void cpqr_id(const CpqrDesc* descs_dev, int ndesc, int max_rows, int max_cols, int s_max,
             double tol, cudaStream_t st) {
  if (ndesc <= 0) return;
  const size_t smem = (size_t)(2 * max_cols + max_rows) * sizeof(double);
  if (smem > 220 * 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "ID block too large for one CTA");
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(cpqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope _ps(PK_CPQR, st);
  cpqr_kernel<<<ndesc, QR_THREADS, smem, st>>>(descs_dev, s_max, tol);
  IA_LAUNCH_CHECK();
}

void assemble_P(const PDesc* descs_dev, int ndesc, int max_cols, cudaStream_t st) {
  if (ndesc <= 0) return;
  dim3 grid(grid_for((int64_t)max_cols * 64, 256, 1024), ndesc);
  ProfScope _ps(PK_ASSEMBLE_P, st);
  assemble_P_kernel<<<grid, 256, 0, st>>>(descs_dev, ndesc);
  IA_LAUNCH_CHECK();
}

void getrf_batched(const LuDesc* descs_dev, int ndesc, int max_n, int* dev_status, cudaStream_t st) {
  if (ndesc <= 0) return;
  (void)max_n;
  ProfScope _ps(PK_GETRF, st);
  getrf_kernel<<<ndesc, LU_THREADS, 0, st>>>(descs_dev, dev_status);
  IA_LAUNCH_CHECK();
}

void getrs_batched(const LuSolveDesc* descs_dev, int ndesc, int max_n, int max_cols,
                   cudaStream_t st) {
  if (ndesc <= 0 || max_cols <= 0) return;
  int cc = std::max(1, std::min(max_cols, (int)(16384 / std::max(1, max_n))));
  const size_t smem = (size_t)max_n * cc * sizeof(double);
  if (smem > 220 * 1024) throw Error(IASKIT_ERR_UNSUPPORTED, "LU block too large");
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(getrs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid(ndesc, ceil_div(max_cols, cc));
  ProfScope _ps(PK_GETRS, st);
  getrs_kernel<<<grid, RS_THREADS, smem, st>>>(descs_dev, cc);
  IA_LAUNCH_CHECK();
}

void gemm_grouped(const GemmDesc* descs_dev, const GemmTile* tiles_dev, int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return;
  ProfScope _ps(PK_GEMM, st);
  gemm_kernel<<<ntiles, G_THREADS, 0, st>>>(descs_dev, tiles_dev);
  IA_LAUNCH_CHECK();
}

void copy_batched(const CopyDesc* descs_dev, int ndesc, int64_t max_entries, cudaStream_t st) {
  if (ndesc <= 0) return;
  dim3 grid(grid_for(max_entries, 256, 1024), std::min(ndesc, 65535));
  ProfScope _ps(PK_MISC, st);
  copy_kernel<<<grid, 256, 0, st>>>(descs_dev, ndesc);
  IA_LAUNCH_CHECK();
}

void form_Z(const ZDesc* descs_dev, int ndesc, int64_t max_entries, cudaStream_t st) {
  if (ndesc <= 0) return;
  dim3 grid(grid_for(max_entries, 256, 1024), std::min(ndesc, 65535));
  ProfScope _ps(PK_MISC, st);
  form_Z_kernel<<<grid, 256, 0, st>>>(descs_dev, ndesc);
  IA_LAUNCH_CHECK();
}

void permute_rows(const double* in, int ldi, double* out, int ldo, const int* perm, int N,
                  int ncols, bool scatter, cudaStream_t st) {
  ProfScope _ps(PK_MISC, st);
  permute_rows_kernel<<<grid_for((int64_t)N * ncols, 256, 8192), 256, 0, st>>>(in, ldi, out, ldo,
                                                                               perm, N, ncols,
                                                                               scatter);
  IA_LAUNCH_CHECK();
}

void kernel_matvec(const double* Xp, int d, double h, int nrhs, const KMatvecDesc* descs_dev,
                   int ndesc, int max_rows, cudaStream_t st) {
  if (ndesc <= 0 || max_rows <= 0) return;
  const size_t smem = (size_t)MV_TILE * d * sizeof(double);
  if (smem > 48 * 1024)
    IA_CUDA(cudaFuncSetAttribute(kernel_matvec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  dim3 grid(ceil_div(max_rows, MV_THREADS), ndesc);
  ProfScope _ps(PK_MATVEC, st);
  kernel_matvec_kernel<<<grid, MV_THREADS, smem, st>>>(Xp, d, -1.0 / (2.0 * h * h), nrhs, descs_dev);
  IA_LAUNCH_CHECK();
}

void check_finite(const double* x, int64_t n, int* dev_status, cudaStream_t st) {
  if (n <= 0) return;
  ProfScope _ps(PK_MISC, st);
  check_finite_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(x, n, dev_status);
  IA_LAUNCH_CHECK();
}

}  // namespace iaskit
