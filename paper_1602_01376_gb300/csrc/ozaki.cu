// FP64 operator products on the BF16 tensor cores by exact slicing (Ozaki, Ogita,
// Oishi and Rump's error-free splitting of a matrix product into products of short
// slices, 2012).  GB300 runs FP64 arithmetic at 1/64 of its FP32 rate, so the refinement's
// operator apply u += K_{c s~} w~ (Evaluate of Sec. II-B, stored blocks of the mixed
// form) is bound by the FP64 pipe; here every FP64 value is split into OZ_S signed 8-bit
// digits that BF16 holds exactly, the digit products run as exact FP32 sums on the
// tensor cores, and the sums are recombined in integers and FP64.
//
// Splitting.  A row r of a block gets the exponent E_r of its largest |a_rk| (so that
// |a_rk| 2^-E_r < 1) and a_rk = 2^E_r sum_i A_i[r, k] 2^(-7 - 8 i) + e with OZ_S = 8
// integer digits |A_i| <= 128 and |e| <= 2^(E_r - 64); a column c of the right-hand sides
// gets F_c and digits W_j the same way.  Then
//     sum_k a_rk w_kc ~ 2^(E_r + F_c - 14) sum_{t=0}^{OZ_S-1} 2^(-8 t) S_t,
//     S_t = sum_{i+j=t} sum_k A_i[r, k] W_j[k, c],
// the products with i + j >= OZ_S dropped (each below 2^-64 of max|a| max|w| per term).
// Every S_t is an integer of magnitude <= 8 * 128 * 2^14 = 2^24 over 128 values of k, so
// an FP32 accumulator holds it exactly: the tensor core accumulates the diagonal t of a
// 128-wide segment of k in one set of TMEM columns (the MMA of digit i of A writes its
// product with [W_0 .. W_{OZ_S-1-i}] starting at diagonal i), and the epilogue adds the
// segments in 64-bit integers.  The truncation errors, about 2^-60 K max|a| max|w| per
// entry, lie below an FP64 product's rounding (2^-53 sum |a| |w|) unless a row's or a
// column's entries span more than 2^7; 7 digits (2^-52 K max|a| max|w|) measurably
// raised the refinement's floor on C4 (1.06e-10 against 3.1e-11).
//
// Records.  A block's digits are stored once per factorization as 128-row tiles of
// 16-column chunks, each chunk the OZ_S operands of one MMA step in the tensor core's
// K-major layout (8-row x 16-byte core matrices), so that one bulk copy brings a chunk
// into shared memory; a block of right-hand sides is split per apply into the matching
// B operands (OZ_S * 16 rows: digit j of column c is row 16 j + c).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.cuh"
#include "tc.cuh"

namespace iaskit {

namespace {

constexpr int OZ_NS = 3;                       // pipeline stages (chunks in flight)
constexpr int OZ_STAGE = OZ_AREC + OZ_BREC;    // bytes of one stage
constexpr int OZ_SEGC = 8;                     // chunks of one exact segment (k = 128)
constexpr int OZ_TCOLS = 256;                  // TMEM columns: two accumulators of OZ_S x 16
constexpr int OZ_HI = 4;                       // diagonals summed into the high 64-bit word
constexpr int OZ_ABUF = 128;                   // column distance of the two accumulators
constexpr long OZ_WAIT = 1L << 22;             // bound of every mbarrier wait (try_wait calls)
constexpr int OZ_THREADS = 160;                // warps 0-3: epilogue (TMEM lanes), warp 4: issue

static_assert(OZ_S * OZ_NR <= OZ_ABUF, "an accumulator holds OZ_S diagonals of 16 columns");
static_assert((long long)OZ_S * OZ_SEGC * OZ_KC * 128 * 128 <= (1ll << 24),
              "a diagonal's sum over one segment stays within FP32's exact integers");
static_assert(OZ_S > OZ_HI && 8 * OZ_S - 1 <= 63, "digits of a 64-bit fixed-point value");

// Digits of a (|a| < 2^E): a = 2^E sum_i dg[i] 2^(-7 - 8 i) + e, |dg[i]| <= 128,
// |e| <= 2^(E - 8 OZ_S).  V = round(|a| 2^(8 OZ_S - 1 - E)) <= 2^(8 OZ_S - 1) from the
// FP64 fields, then signed base-256 digits from the lowest.
__device__ __forceinline__ void oz_digits(double a, int E, int (&dg)[OZ_S]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
  int ex = (int)((bits >> 52) & 0x7FF);
  unsigned long long M = bits & ((1ull << 52) - 1);
  if (ex) M |= 1ull << 52;
  else ex = 1;
  const int shift = ex - 1075 + 8 * OZ_S - 1 - E;  // V = M 2^shift
  unsigned long long V;
  if (M == 0) V = 0;
  else if (shift >= 0) V = M << shift;
  else if (-shift >= 64) V = 0;
  else V = ((M >> (-shift - 1)) + 1) >> 1;  // round half up
#pragma unroll
  for (int i = OZ_S - 1; i >= 1; --i) {
    int d = (int)(V & 255u);
    if (d >= 128) d -= 256;
    dg[i] = d;
    V = (V - (unsigned long long)(long long)d) >> 8;
  }
  dg[0] = (int)V;
  if (bits >> 63)
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) dg[i] = -dg[i];
}

// BF16 bits of a small integer (|d| <= 256: the FP32 value's low 16 bits are zero)
__device__ __forceinline__ uint32_t oz_bf16(int d) { return __float_as_uint((float)d) >> 16; }

// Byte offset of (row n, column k) of a K-major 16-column operand chunk
__device__ __forceinline__ uint32_t oz_off(int n, int k) {
  return (uint32_t)((n >> 3) * 256 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2);
}

template <typename Desc>
__device__ __forceinline__ int oz_find(const Desc* d, int nd, int b) {
  int lo = 0, hi = nd - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d[mid].tile0 <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One block per 128-row tile: row exponents, then the digits of 8 columns at a time,
// each written as one 16-byte core-matrix row per digit.
__global__ void __launch_bounds__(OZ_TM) oz_split_kernel(const OzSplitDesc* descs, int nd) {
  const OzSplitDesc D = descs[oz_find(descs, nd, (int)blockIdx.x)];
  const int t = (int)blockIdx.x - D.tile0;
  const int r = t * OZ_TM + (int)threadIdx.x;
  const bool valid = r < D.rows;
  const double* src = D.src + (valid ? r : 0);
  double mx = 0.0;
  if (valid)
    for (int k = 0; k < D.cols; ++k) mx = fmax(mx, fabs(src[(size_t)k * D.ld]));
  int E = 0;
  if (mx > 0.0) frexp(mx, &E);
  if (valid) D.rexp[r] = E;
  const int nch = (D.cols + OZ_KC - 1) / OZ_KC;
  unsigned char* base = D.rec + (size_t)t * nch * OZ_AREC + oz_off((int)threadIdx.x, 0);
  for (int h = 0; h < 2 * nch; ++h) {
    uint32_t pk[OZ_S][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = h * 8 + 2 * q;
      int d0[OZ_S], d1[OZ_S];
      oz_digits(valid && k < D.cols ? src[(size_t)k * D.ld] : 0.0, E, d0);
      oz_digits(valid && k + 1 < D.cols ? src[(size_t)(k + 1) * D.ld] : 0.0, E, d1);
#pragma unroll
      for (int i = 0; i < OZ_S; ++i) pk[i][q] = oz_bf16(d0[i]) | (oz_bf16(d1[i]) << 16);
    }
    unsigned char* dst = base + (size_t)(h >> 1) * OZ_AREC + (h & 1) * 128;
#pragma unroll
    for (int i = 0; i < OZ_S; ++i)
      *reinterpret_cast<uint4*>(dst + i * (OZ_TM * OZ_KC * 2)) = make_uint4(pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
  }
}

// One block per right-hand-side block: column exponents (8 threads per column), then
// the digits of 8 values of one column at a time (columns >= nrhs are zero).
__global__ void __launch_bounds__(128) oz_vec_kernel(const OzVecDesc* descs) {
  const OzVecDesc D = descs[blockIdx.x];
  __shared__ int Fs[OZ_NR];
  const int tid = (int)threadIdx.x, c = tid >> 3, sub = tid & 7;
  double mx = 0.0;
  if (c < D.nrhs)
    for (int k = sub; k < D.K; k += 8) mx = fmax(mx, fabs(D.w[(size_t)k + (size_t)c * D.ldw]));
#pragma unroll
  for (int o = 4; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int F = 0;
  if (mx > 0.0) frexp(mx, &F);
  if (sub == 0) {
    Fs[c] = F;
    D.cexp[c] = F;
  }
  __syncthreads();
  const int nch = (D.K + OZ_KC - 1) / OZ_KC;
  for (int u = tid; u < nch * 2 * OZ_NR; u += 128) {
    const int cc = u % OZ_NR, h = u / OZ_NR;
    const bool live = cc < D.nrhs;
    const int Fc = Fs[cc];
    const double* col = D.w + (size_t)(live ? cc : 0) * D.ldw;
    uint32_t pk[OZ_S][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = h * 8 + 2 * q;
      int d0[OZ_S], d1[OZ_S];
      oz_digits(live && k < D.K ? col[k] : 0.0, Fc, d0);
      oz_digits(live && k + 1 < D.K ? col[k + 1] : 0.0, Fc, d1);
#pragma unroll
      for (int i = 0; i < OZ_S; ++i) pk[i][q] = oz_bf16(d0[i]) | (oz_bf16(d1[i]) << 16);
    }
    unsigned char* dst = D.rec + (size_t)(h >> 1) * OZ_BREC;
#pragma unroll
    for (int i = 0; i < OZ_S; ++i)
      *reinterpret_cast<uint4*>(dst + oz_off(i * OZ_NR + cc, (h & 1) * 8)) =
          make_uint4(pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
  }
}

// One block per 128-row tile of a block: warp 4 (one thread) brings the chunks in by
// bulk copy (OZ_NS stages) and issues OZ_S MMAs per chunk into the accumulator of the
// chunk's segment (two accumulators alternate); warps 0-3 read a finished segment's
// diagonals from TMEM (lane = row), convert them to integers and add them into 64-bit
// sums, and at the end add 2^(E_r + F_c - 14) sum_t 2^(-8 t) S_t into the output (or
// write it).  Every
// wait is bounded; a wait that gives up sets DEV_TIMEOUT, the issuing thread stops,
// waits (bounded) for its MMAs and copies in flight, and the block frees its TMEM.
__global__ void __launch_bounds__(OZ_THREADS, 2) oz_apply_kernel(const OzApplyDesc* descs, int nd, int* status) {
  extern __shared__ __align__(1024) unsigned char oz_sh[];
  __shared__ uint64_t full[OZ_NS], empty[OZ_NS], segfull[2], epidone[2], fin;
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_s;
  const int tid = (int)threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const OzApplyDesc D = descs[oz_find(descs, nd, (int)blockIdx.x)];
  const int t = (int)blockIdx.x - D.tile0;
  const int nch = D.nch, nseg = (nch + OZ_SEGC - 1) / OZ_SEGC;
  if (warp == 0) tc::tmem_alloc(&tslot, OZ_TCOLS);
  if (tid == 0) {
    for (int s = 0; s < OZ_NS; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&segfull[b], 1);
      tc::mbar_init(&epidone[b], 4 * 32);
    }
    tc::mbar_init(&fin, 1);
    abort_s = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  if (warp == 4) {
    if (lane == 0) {
      const unsigned char* arec = D.arec + (size_t)t * nch * OZ_AREC;
      auto load = [&](int c) {
        const int s = c % OZ_NS;
        unsigned char* dst = oz_sh + s * OZ_STAGE;
        tc::mbar_expect_tx(&full[s], OZ_STAGE);
        tc::bulk_g2s(dst, arec + (size_t)c * OZ_AREC, OZ_AREC, &full[s]);
        tc::bulk_g2s(dst + OZ_AREC, D.brec + (size_t)c * OZ_BREC, OZ_BREC, &full[s]);
      };
      int loaded = 0, issued = 0;
      bool ok = true;
      for (; loaded < min(OZ_NS, nch); ++loaded) load(loaded);
      for (int c = 0; c < nch; ++c) {
        const int s = c % OZ_NS, seg = c / OZ_SEGC, buf = seg & 1, kc = c % OZ_SEGC;
        ok = tc::mbar_wait(&full[s], (uint32_t)((c / OZ_NS) & 1), OZ_WAIT);
        if (ok && kc == 0 && seg >= 2)  // the epilogue has read this accumulator's segment seg - 2
          ok = tc::mbar_wait(&epidone[buf], (uint32_t)(((seg >> 1) - 1) & 1), OZ_WAIT);
        if (!ok) break;
        tc::fence_after_sync();
        const uint32_t sa = tc::smem_addr(oz_sh + s * OZ_STAGE);
        const uint64_t bdesc = tc::smem_desc(sa + OZ_AREC, 128, 256);
#pragma unroll
        for (int i = 0; i < OZ_S; ++i) {
          const uint64_t adesc = tc::smem_desc(sa + (uint32_t)(i * OZ_TM * OZ_KC * 2), 128, 256);
          tc::mma_f16(tmem + (uint32_t)(buf * OZ_ABUF + i * OZ_NR), adesc, bdesc,
                      tc::idesc_bf16(OZ_TM, (OZ_S - i) * OZ_NR), !(kc == 0 && i == 0));
        }
        tc::mma_commit(&empty[s]);
        issued = c + 1;
        if (kc == OZ_SEGC - 1 || c == nch - 1) tc::mma_commit(&segfull[buf]);
        if (c >= 1 && c - 1 + OZ_NS < nch) {  // chunk c - 1's MMAs release its stage
          ok = tc::mbar_wait(&empty[(c - 1) % OZ_NS], (uint32_t)(((c - 1) / OZ_NS) & 1), OZ_WAIT);
          if (!ok) break;
          load(c - 1 + OZ_NS);
          ++loaded;
        }
      }
      if (!ok) {
        atomicOr(status, DEV_TIMEOUT);
        abort_s = 1;
        tc::mma_commit(&fin);  // every MMA issued so far, then the copies not yet seen complete
        tc::mbar_wait(&fin, 0, OZ_WAIT);
        for (int c = issued; c < loaded; ++c)
          if (!tc::mbar_wait(&full[c % OZ_NS], (uint32_t)((c / OZ_NS) & 1), OZ_WAIT)) break;
      }
    }
  } else {
    long long hi[OZ_NR], lo[OZ_NR];
#pragma unroll
    for (int c = 0; c < OZ_NR; ++c) hi[c] = lo[c] = 0;
    bool good = true;
    for (int seg = 0; seg < nseg; ++seg) {
      const int buf = seg & 1;
      bool got = false;
      for (long it = 0; it < OZ_WAIT && !got; it += 64) {
        got = tc::mbar_wait(&segfull[buf], (uint32_t)((seg >> 1) & 1), 64);
        if (abort_s) break;
      }
      got = __all_sync(0xffffffffu, got) != 0;  // tcgen05.ld needs the whole warp
      if (!got) {
        if (lane == 0) atomicOr(status, DEV_TIMEOUT);
        abort_s = 1;
        good = false;
        break;
      }
      tc::fence_after_sync();
#pragma unroll
      for (int q = 0; q < OZ_S; ++q) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * OZ_ABUF + q * OZ_NR), v);
#pragma unroll
        for (int c = 0; c < OZ_NR; ++c) {
          const long long s = (long long)__float2int_rn(v[c]);
          if (q < OZ_HI) hi[c] += s * (1ll << (8 * (OZ_HI - 1 - q)));
          else lo[c] += s * (1ll << (8 * (OZ_S - 1 - q)));
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(&epidone[buf]);
    }
    const int row = t * OZ_TM + warp * 32 + lane;
    if (good && row < D.rows) {
      const int E = D.rexp[row];
#pragma unroll
      for (int c = 0; c < OZ_NR; ++c)
        if (c < D.nrhs) {
          const int e = E + D.cexp[c];
          double* o = D.out + (size_t)row + (size_t)c * D.ldo;
          const double y = ldexp((double)hi[c], e - 14 - 8 * (OZ_HI - 1)) +
                           ldexp((double)lo[c], e - 14 - 8 * (OZ_S - 1));
          *o = D.add ? *o + y : y;
        }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_free(tmem, OZ_TCOLS);
}

// ------------------------------------------------------------ kernel blocks
// Gaussian kernel blocks K_ij = exp(-(|x_i|^2 + |y_j|^2 - 2 x_i.y_j) / (2 h^2)) (+ diag on
// the diagonal) with the dot products x_i.y_j on the tensor cores: every point's
// coordinates are split once into OZ_S digits under the point's own power of two (the
// same splitting as above, here with K = the dimension, at most 64, so a diagonal sums at
// most 8 * 64 products of 2^14 and stays exact), and the Gram form, exp and the diagonal
// shift run in FP64 on the dot products recombined from the diagonals.  The dot product's
// error, about 2^-60 d max|x_i| max|y_j|, is below the Gram form's own cancellation
// error 2^-52 (|x_i|^2 + |y_j|^2).

// Point digits: XE[p] = exponent of the point's largest |coordinate|, XD[(p OZ_S + i) DP
// + k] = digit i of coordinate k (zero for k >= d).  DP / 8 threads per point.
__global__ void oz_points_kernel(const double* X, int N, int d, int DP, uint16_t* XD, int* XE) {
  const int g = DP / 8;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long p = e / g;
  const int kq = (int)(e % g);
  const bool valid = p < N;
  double mx = 0.0;
  if (valid)
    for (int k = kq * 8; k < min(d, kq * 8 + 8); ++k) mx = fmax(mx, fabs(X[(size_t)p * d + k]));
  for (int o = g / 2; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int E = 0;
  if (mx > 0.0) frexp(mx, &E);
  if (!valid) return;
  if (kq == 0) XE[p] = E;
  uint32_t pk[OZ_S][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = kq * 8 + 2 * q;
    int d0[OZ_S], d1[OZ_S];
    oz_digits(k < d ? X[(size_t)p * d + k] : 0.0, E, d0);
    oz_digits(k + 1 < d ? X[(size_t)p * d + k + 1] : 0.0, E, d1);
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) pk[i][q] = oz_bf16(d0[i]) | (oz_bf16(d1[i]) << 16);
  }
#pragma unroll
  for (int i = 0; i < OZ_S; ++i)
    *reinterpret_cast<uint4*>(XD + ((size_t)p * OZ_S + i) * DP + kq * 8) =
        make_uint4(pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
}

constexpr int OZK_TC = 32;        // columns per tile: OZ_S digits x 32 = 256 B-operand rows
constexpr int OZK_THREADS = 256;  // 8 warps: warp w reads TMEM lanes 32 (w % 4), columns 16 (w / 4)
constexpr long OZK_WAIT = 1L << 22;
constexpr double OZ_LO_SCALE = 1.0 / (double)(1ull << (8 * (OZ_S - OZ_HI)));  // lo's weight against hi

__device__ __forceinline__ double oz_pow2(int e) {
  return (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52) : ldexp(1.0, e);
}

// exp(x) for x <= 0 by Tang's table-driven method (ACM TOMS 15(2), 1989): x = (256 m + j)
// ln2 / 256 + r with |r| <= ln2 / 512 (Cody and Waite's two-part reduction: L_hi has its
// 18 low bits clear, so that n L_hi is exact for |n| < 2^18), exp(x) = 2^m 2^(j/256)
// (1 + p(r)), p the Taylor polynomial of e^r - 1 to degree 4 (truncation r^5 / 120 <
// 2^-54 relative).  n is rounded by adding 1.5 * 2^52 (the sum's low bits hold n in two's
// complement), which takes the place of a multiply, a rounding and a conversion on the
// FP64 pipe.  The 256 values 2^(j/256), rounded to FP64 from extended precision, and the
// constants come from the host (OzExp).  About 1 ulp in all; arguments below -708
// (results near the subnormal range) take the library's exp.
constexpr int OZ_EXP_J = 256;
struct OzExp {
  double T[OZ_EXP_J];
  double inv_l, l_hi, l_lo;  // 256 / ln2, and ln2 / 256 = l_hi + l_lo
};
__device__ __forceinline__ double oz_exp_neg(double x, const double* T, double inv_l, double l_hi, double l_lo) {
  if (x < -708.0) return exp(x);
  constexpr double SHIFT = 6755399441055744.0;  // 1.5 * 2^52
  const double ts = fma(x, inv_l, SHIFT);      // n = nearest integer to x / (ln2 / 256)
  const int n = __double2loint(ts);
  const double nf = ts - SHIFT;
  double r = fma(-nf, l_hi, x);
  r = fma(-nf, l_lo, r);
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  const double p = fma(r * r, q, r);
  const double t = T[n & (OZ_EXP_J - 1)];
  return fma(t, p, t) * __longlong_as_double((long long)((n >> 8) + 1023) << 52);
}

// One block per 128-row tile of a descriptor (rows row0 + i, consecutive points): the
// tile's digits stay in shared memory (A: OZ_S operands of 128 x DP); per tile of 32
// columns the columns' digits are gathered (B: OZ_S * 32 rows, digit j of column c at row
// 32 j + c) and one thread issues OZ_S MMAs per 16 coordinates into one of two TMEM
// accumulators, so that the MMAs of tile c + 1 run while all threads finish tile c.
template <int DP>
__global__ void __launch_bounds__(OZK_THREADS, 1) oz_kblock_kernel(const uint16_t* XD, const int* XE, const double* xn,
                                                                   const OzKDesc* descs, int nd, int* status,
                                                                   const OzExp ex) {
  extern __shared__ __align__(1024) unsigned char ok_sh[];
  constexpr int ABYTES = OZ_TM * DP * 2;  // one digit operand of the row tile
  constexpr int BROWS = OZ_S * OZK_TC;
  constexpr int BBYTES = BROWS * DP * 2;
  constexpr uint32_t SBO = (DP / 8) * 128;
  constexpr int PCS = DP / 8;              // 16-byte pieces of one digit row
  unsigned char* As = ok_sh;
  unsigned char* Bs = ok_sh + OZ_S * ABYTES;
  __shared__ int pj_s[2][OZK_TC], ej_s[2][OZK_TC], idj_s[2][OZK_TC];
  __shared__ double nj_s[2][OZK_TC];
  __shared__ uint64_t mbar[2], fin;
  __shared__ uint32_t tslot;
  __shared__ double exp_tab[OZ_EXP_J];
  const int tid = (int)threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < OZ_EXP_J; e += (int)blockDim.x) exp_tab[e] = ex.T[e];  // read after the barriers below
  const OzKDesc D = descs[oz_find(descs, nd, (int)blockIdx.x)];
  const int i0 = ((int)blockIdx.x - D.tile0) * OZ_TM;
  const int nct = (D.ncols + OZK_TC - 1) / OZK_TC;
  if (warp == 0) tc::tmem_alloc(&tslot, 512);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_init(&fin, 1);
  }
  for (int e = tid; e < OZ_S * OZ_TM * PCS; e += OZK_THREADS) {
    const int kq = e % PCS, r = (e / PCS) % OZ_TM, i = e / (PCS * OZ_TM);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (i0 + r < D.nrows)
      v = *reinterpret_cast<const uint4*>(XD + ((size_t)(D.row0 + i0 + r) * OZ_S + i) * DP + kq * 8);
    *reinterpret_cast<uint4*>(As + i * ABYTES + (r >> 3) * SBO + kq * 128 + (r & 7) * 16) = v;
  }
  auto gather = [&](int ct, int b) {  // all threads; ends with the operand visible to the MMA
    if (tid < OZK_TC) {
      const int j = ct * OZK_TC + tid;
      int p = -1;
      if (j < D.ncols) p = D.colsA ? (j < D.nA ? D.colsA[j] : D.colsB[j - D.nA]) : D.col0 + j;
      pj_s[b][tid] = p;
      idj_s[b][tid] = p >= 0 && D.ident ? D.ident[p] : p;
      ej_s[b][tid] = p >= 0 ? XE[p] : 0;
      nj_s[b][tid] = p >= 0 ? xn[p] : 0.0;
    }
    __syncthreads();
    unsigned char* Bb = Bs + b * BBYTES;
    for (int e = tid; e < BROWS * PCS; e += OZK_THREADS) {
      const int kq = e % PCS, n = e / PCS, c = n % OZK_TC, jd = n / OZK_TC;
      const int p = pj_s[b][c];
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (p >= 0) v = *reinterpret_cast<const uint4*>(XD + ((size_t)p * OZ_S + jd) * DP + kq * 8);
      *reinterpret_cast<uint4*>(Bb + (n >> 3) * SBO + kq * 128 + (n & 7) * 16) = v;
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
  };
  auto issue = [&](int b, uint32_t tmem) {  // thread 0
    tc::fence_after_sync();
    const uint32_t a0 = tc::smem_addr(As), b0 = tc::smem_addr(Bs + b * BBYTES);
#pragma unroll 1
    for (int ks = 0; ks < DP / 16; ++ks)
#pragma unroll
      for (int i = 0; i < OZ_S; ++i)
        tc::mma_f16(tmem + (uint32_t)(b * 256 + i * OZK_TC), tc::smem_desc(a0 + i * ABYTES + ks * 256, 128, SBO),
                    tc::smem_desc(b0 + ks * 256, 128, SBO), tc::idesc_bf16(OZ_TM, (OZ_S - i) * OZK_TC),
                    !(ks == 0 && i == 0));
    tc::mma_commit(&mbar[b]);
  };
  if (nct > 0) gather(0, 0);  // block-uniform
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  if (tid == 0 && nct > 0) issue(0, tmem);
  const int q = warp & 3, hh = warp >> 2;
  const int r = q * 32 + lane, i = i0 + r;
  const bool rv = i < D.nrows;
  const int pi = D.row0 + (rv ? i : 0);
  const int idi = D.ident ? D.ident[pi] : pi;
  const int Ei = XE[pi];
  const double ni = xn[pi];
  bool failed = false;
  for (int ct = 0; ct < nct; ++ct) {
    const int b = ct & 1;
    if (ct + 1 < nct) {  // MMA ct - 1 is complete and its accumulator read: reuse both
      gather(ct + 1, b ^ 1);
      if (tid == 0) issue(b ^ 1, tmem);
    }
    const bool got = tc::mbar_wait(&mbar[b], (uint32_t)((ct >> 1) & 1), OZK_WAIT);
    if (__syncthreads_or(!got)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    long long hi[16], lo[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0;
#pragma unroll
    for (int t = 0; t < OZ_S; ++t) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 256 + t * OZK_TC + hh * 16), v);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const long long sv = (long long)__float2int_rn(v[c]);
        if (t < OZ_HI) hi[c] += sv * (1ll << (8 * (OZ_HI - 1 - t)));
        else lo[c] += sv * (1ll << (8 * (OZ_S - 1 - t)));
      }
    }
    if (rv) {
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int cc = hh * 16 + c, j = ct * OZK_TC + cc;
        if (j >= D.ncols) continue;
        const int e = Ei + ej_s[b][cc] - 14 - 8 * (OZ_HI - 1);
        const double dot = fma((double)lo[c], OZ_LO_SCALE, (double)hi[c]) * oz_pow2(e);
        const double d2 = fmax((ni + nj_s[b][cc]) - 2.0 * dot, 0.0);
        double kv = oz_exp_neg(d2 * D.scale, exp_tab, ex.inv_l, ex.l_hi, ex.l_lo);
        if (idi == idj_s[b][cc]) kv += D.diag;
        D.out[(size_t)i + (size_t)j * D.ld] = kv;
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // accumulator b and its column data are free for tile ct + 2
  }
  if (failed) {
    if (tid == 0) {
      atomicOr(status, DEV_TIMEOUT);
      tc::mma_commit(&fin);  // every MMA issued so far
      tc::mbar_wait(&fin, 0, OZK_WAIT);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_free(tmem, 512);
}

}  // namespace

int oz_dpad(int d) { return d >= 1 && d <= 64 ? (d + 15) / 16 * 16 : 0; }

void oz_points(const double* X, int N, int d, uint16_t* XD, int* XE, cudaStream_t st) {
  const int DP = oz_dpad(d);
  if (N <= 0 || DP == 0) return;
  ProfScope _ps(PK_OZ_SPLIT, st);
  const long long thr = (long long)N * (DP / 8);
  oz_points_kernel<<<(unsigned)((thr + 255) / 256), 256, 0, st>>>(X, N, d, DP, XD, XE);
  IA_LAUNCH_CHECK();
}

// The table and constants of oz_exp_neg, in long double (then rounded to FP64) once.
static const OzExp& oz_exp_table() {
  static const OzExp tab = [] {
    OzExp e{};
    for (int j = 0; j < OZ_EXP_J; ++j) e.T[j] = (double)exp2l((long double)j / (long double)OZ_EXP_J);
    const long double L = logl(2.0L) / (long double)OZ_EXP_J;
    e.inv_l = (double)(1.0L / L);
    double hi = (double)L;
    unsigned long long b;
    std::memcpy(&b, &hi, sizeof b);
    b &= ~((1ull << 18) - 1);
    std::memcpy(&hi, &b, sizeof b);
    e.l_hi = hi;
    e.l_lo = (double)(L - (long double)hi);
    return e;
  }();
  return tab;
}

template <int DP>
static void launch_kblock(const uint16_t* XD, const int* XE, const double* xn, const OzKDesc* descs_dev, int ndesc,
                          int ntiles, int* status, cudaStream_t st) {
  // at least 116 KB, so that one block holds an SM (its 512 TMEM columns are all of them)
  const int smem = std::max(OZ_S * OZ_TM * DP * 2 + 2 * OZ_S * OZK_TC * DP * 2, 116 * 1024);
  static bool attr = false;
  if (!attr) {
    IA_CUDA(cudaFuncSetAttribute(oz_kblock_kernel<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr = true;
  }
  oz_kblock_kernel<DP><<<ntiles, OZK_THREADS, smem, st>>>(XD, XE, xn, descs_dev, ndesc, status, oz_exp_table());
  IA_LAUNCH_CHECK();
}

void oz_kblocks(const uint16_t* XD, const int* XE, const double* xn, int d, const OzKDesc* descs_dev, int ndesc,
                int ntiles, int* status, cudaStream_t st) {
  if (ndesc <= 0 || ntiles <= 0) return;
  ProfScope _ps(PK_KBLOCK_OZ, st);
  switch (oz_dpad(d)) {
    case 16: launch_kblock<16>(XD, XE, xn, descs_dev, ndesc, ntiles, status, st); break;
    case 32: launch_kblock<32>(XD, XE, xn, descs_dev, ndesc, ntiles, status, st); break;
    case 48: launch_kblock<48>(XD, XE, xn, descs_dev, ndesc, ntiles, status, st); break;
    case 64: launch_kblock<64>(XD, XE, xn, descs_dev, ndesc, ntiles, status, st); break;
    default: throw Error(IASKIT_ERR_UNSUPPORTED, "sliced kernel blocks: dimension above 64");
  }
}

size_t oz_arec_bytes(int rows, int cols) {
  if (rows <= 0 || cols <= 0) return 0;
  return (size_t)ceil_div((size_t)rows, OZ_TM) * ceil_div((size_t)cols, OZ_KC) * OZ_AREC;
}
size_t oz_brec_bytes(int K) { return K <= 0 ? 0 : (size_t)ceil_div((size_t)K, OZ_KC) * OZ_BREC; }

void oz_split_blocks(const OzSplitDesc* descs_dev, int ndesc, int ntiles, cudaStream_t st) {
  if (ndesc <= 0 || ntiles <= 0) return;
  ProfScope _ps(PK_OZ_SPLIT, st);
  oz_split_kernel<<<ntiles, OZ_TM, 0, st>>>(descs_dev, ndesc);
  IA_LAUNCH_CHECK();
}

void oz_split_vecs(const OzVecDesc* descs_dev, int ndesc, cudaStream_t st) {
  if (ndesc <= 0) return;
  ProfScope _ps(PK_OZ_SPLIT, st);
  oz_vec_kernel<<<ndesc, 128, 0, st>>>(descs_dev);
  IA_LAUNCH_CHECK();
}

void oz_apply(const OzApplyDesc* descs_dev, int ndesc, int ntiles, int* status, cudaStream_t st) {
  if (ndesc <= 0 || ntiles <= 0) return;
  static bool attr = false;
  const int smem = OZ_NS * OZ_STAGE;
  if (!attr) {
    IA_CUDA(cudaFuncSetAttribute(oz_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr = true;
  }
  ProfScope _ps(PK_OZ, st);
  oz_apply_kernel<<<ntiles, OZ_THREADS, smem, st>>>(descs_dev, ndesc, status);
  IA_LAUNCH_CHECK();
}

}  // namespace iaskit
