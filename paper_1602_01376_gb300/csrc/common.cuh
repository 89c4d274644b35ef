// Shared device/host utilities of the INV-ASKIT CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/iaskit.h"
#include "prof.cuh"

namespace iaskit {

// ------------------------------------------------------------------ errors
// Host code reports failures by throwing Error; the C ABI turns it into a status.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& msg) : std::runtime_error(msg), code(c) {}
};

#define IA_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t _e = (call);                                                           \
    if (_e != cudaSuccess) {                                                           \
      if (_e == cudaErrorMemoryAllocation)                                             \
        throw ::iaskit::Error(IASKIT_ERR_NOMEM, std::string(#call ": ") +              \
                                                    cudaGetErrorString(_e));           \
      throw ::iaskit::Error(IASKIT_ERR_CUDA, std::string(#call ": ") +                 \
                                                 cudaGetErrorString(_e));              \
    }                                                                                  \
  } while (0)

#define IA_LAUNCH_CHECK()            \
  do {                                 \
    ++::iaskit::prof().launches;       \
    IA_CUDA(cudaGetLastError());       \
  } while (0)

// Device status bits (atomicOr into a device word, read back by the host).
enum : int {
  DEV_SINGULAR = 1,      // exact zero pivot
  DEV_BADINPUT = 2,      // non-finite value
  DEV_OVERFLOW = 4,      // an internal bound was exceeded (reported as UNSUPPORTED)
  DEV_TIMEOUT = 8,       // a bounded wait expired
};

// ------------------------------------------------------------ device memory
// A growable device buffer.  Reallocates only when a larger size is requested,
// so repeated factorizations of the same size allocate nothing.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void* ensure(size_t n) {
    if (n == 0) n = 16;
    if (n > bytes) {
      // work already queued may still read the old block: drain the device first
      if (p) cudaDeviceSynchronize();
      release();
      IA_CUDA(cudaMalloc(&p, n));
      bytes = n;
    }
    return p;
  }
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
  template <typename T>
  T* ensure_n(size_t count) { return static_cast<T*>(ensure(count * sizeof(T))); }
};

template <typename T>
inline void h2d(T* dst, const T* src, size_t n, cudaStream_t st) {
  if (n) IA_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, st));
}
template <typename T>
inline void d2h(T* dst, const T* src, size_t n, cudaStream_t st) {
  if (n) IA_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToHost, st));
}

inline unsigned ceil_div(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------ device helpers
// Monotone map double -> uint64: a < b  <=>  key(a) < key(b) for non-NaN inputs;
// -0.0 is mapped like +0.0 so that numerically equal values get equal keys.
__device__ __forceinline__ uint64_t orderable_key(double x) {
  if (x == 0.0) x = 0.0;
  uint64_t b = (uint64_t)__double_as_longlong(x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_to_double(uint64_t k) {
  uint64_t b = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Argmax over (value, index): larger value wins, equal values go to the lower index.
__device__ __forceinline__ void argmax_merge(double& v, int& i, double v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}
__device__ __forceinline__ void warp_argmax(double& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    argmax_merge(v, i, v2, i2);
  }
}

// SplitMix64 (Steele, Lea, Flood 2014): output for state x (advance by the golden
// gamma, then the variant-13 finaliser).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace iaskit
