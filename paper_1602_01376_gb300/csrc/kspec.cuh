// The kernel function of a factorization: the Gaussian of eq. (gaussian) (the default)
// or a polynomial kernel.  The paper reports tests with a polynomial kernel (Sec. IV,
// Tab. weak) without its degree or constants; the one built here is
//   K(x, y) = (x . y / h^2 + c)^p,  integer p >= 1, c >= 0 (options "poly_p", "poly_c"),
// with the factorization's h as its length scale.  Descriptors carry one per-problem
// `scale`: -1 / (2 h^2) for the Gaussian, 1 / h^2 for the polynomial.  Every
// translation unit that evaluates kernel values holds the spec in constant memory and
// exposes a setter, which the host calls (stream-ordered) before such launches.
#pragma once
#include <cuda_runtime.h>

namespace iaskit {

struct KernelSpec {
  int poly = 0;    // 0 Gaussian, 1 polynomial
  int p = 2;       // polynomial degree
  double c = 1.0;  // polynomial constant
};

// t^p for a small integer p >= 1 by repeated multiplication (each product rounded).
template <typename T>
__device__ __forceinline__ T kspec_pow(T t, int p) {
  T v = t;
  for (int i = 1; i < p; ++i) v *= t;
  return v;
}

// Kernel value from the dot product (polynomial) or the squared distance (Gaussian).
__device__ __forceinline__ double kspec_value(const KernelSpec& k, double dot, double d2, double scale) {
  return k.poly ? kspec_pow(fma(dot, scale, k.c), k.p) : exp(d2 * scale);
}

}  // namespace iaskit

// Declares this translation unit's constant copy of the spec and its host setter.
#define IA_KERNEL_SPEC_TU(setter)                                                                  \
  namespace iaskit {                                                                               \
  __constant__ KernelSpec g_kspec;                                                                 \
  void setter(const KernelSpec& k, cudaStream_t st) {                                              \
    IA_CUDA(cudaMemcpyToSymbolAsync(g_kspec, &k, sizeof(KernelSpec), 0, cudaMemcpyHostToDevice, st)); \
  }                                                                                                \
  }
