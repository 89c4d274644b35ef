// Per-kernel-class timing with CUDA events and a count of kernel launches.
//
// When enabled (option "profile"), every launcher brackets its kernel with a pair
// of events on the launching stream; the pairs are resolved after the next stream
// synchronization of an API call and summed per class.  The launch counter counts
// every kernel launch of the library, enabled or not.
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace iaskit {

enum ProfKind {
  PK_TREE = 0,
  PK_KNN,
  PK_SAMPLE,
  PK_KBLOCK,
  PK_CPQR,
  PK_ASSEMBLE_P,
  PK_GETRF,
  PK_GETRS,
  PK_GEMM,
  PK_MATVEC,
  PK_MISC,
  PK_KBLOCK32,   // FP32 variants of the dense kernels (mixed-precision form)
  PK_CPQR32,
  PK_GETRF32,
  PK_GETRS32,
  PK_GEMM32,
  PK_LEARN,      // learned sampling: candidates, features, selection, streams, labels
  PK_MLP,        // BF16 MLP forward / backward / Adam (tensor cores)
  PK_JUDGE,      // held-out ID error of the learned and plain samples
  PK_GEMM_PAIR,  // FP64-accurate products on FP32 pairs (operator of the mixed form)
  PK_KBLOCK_PAIR,  // kernel blocks evaluated on FP32 pairs (operator of the mixed form)
  PK_NEAR,         // near-field correction S of the kNN-separated operator
  PK_PREDICT,      // exact kernel sums at test points (kernel regression, eps_M)
  PK_OZ,           // FP64 operator products by exact BF16 slices (tensor cores)
  PK_OZ_SPLIT,     // splitting FP64 blocks and right-hand sides into BF16 digits
  PK_KBLOCK_OZ,    // FP64 kernel blocks with the dot products on the tensor cores
  PK_GETRI32,      // explicit inverses of the FP32 LUs (leaf blocks, reduced systems)
  PK_COUNT
};

// The FP32 class of a dense kernel class when T is float.
template <typename T>
inline int pk_of(int kind) {
  if (sizeof(T) != 4) return kind;
  switch (kind) {
    case PK_KBLOCK: return PK_KBLOCK32;
    case PK_CPQR: return PK_CPQR32;
    case PK_GETRF: return PK_GETRF32;
    case PK_GETRS: return PK_GETRS32;
    case PK_GEMM: return PK_GEMM32;
    default: return kind;
  }
}

const char* prof_name(int kind);

struct Profiler {
  bool enabled = false;
  double ms[PK_COUNT] = {};
  long long calls[PK_COUNT] = {};
  double flops[PK_COUNT] = {};
  double bytes[PK_COUNT] = {};  // algorithmic device-memory bytes (memory-bound classes)
  long long launches = 0;
  struct Pending {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get_event();
  void resolve();  // call after the stream has been synchronized
  void reset();
};

Profiler& prof();

// RAII bracket of one launch: records start/stop events when profiling is enabled.
struct ProfScope {
  int kind;
  cudaStream_t st;
  cudaEvent_t b = nullptr;
  ProfScope(int k, cudaStream_t s);
  ~ProfScope();
};

}  // namespace iaskit
