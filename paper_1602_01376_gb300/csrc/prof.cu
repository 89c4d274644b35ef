// Kernel-class timers (see prof.cuh).
#include "prof.cuh"

namespace iaskit {

const char* prof_name(int k) {
  static const char* names[PK_COUNT] = {"tree", "knn", "sampling", "kernel_blocks", "cpqr_id",
                                        "assemble_P", "getrf", "getrs", "gemm", "kernel_matvec",
                                        "misc", "kernel_blocks_f32", "cpqr_id_f32", "getrf_f32",
                                        "getrs_f32", "gemm_f32", "learned_sampling", "mlp_bf16",
                                        "id_judge", "gemm_pair",
                                        "kernel_blocks_pair", "near_field", "predict",
                                        "operator_slices", "slice_split", "kernel_blocks_sliced",
                                        "getri_f32"};
  return (k >= 0 && k < PK_COUNT) ? names[k] : "?";
}

Profiler& prof() {
  static Profiler p;
  return p;
}

cudaEvent_t Profiler::get_event() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Profiler::resolve() {
  for (const Pending& p : pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ms[p.kind] += t;
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
}

void Profiler::reset() {
  resolve();
  for (int k = 0; k < PK_COUNT; ++k) {
    ms[k] = 0;
    calls[k] = 0;
    flops[k] = 0;
    bytes[k] = 0;
  }
}

ProfScope::ProfScope(int k, cudaStream_t s) : kind(k), st(s) {
  Profiler& p = prof();
  p.calls[k] += 1;
  if (p.enabled) {
    b = p.get_event();
    cudaEventRecord(b, s);
  }
}

ProfScope::~ProfScope() {
  Profiler& p = prof();
  if (b) {
    cudaEvent_t e = p.get_event();
    cudaEventRecord(e, st);
    p.pending.push_back(Profiler::Pending{kind, b, e});
  }
}

}  // namespace iaskit
