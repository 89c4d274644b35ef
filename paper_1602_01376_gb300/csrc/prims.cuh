// Device-wide primitives written for this library: exclusive scan and a stable
// LSD radix sort.  Used by the tree partition and the row sampling.
#pragma once
#include "common.cuh"

namespace iaskit {

// out[i] = sum_{j < i} in[j] for i < n (in and out may alias).  Returns nothing;
// uses `tmp` for per-block partial sums.
void exclusive_scan_i32(const int* in, int* out, size_t n, DevBuf& tmp, cudaStream_t st);

// Stable LSD radix sort of `keys` (and the payload `vals` when not null) by bits
// [0, nbits) of the keys, 8 bits per pass.  `alt_keys` / `alt_vals` / `hist` are
// scratch buffers grown as needed.  The result is left in `keys` / `vals`.
void radix_sort_u64(uint64_t* keys, uint32_t* vals, size_t n, int nbits, DevBuf& alt_keys,
                    DevBuf& alt_vals, DevBuf& hist, DevBuf& scan_tmp, cudaStream_t st);

}  // namespace iaskit
