// lmf_keymap.h -- dense renumbering of sparse join keys (lmf_keymap.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace lmf {

// Renumbers the n int32 device columns cols[i] (rows[i] values each) by the
// rank of every value among the distinct values of the first n_child columns
// (the child sides of one join attribute's edges; their largest value is
// max_key >= 0).  Writes the renumbered copies to out[i] (device arrays of
// rows[i] int32, owned by the caller), values no child holds as -1, and the
// number of distinct child values to *n_keys.  Synchronous on stream s;
// allocates and frees 2 * (max_key / 32 + 1) words of scratch.
cudaError_t keymap_renumber(const int32_t* const* cols, const int64_t* rows, int n, int n_child, int32_t max_key,
                            int32_t* const* out, int64_t* n_keys, cudaStream_t s);

}  // namespace lmf
