// lmf_gram_tc.h -- the root scan with the Gram on sm_103a tensor cores
// (tcgen05.mma, operands in shared memory, accumulator in tensor memory).
#pragma once

#include <cstdint>
#include <functional>

#include "lmf_internal.h"

namespace lmf {

struct GramTcPlan {
  int m = 0;              // z length
  int grid = 0;           // CTAs
  int64_t n_tiles = 0;    // tiles of kTcRows root rows
  size_t smem = 0;        // dynamic shared memory per CTA
  size_t part_off = 0;    // arena offset of per-CTA partial Gram blocks
};

bool gram_tc_supported(int m);
void gram_tc_shape(int m, int64_t N, int num_sms, int tile_rows, GramTcPlan* tp);
void gram_tc_alloc(GramTcPlan* tp, const std::function<size_t(size_t)>& take);
void gram_tc_finish(GramTcPlan* tp, RootParams& rp, char* base);
cudaError_t gram_tc_launch(GramTcPlan* tp, const RootParams& rp, cudaStream_t s);

}  // namespace lmf
