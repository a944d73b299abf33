// lmf_gram_tc.h -- the root scan with the Gram on sm_103a tensor cores
// (tcgen05.mma, operands in shared memory, accumulators in tensor memory).
#pragma once

#include <cstdint>
#include <functional>

#include "lmf_internal.h"

namespace lmf {

struct GramTcPlan {
  int m = 0;              // z length (<= 32)
  int grid = 0;           // persistent CTAs
  int num_sms = 0;
  int64_t n_tiles = 0;    // tiles of 128 root rows
  size_t smem = 0;        // dynamic shared memory per CTA
  size_t part_off = 0;    // arena offset of per-CTA partial blocks [grid][3][32][32] f64
  double* part = nullptr;
};

// z lengths the kernel handles (one 32-feature block per split piece)
bool gram_tc_supported(int m);
// dynamic shared memory of one CTA
size_t gram_tc_smem(int n_rowcat, int cache_cells, int res_cells);
void gram_tc_shape(int m, int64_t N, int num_sms, int tile_rows, GramTcPlan* tp);
// shared memory / grid for a row-category vector of n_rowcat entries
cudaError_t gram_tc_configure(GramTcPlan* tp, int n_rowcat, int ctas_per_sm, int cache_cells, int res_cells);
void gram_tc_alloc(GramTcPlan* tp, const std::function<size_t(size_t)>& take);
void gram_tc_finish(GramTcPlan* tp, RootParams& rp, char* base);
cudaError_t gram_tc_launch(GramTcPlan* tp, const RootParams& rp, cudaStream_t s);
// the bounded mbarrier wait of k_root_tc against a barrier nothing arrives at;
// sets kStatusTimeout in *status when it gives up
cudaError_t gram_tc_wait_selftest(uint32_t* status, cudaStream_t s);
// ordered FP64 combine of the per-CTA blocks into G (m x m) and the count
cudaError_t gram_tc_combine(GramTcPlan* tp, const RootParams& rp, double* G, long long* count, cudaStream_t s);

}  // namespace lmf
