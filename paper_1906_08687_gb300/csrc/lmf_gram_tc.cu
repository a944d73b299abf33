// lmf_gram_tc.cu -- root scan with the split-bf16 Gram on tcgen05 tensor cores.
#include "lmf_gram_tc.h"

namespace lmf {

bool gram_tc_supported(int) { return false; }
void gram_tc_shape(int m, int64_t, int, int, GramTcPlan* tp) { tp->m = m; tp->grid = 1; }
void gram_tc_alloc(GramTcPlan*, const std::function<size_t(size_t)>&) {}
void gram_tc_finish(GramTcPlan*, RootParams&, char*) {}
cudaError_t gram_tc_launch(GramTcPlan*, const RootParams&, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace lmf
