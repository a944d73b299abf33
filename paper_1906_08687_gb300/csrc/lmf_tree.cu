// lmf_tree.cu -- filtered (tree-node) aggregates.
#include "lmf_tree.h"

namespace lmf {

struct TreePlanImpl {};
TreePlan::~TreePlan() { delete impl; }

lmf_status tree_plan(const std::vector<TreeAggIn>&, const std::map<std::string, int>&, TreePlan*,
                     std::string* msg) {
  *msg = "threshold-filtered aggregates are not built yet";
  return LMF_ERR_UNSUPPORTED;
}
void tree_alloc_zeroed(TreePlan*, const std::function<size_t(size_t)>&) {}
void tree_alloc(TreePlan*, const std::function<size_t(size_t)>&) {}
lmf_status tree_finish(TreePlan*, char*, long long*, double*, const std::vector<int64_t>&,
                       const std::vector<int>&, const std::vector<int32_t>&, uint32_t*, int64_t, int,
                       const std::map<std::string, double>&, double, const RootParams&) {
  return LMF_ERR_UNSUPPORTED;
}
cudaError_t tree_launch(TreePlan*, const RootParams&, cudaStream_t, int*) { return cudaErrorNotSupported; }

}  // namespace lmf
