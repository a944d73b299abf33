// lmf_tree.h -- filtered aggregates (regression-tree node batches, Sec. 2 Eq.
// regression-tree): products of threshold indicators times a monomial of
// degree <= 2, evaluated as per-node histograms over sorted thresholds.
#pragma once

#include <cstdint>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "lmf.h"
#include "lmf_internal.h"

namespace lmf {

struct TreeFactorIn {
  std::string attr;
  int kind, power;
  double thr;
};
struct TreeAggIn {
  std::vector<TreeFactorIn> factors;
};

struct TreePlanImpl;  // defined in lmf_tree.cu
struct TreePlan {
  TreePlanImpl* impl = nullptr;
  ~TreePlan();
};

// decompose the batch: nodes, split attributes, threshold lists, moments
lmf_status tree_plan(const std::vector<TreeAggIn>& in, const std::map<std::string, int>& zidx,
                     TreePlan* tp, std::string* msg);
// device buffers: accumulators that every run starts from zero ...
void tree_alloc_zeroed(TreePlan* tp, const std::function<size_t(size_t)>& take);
// ... and tables written once at plan time
void tree_alloc(TreePlan* tp, const std::function<size_t(size_t)>& take);
lmf_status tree_finish(TreePlan* tp, char* base, long long* res_i64, double* res_f64,
                       const std::vector<int64_t>& agg_off, const std::vector<int>& filt_idx,
                       const std::vector<int32_t>& agg_dtype, uint32_t* status, int64_t N,
                       int num_sms, const std::map<std::string, double>& bound, double W,
                       const RootParams& rp);
cudaError_t tree_launch(TreePlan* tp, const RootParams& rp, cudaStream_t s, int* n_kernels);

}  // namespace lmf
