// lmf_tree.h -- threshold-filtered aggregates: the regression-tree node batch
// of Sec. 2 (Eq. regression-tree), RT(1 a, y a, y^2 a) with a a product of
// threshold indicators, evaluated for many (node, attribute, threshold)
// triples at once as per-node histograms over the sorted thresholds.
#pragma once

#include <cstdint>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "lmf.h"
#include "lmf_internal.h"
#include "lmf_jit.h"

namespace lmf {

struct TreeFactorIn {
  std::string attr;
  int kind, power;
  double thr;
};
struct TreeAggIn {
  std::vector<TreeFactorIn> factors;
};

struct TreePlanImpl;  // lmf_tree.cu
struct TreePlan {
  TreePlanImpl* impl = nullptr;
  ~TreePlan();
};

// Decompose the batch into nodes (conjunctions), split attributes with their
// sorted thresholds and moments (monomials of degree <= 2).
lmf_status tree_plan(const std::vector<TreeAggIn>& in, const std::map<std::string, int>& zidx,
                     TreePlan* tp, std::string* msg);
// Device buffers: the histogram (reset every run) ...
void tree_alloc_zeroed(TreePlan* tp, int64_t N, const std::function<size_t(size_t)>& take);
// ... plan tables and outputs (written once).
void tree_alloc(TreePlan* tp, int64_t N, const std::function<size_t(size_t)>& take);
lmf_status tree_finish(TreePlan* tp, char* base, long long* res_i64, double* res_f64,
                       const std::vector<int64_t>& agg_off, const std::vector<int>& filt_idx,
                       const std::vector<int32_t>& agg_dtype, uint32_t* status, int64_t N,
                       int num_sms, const std::map<std::string, double>& bound, double W,
                       const RootParams& rp, int res_q);
// What the plan-time compiler needs (jit_tree_source); the compiled pass, when
// set, replaces the library's interpreted kernel
void tree_jit_spec(const TreePlan* tp, TreeJitSpec* out);
void tree_set_jit(TreePlan* tp, cudaKernel_t k);
cudaError_t tree_launch(TreePlan* tp, const RootParams& rp, cudaStream_t s, int* n_kernels);
// The autotuner times the pass over its CTAs-per-SM candidates at the first
// run and keeps the fastest.
bool tree_needs_tuning(const TreePlan* tp);
cudaError_t tree_autotune(TreePlan* tp, const RootParams& rp, cudaStream_t s);
// chosen shape, for reporting: slices (1), split attributes, nodes, CTAs per SM, chunk rows (0)
void tree_shape(const TreePlan* tp, int* out5);
void tree_counts(const TreePlan* tp, int32_t* nodes, int32_t* groups);

}  // namespace lmf
