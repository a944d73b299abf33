// lmf_jit.h -- plan-time compilation of the root scan and the tree pass.
//
// The paper's engine compiles each aggregate batch into code specialised to
// it (Sec. 1.2, compilation layer; App. C).  Here the plain root scan's row
// pass is generated from the finished plan with every layout fact as a
// constant (record words, z slots, fixed-point scales, category domains,
// shared-memory offsets) and compiled for sm_103a by NVRTC; the tile loop and
// the Gram phase are the same device code as the interpreted kernel
// (lmf_root_plain.cuh), so both compute the same values in the same order.
// The tree pass of filtered aggregates is compiled the same way (its row pass
// and its node search generated, lmf_jit_tree.cu; its body lmf_tree_dev.cuh).
#pragma once

#include <string>
#include <vector>

#include "lmf_internal.h"

namespace lmf {

// NVRTC can be loaded (libnvrtc is looked up at run time, never linked)
bool jit_available();

// CUDA source of the plain root scan for a plan: rp carries the plan's
// constants (its device pointers are read from the kernel parameter at run
// time, so plans of the same shape share the source), direct all of its
// per-row tables; min_ctas the CTAs per SM its launch bounds ask for.  The
// kernel is named lmf_root_plain_jit.
std::string jit_plain_source(const RootParams& rp, int mp, const std::vector<DirectAgg>& direct, int min_ctas);
// the same row pass inside the tensor-core scan (lmf_root_tc.cuh); the
// kernel is named lmf_root_tc_jit
std::string jit_tc_source(const RootParams& rp, const std::vector<DirectAgg>& direct);
std::string jit_source(const RootParams& rp, int mp, const std::vector<DirectAgg>& direct, int min_ctas, bool tc);

// Shared-memory layout of the key-level root scan (lmf_root_lean.cuh) for a
// plan: the generated row pass carries it as constants, the planner sizes the
// launch with it.  Per CTA, 256 rows: the fixed-point tile [256][zi_ld] int64
// (column 0 the row's count, then every value a reverse view sums, exact
// integers at the value's fixed-point scale), the root features of the row
// Gram [256][mpx] floats, the z rows of per-row tables that sum a feature
// [256][zf_ld] floats, staging for bulk reductions [256][stage_w] int64, the
// row categories of per-row tables [256][cat_w] int32, then the hot-cell and
// resident-key counters (never below kLeanFoldStage: between tiles the row
// Gram's chains are summed through the start of shared memory).
constexpr int kLeanFoldStage = 16 * 256 * 4;  // the row Gram's fold staging at the start of shared memory
struct LeanShape {
  int mpx = 4;                  // width of the row-level Gram block (multiple of 4)
  int ncol = 1;                 // columns of the fixed-point tile
  int zi_ld = 2;                // int64 words per fixed-point row (even: 16-byte rows)
  int col_of_z[kMaxZ];          // column of a z index in the fixed-point tile, -1: none
  float col_scale[kMaxZ];       // fixed-point scale of each column (1 for the count)
  int zf_ld = 0;                // floats per z row of per-row tables (0: none staged)
  int stage_w = 0;              // int64 words staged per row for bulk reductions (even)
  int stage_at[kMaxGroups];     // per reverse view: -1 not bulk, -2 bulk straight from the
                                // fixed-point row (its slots are columns 1..n), else first staged word
  int cat_w = 0;                // row categories staged per row
  int racc = 1;                 // 32-word chunks of the resident view's record
  uint32_t xg_off = 0, zf_off = 0, stage_off = 0, cat_off = 0, cache_off = 0;
  size_t smem = 0;              // dynamic shared memory of one CTA, counters included
};
LeanShape lean_shape(const RootParams& rp, bool direct_z);
// CUDA source of the key-level root scan of a plan (kernel lmf_root_lean_jit)
std::string jit_lean_source(const RootParams& rp, const std::vector<DirectAgg>& direct, int min_ctas);

// What the compiled tree pass needs from a tree plan (lmf_tree.cu): the z
// width, and per group of mutually exclusive nodes the decision tree over the
// nodes' predicates (entries: a split z <= thr to left / right, or a leaf
// listing candidate nodes [left, left + right) of cand) and every node's
// predicates (z, op 0: z <= thr, 1: z > thr).
struct TreeJitSpec {
  struct Entry {
    int z, leaf;
    float thr;
    int left, right;
  };
  struct Pred {
    int z, op;
    float thr;
  };
  int mp = 16;
  std::vector<int> droot;
  std::vector<Entry> dt;
  std::vector<int> cand;
  std::vector<std::vector<Pred>> preds;
};
// CUDA source of the tree pass for a plan (kernel lmf_tree_jit): the row pass
// (root columns and view records straight into the row's z) and the node
// search (the decision tree as nested comparisons against constants)
// generated, the rest the library's tree_body (lmf_tree_dev.cuh)
std::string jit_tree_source(const RootParams& rp, const TreeJitSpec& t);

// compiles src for sm_103a, or finds it in the process-wide cache of compiled
// sources; on failure returns false with NVRTC's log in *log
bool jit_kernel(const std::string& src, const char* name, cudaKernel_t* k, std::string* log);
// compiles every (source, kernel name) job into that cache on up to `threads`
// host threads (device `device` current in each); returns how many compiled
int jit_kernels_parallel(const std::vector<std::pair<std::string, const char*>>& jobs, int threads, int device);

}  // namespace lmf
