// lmf_jit.h -- plan-time compilation of the root scan.
//
// The paper's engine compiles each aggregate batch into code specialised to
// it (Sec. 1.2, compilation layer; App. C).  Here the plain root scan's row
// pass is generated from the finished plan with every layout fact as a
// constant (record words, z slots, fixed-point scales, category domains,
// shared-memory offsets) and compiled for sm_103a by NVRTC; the tile loop and
// the Gram phase are the same device code as the interpreted kernel
// (lmf_root_plain.cuh), so both compute the same values in the same order.
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

// compiles src for sm_103a, or finds it in the process-wide cache of compiled
// sources; on failure returns false with NVRTC's log in *log
bool jit_kernel(const std::string& src, const char* name, cudaKernel_t* k, std::string* log);

}  // namespace lmf
