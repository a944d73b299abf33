// lmf_jit_tree.cu -- source generator for the tree pass compiled for a plan
// (see lmf_jit.h): the row pass of the root (features and the views' counts
// and means, no categories) and the node search as nested comparisons, over
// the body of the pass in lmf_tree_dev.cuh.  Compiled and loaded by
// jit_kernel like the root scan.
#include "lmf_jit.h"

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <functional>
#include <sstream>

namespace lmf {

namespace {

std::string tree_flit(float v) {  // exact float literal; infinities and NaNs by their bits
  char b[48];
  if (!std::isfinite(v)) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    std::snprintf(b, sizeof b, "__uint_as_float(0x%08xu)", u);
    return b;
  }
  std::snprintf(b, sizeof b, "%.9e", static_cast<double>(v));
  return std::string(b) + "f";
}

// decision trees beyond these sizes are searched through the device tables
constexpr size_t kJitTreeMaxEntries = 4096;
constexpr size_t kJitTreeMaxChecks = 32768;

}  // namespace

std::string jit_tree_source(const RootParams& rp, const TreeJitSpec& t) {
  std::ostringstream o;
  o << "// plan-specialised tree pass (generated)\n#include \"lmf_tree_dev.cuh\"\nnamespace lmf {\n"
    << "struct JitTreeRow {\n"
    << "  static __device__ __forceinline__ long long row(const RootParams& p, int64_t r, float* zrow, int32_t* crow) {\n"
    << "    (void)crow;\n    long long w = 1;\n    zrow[0] = 1.f;\n";
  for (int i = 0; i < rp.n_x; ++i) {
    if (rp.x[i].dtype == 2)
      o << "    zrow[" << 1 + i << "] = static_cast<float>(__ldcs(static_cast<const double*>(p.x[" << i << "].p) + r));\n";
    else
      o << "    zrow[" << 1 + i << "] = __ldcs(static_cast<const float*>(p.x[" << i << "].p) + r);\n";
  }
  for (int g = 0; g < rp.n_grp; ++g) {
    const GroupDesc& G = rp.grp[g];
    const int nw = G.n_cnt + G.n_mu;  // categories are not read by the tree pass
    o << "    {\n      const int32_t fk = p.grp[" << g << "].fk[r];\n"
      << "      if (fk < 0 || fk >= " << G.K << ") {\n        w = 0;\n      } else {\n"
      << "        const uint4* rec = reinterpret_cast<const uint4*>(p.grp[" << g << "].rec + static_cast<int64_t>(fk) * "
      << G.stride << ");\n";
    const char* comp[4] = {"v.x", "v.y", "v.z", "v.w"};
    for (int q = 0; q * 4 < nw; ++q) {
      o << "        {\n          const uint4 v = __ldg(rec + " << q << ");\n";
      for (int e = 0; e < 4; ++e) {
        const int wd = 4 * q + e;
        if (wd < G.n_cnt) o << "          w *= static_cast<long long>(" << comp[e] << ");\n";
        else if (wd < nw)
          o << "          zrow[" << rp.grp_zoff[g] + wd - G.n_cnt << "] = __uint_as_float(" << comp[e] << ");\n";
      }
      o << "        }\n";
    }
    o << "      }\n    }\n";
  }
  o << "    return w;\n  }\n"
    << "  static __device__ __forceinline__ int node(const TreeDev& d, int g, const float* zrow) {\n    (void)d;\n";
  // the decision tree as nested comparisons; a leaf checks its candidates'
  // predicates in order, the first that holds is the row's node.  A tree too
  // large to spell out keeps the search over the device tables.
  size_t checks = 0;
  for (const auto& e : t.dt)
    if (e.leaf)
      for (int c = e.left; c < e.left + e.right; ++c) checks += 1 + t.preds[t.cand[c]].size();
  // the end of node() and the kernel over the library's body of the pass
  auto finish = [&](const char* last) {
    o << "    " << last << "\n  }\n};\n}  // namespace lmf\n"
      << "extern \"C\" __global__ void __launch_bounds__(lmf::kTreeThreads, 2) lmf_tree_jit(\n"
      << "    const __grid_constant__ lmf::RootParams p, const __grid_constant__ lmf::TreeDev d) {\n"
      << "  lmf::tree_body<lmf::JitTreeRow, " << t.mp << ">(p, d);\n}\n";
    return o.str();
  };
  if (t.dt.size() > kJitTreeMaxEntries || checks > kJitTreeMaxChecks) return finish("return tree_node_of(d, g, zrow);");
  std::function<void(int, int)> gen = [&](int i, int ind) {
    const std::string sp(static_cast<size_t>(ind), ' ');
    const TreeJitSpec::Entry& e = t.dt[i];
    if (!e.leaf) {
      o << sp << "if (zrow[" << e.z << "] <= " << tree_flit(e.thr) << ") {\n";
      gen(e.left, ind + 2);
      o << sp << "} else {\n";
      gen(e.right, ind + 2);
      o << sp << "}\n";
      return;
    }
    for (int c = e.left; c < e.left + e.right; ++c) {
      const int n = t.cand[c];
      o << sp << "if (true";
      for (const auto& pr : t.preds[n])
        o << " && zrow[" << pr.z << "] " << (pr.op == 0 ? "<=" : ">") << " " << tree_flit(pr.thr);
      o << ") return " << n << ";\n";
    }
    o << sp << "return static_cast<int>(kNoNode);\n";
  };
  for (size_t g = 0; g < t.droot.size(); ++g) {
    o << "    if (g == " << g << ") {\n";
    gen(t.droot[g], 6);
    o << "    }\n";
  }
  return finish("return static_cast<int>(kNoNode);");
}

}  // namespace lmf
