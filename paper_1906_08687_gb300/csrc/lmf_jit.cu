// lmf_jit.cu -- source generator and NVRTC driver for the plan-specialised
// root scan (see lmf_jit.h).
#include "lmf_jit.h"

#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>

// the device headers the generated source includes, as text (written by the
// build from lmf_internal.h, lmf_rowpass.cuh, lmf_root_plain.cuh and
// lmf_root_tc.cuh)
#include "lmf_jit_headers.inc"

namespace lmf {

namespace {

// ---- NVRTC, resolved with dlopen --------------------------------------------
struct Nvrtc {
  bool ok = false;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) get_log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) get_cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  decltype(&nvrtcGetErrorString) err = nullptr;
};

const Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    void* h = nullptr;
    for (const char* nm : names)
      if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) return;
    n.create = reinterpret_cast<decltype(n.create)>(dlsym(h, "nvrtcCreateProgram"));
    n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(h, "nvrtcCompileProgram"));
    n.log_size = reinterpret_cast<decltype(n.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
    n.get_log = reinterpret_cast<decltype(n.get_log)>(dlsym(h, "nvrtcGetProgramLog"));
    n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
    n.get_cubin = reinterpret_cast<decltype(n.get_cubin)>(dlsym(h, "nvrtcGetCUBIN"));
    n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
    n.err = reinterpret_cast<decltype(n.err)>(dlsym(h, "nvrtcGetErrorString"));
    n.ok = n.create && n.compile && n.log_size && n.get_log && n.cubin_size && n.get_cubin && n.destroy && n.err;
  });
  return n;
}

// compiled sources -> kernels; libraries stay loaded for the process
std::mutex g_cache_mu;
std::map<std::string, cudaKernel_t> g_cache;

// ---- source generation --------------------------------------------------------
std::string flit(float v) {  // exact float literal
  char b[48];
  std::snprintf(b, sizeof b, "%.9e", static_cast<double>(v));
  return std::string(b) + "f";
}

void gen_record_word(std::ostringstream& o, const RootParams& rp, int g, int wd, const char* v) {
  const GroupDesc& G = rp.grp[g];
  if (wd < G.n_cnt) {
    o << "          w *= static_cast<long long>(" << v << ");\n";
  } else if (wd < G.n_cnt + G.n_mu) {
    o << "          zrow[" << rp.grp_zoff[g] + (wd - G.n_cnt) << "] = __uint_as_float(" << v << ");\n";
  } else if (wd < G.n_cnt + G.n_mu + G.n_cat) {
    o << "          crow[" << rp.grp_catoff[g] + (wd - G.n_cnt - G.n_mu) << "] = static_cast<int32_t>(" << v
      << ");\n";
  }
}

}  // namespace

bool jit_available() { return nvrtc().ok; }

std::string jit_plain_source(const RootParams& rp, int mp, const std::vector<DirectAgg>& direct, int min_ctas) {
  return jit_source(rp, mp, direct, min_ctas, false);
}

std::string jit_tc_source(const RootParams& rp, const std::vector<DirectAgg>& direct) {
  return jit_source(rp, 32, direct, 1, true);
}

std::string jit_source(const RootParams& rp, int mp, const std::vector<DirectAgg>& direct, int min_ctas, bool tc) {
  std::ostringstream o;
  const bool unit_w = rp.unit_w != 0;
  o << "// plan-specialised root scan (generated)\n#include \"" << (tc ? "lmf_root_tc.cuh" : "lmf_root_plain.cuh")
    << "\"\nnamespace lmf {\n";
  // slot tables of the reverse views summed per run: one entry per lane
  for (int r = 0; r < rp.n_rv; ++r) {
    const RevView& R = rp.rv[r];
    if (R.n_slot == 0) continue;
    const int n = (R.n_slot + 31) / 32 * 32;
    o << "__device__ const int8_t kZi" << r << "[" << n << "] = {";
    for (int s = 0; s < n; ++s) o << (s < R.n_slot ? R.slot_z[s] : 0) << (s + 1 < n ? "," : "");
    o << "};\n__device__ const float kSc" << r << "[" << n << "] = {";
    for (int s = 0; s < n; ++s) o << flit(s < R.n_slot ? R.slot_scale[s] : 0.f) << (s + 1 < n ? "," : "");
    o << "};\n";
  }
  o << "struct JitRowPass {\n"
    << "  static __device__ __forceinline__ constexpr int fold(const RootParams&) { return " << rp.fold << "; }\n"
       "  template <int MP>\n"
       "  static __device__ __forceinline__ long long run(const RootParams& p, int64_t row, float* zrow, int ldz,\n"
       "                                                  int32_t* crow, uint32_t* cache, uint32_t* res_hist,\n"
       "                                                  long long res_key) {\n"
       "    const int lane = threadIdx.x & 31;\n"
       "#pragma unroll\n"
       "    for (int i = 0; i < MP; i += 4) *reinterpret_cast<float4*>(zrow + i) = make_float4(0.f, 0.f, 0.f, 0.f);\n"
       "    long long w = 0;\n";
  // the root's columns are read once per launch: streaming loads (evict
  // first), so they do not push the views the atomics update out of L2
  for (int g = 0; g < rp.n_grp; ++g) o << "    int32_t fk" << g << " = -1;\n";
  o << "    if (row < p.N) {\n"
       "      w = 1;\n"
       "      zrow[0] = 1.f;\n";
  for (int i = 0; i < rp.n_x; ++i) {
    if (rp.x[i].dtype == 2)
      o << "      zrow[" << 1 + i << "] = static_cast<float>(__ldcs(static_cast<const double*>(p.x[" << i
        << "].p) + row));\n";
    else
      o << "      zrow[" << 1 + i << "] = __ldcs(static_cast<const float*>(p.x[" << i << "].p) + row);\n";
  }
  for (int g = 0; g < rp.n_grp; ++g) {
    const GroupDesc& G = rp.grp[g];
    const int nw = G.n_cnt + G.n_mu + G.n_cat;
    o << "      {\n        const int32_t fk = __ldcs(p.grp[" << g << "].fk + row);\n"
      << "        fk" << g << " = fk;\n"
      << "        if (fk < 0 || fk >= " << G.K << ") {\n          w = 0;\n        } else {\n"
      << "          const uint4* rec = reinterpret_cast<const uint4*>(p.grp[" << g
      << "].rec + static_cast<int64_t>(fk) * " << G.stride << ");\n";
    for (int q = 0; q < (nw + 3) / 4; ++q) {
      o << "          {\n          const uint4 v = __ldg(rec + " << q << ");\n";
      const char* comp[4] = {"v.x", "v.y", "v.z", "v.w"};
      for (int e = 0; e < 4; ++e) gen_record_word(o, rp, g, 4 * q + e, comp[e]);
      o << "          }\n";
    }
    o << "        }\n      }\n";
  }
  for (int i = 0; i < rp.n_rcat; ++i) {
    o << "      {\n        int32_t v = __ldcs(p.rcat[" << i << "] + row);\n"
      << "        if (v < 0 || v >= " << rp.rcat_dom[i] << ") {\n"
      << "          atomicOr(p.status, kStatusCatRange);\n          v = 0;\n        }\n"
      << "        crow[" << rp.n_rowcat - rp.n_rcat + i << "] = v;\n      }\n";
  }
  o << "      if (w == 0) {\n#pragma unroll\n"
       "        for (int i = 0; i < MP; i += 4) *reinterpret_cast<float4*>(zrow + i) = make_float4(0.f, 0.f, 0.f, "
       "0.f);\n      }\n    }\n"
       "    __syncwarp();\n"
       "    const bool live = w != 0;\n";
  if (rp.res_cells > 0)
    o << "    const long long fres = (live && res_key >= 0) ? static_cast<long long>(fk" << rp.res_grp
      << ") : -2ll;\n";
  else
    o << "    const long long fres = -2ll;\n";
  // reverse views
  for (int r = 0; r < rp.n_rv; ++r) {
    const RevView& R = rp.rv[r];
    o << "    {  // reverse view " << r << "\n"
      << "      const long long fk = live ? static_cast<long long>(fk" << R.grp << ") : -1ll;\n";
    o << "      const WarpRuns q = warp_runs(fk);\n"
      << "      rv_count_runs(q, " << (unit_w ? "true" : "false") << ", fk, w, p.rv[" << r << "].hist);\n";
    for (int s0 = 0; s0 < R.n_slot; s0 += 32) {
      o << "      {\n        const int s = " << s0 << " + lane;\n"
        << "        rv_slot_runs(q, " << (unit_w ? "true" : "false") << ", fk, w, zrow - lane * ldz, ldz, s < "
        << R.n_slot << ", kZi" << r << "[s], kSc" << r << "[s], p.rv[" << r << "].R, " << R.n_slot << ", s);\n"
        << "      }\n";
    }
    o << "    }\n";
  }
  // category views
  for (int v = 0; v < rp.n_cv; ++v) {
    const CatView& C = rp.cv[v];
    o << "    {  // category view " << v << "\n"
      << "      const long long fk = live ? static_cast<long long>(fk" << C.grp << ") : -1ll;\n"
      << "      const int b = live ? crow[" << C.bcat << "] : 0;\n";
    if (C.res_off >= 0) {
      o << "      if (res_key >= 0) {\n        if (live) {\n"
        << "          if (fk == res_key) rp_red_shared_u32(res_hist + " << C.res_off << " + b, static_cast<uint32_t>(w));\n"
        << "          else rp_red_u32(p.cv[" << v << "].V + fk * " << C.dom << " + b, static_cast<uint32_t>(w));\n"
        << "        }\n      } else {\n        root_cv_one(p.cv[" << v << "], fk, b, w, res_hist, res_key);\n      }\n";
    } else if (C.runs) {
      o << "      root_cv_one(p.cv[" << v << "], fk, b, w, res_hist, res_key);\n";
    } else {
      o << "      if (live) rp_red_u32(p.cv[" << v << "].V + fk * " << C.dom << " + b, static_cast<uint32_t>(w));\n";
    }
    o << "    }\n";
  }
  // per-row tables: the common kinds straight-line, the rest through the
  // interpreted routine
  const int n_inl = rp.n_direct < kDirInline ? rp.n_direct : kDirInline;
  for (int d = 0; d < n_inl; ++d) {
    const DirectAgg& A = direct[d];
    const bool count_pair = A.n_gb == 2 && A.z < 0 && unit_w;
    const char* generic = "root_direct_one(p, p.dir[%d], row, zrow, crow, w, cache, res_hist, res_key, fres);";
    char gl[160];
    std::snprintf(gl, sizeof gl, generic, d);
    o << "    {  // per-row table " << d << "\n";
    if (count_pair && A.res_off >= 0) {
      const int other = A.res_q == 0 ? 1 : 0;
      o << "      if (res_key >= 0) {\n        if (live) {\n          if (fres == res_key) {\n"
        << "            rp_red_shared_u32(res_hist + " << A.res_off << " + crow[" << A.cat[other] << "]"
        << (A.res_lanes ? " * 32 + lane" : "") << ", static_cast<uint32_t>(w));\n"
        << "          } else {\n"
        << "            rp_direct_add(p, p.dir[" << d << "], static_cast<int64_t>(crow[" << A.cat[0] << "]) * "
        << A.dom[1] << " + crow[" << A.cat[1] << "], crow, w, cache);\n"
        << "          }\n        }\n      } else {\n        " << gl << "\n      }\n";
    } else if (count_pair && A.res_off < 0 && !A.runs) {
      o << "      if (live) {\n        const int a = crow[" << A.cat[0] << "], b = crow[" << A.cat[1] << "];\n";
      if (A.cache_off >= 0 && rp.cache_cells > 0) {
        o << "        const int ha = __ldg(p.hot_lut + " << rp.hot_lut_off[A.cat[0]] << " + a);\n"
          << "        const int hb = __ldg(p.hot_lut + " << rp.hot_lut_off[A.cat[1]] << " + b);\n"
          << "        if (ha >= 0 && hb >= 0) {\n"
          << "          rp_red_shared_u32(cache + " << A.cache_off << " + ha * " << rp.hot_h
          << " + hb, static_cast<uint32_t>(w));\n"
          << "        } else {\n"
          << "          rp_add_ll(p.dir[" << d << "].out + static_cast<int64_t>(a) * " << A.dom[1] << " + b, w);\n"
          << "        }\n";
      } else {
        o << "        rp_add_ll(p.dir[" << d << "].out + static_cast<int64_t>(a) * " << A.dom[1] << " + b, w);\n";
      }
      o << "      }\n";
    } else {
      o << "      " << gl << "\n";
    }
    o << "    }\n";
  }
  if (rp.n_direct > kDirInline)
    o << "    for (int d = " << kDirInline << "; d < " << rp.n_direct
      << "; ++d) root_direct_one(p, p.direct[d], row, zrow, crow, w, cache, res_hist, res_key, fres);\n";
  if (rp.n_om > 0) {
    o << "    if (live) {\n"
         "      for (int o = 0; o < p.n_om; ++o) {\n"
         "        const OmegaAcc& O = p.om[o];\n"
         "        const GroupDesc& G = p.grp[O.grp];\n"
         "        const int32_t fk = G.fk[row];\n"
         "        const long long ce = static_cast<long long>(G.rec[static_cast<int64_t>(fk) * G.stride + "
         "O.cnt_word]);\n"
         "        rp_red_u64(O.omega + fk, static_cast<unsigned long long>(w / ce));\n"
         "      }\n    }\n";
  }
  o << "    (void)lane;\n    (void)fres;\n    return w;\n  }\n};\n}  // namespace lmf\n";
  if (tc)
    o << "extern \"C\" __global__ void __launch_bounds__(128) lmf_root_tc_jit(const __grid_constant__ "
         "lmf::RootParams p, int64_t n_tiles, double* part) {\n"
      << "  lmf::root_tc_body<lmf::JitRowPass>(p, n_tiles, part);\n}\n";
  else
    o << "extern \"C\" __global__ void __launch_bounds__(256, " << min_ctas << ") lmf_root_plain_jit(const __grid_constant__ "
         "lmf::RootParams p, int64_t n_tiles) {\n"
      << "  lmf::root_plain_body<" << mp << ", lmf::JitRowPass>(p, n_tiles);\n}\n";
  return o.str();
}

bool jit_kernel(const std::string& src, const char* name, cudaKernel_t* k, std::string* log) {
  const Nvrtc& n = nvrtc();
  if (!n.ok) {
    if (log) *log = "NVRTC not available";
    return false;
  }
  const std::string key = std::string(name) + '\n' + src;
  {
    std::lock_guard<std::mutex> g(g_cache_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *k = it->second;
      return true;
    }
  }
  nvrtcProgram prog = nullptr;
  const int nh = static_cast<int>(sizeof(kJitHeaderNames) / sizeof(kJitHeaderNames[0]));
  if (n.create(&prog, src.c_str(), "lmf_root_plain_jit.cu", nh, kJitHeaderSrc, kJitHeaderNames) != NVRTC_SUCCESS) {
    if (log) *log = "nvrtcCreateProgram failed";
    return false;
  }
  const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo", "--device-as-default-execution-space"};
  const nvrtcResult rc = n.compile(prog, 4, opts);
  if (rc != NVRTC_SUCCESS) {
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string l(ls, '\0');
    if (ls) n.get_log(prog, &l[0]);
    if (log) *log = std::string(n.err(rc)) + ": " + l;
    n.destroy(&prog);
    return false;
  }
  size_t cs = 0;
  n.cubin_size(prog, &cs);
  std::vector<char> cubin(cs);
  n.get_cubin(prog, cubin.data());
  n.destroy(&prog);
  cudaLibrary_t lib = nullptr;
  cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e == cudaSuccess) e = cudaLibraryGetKernel(k, lib, name);
  if (e != cudaSuccess) {
    if (log) *log = std::string("loading the compiled kernel: ") + cudaGetErrorString(e);
    return false;
  }
  std::lock_guard<std::mutex> g(g_cache_mu);
  g_cache[key] = *k;
  return true;
}

}  // namespace lmf
