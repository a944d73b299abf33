// lmf_jit.cu -- source generator and NVRTC driver for the plan-specialised
// root scan (see lmf_jit.h).
#include "lmf_jit.h"

#include <dlfcn.h>
#include <nvrtc.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <functional>
#include <map>
#include <atomic>
#include <mutex>
#include <set>
#include <thread>
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

// category views, per-row tables and omega accumulators of one root row (every
// lane of the warp runs this code); cat(i) is the expression of row category i
void gen_grouped(std::ostringstream& o, const RootParams& rp, const std::vector<DirectAgg>& direct,
                 const std::function<std::string(int)>& cat) {
  const bool unit_w = rp.unit_w != 0;
  // category views
  for (int v = 0; v < rp.n_cv; ++v) {
    const CatView& C = rp.cv[v];
    o << "    {  // category view " << v << "\n"
      << "      const long long fk = live ? static_cast<long long>(fk" << C.grp << ") : -1ll;\n"
      << "      const int b = live ? " << cat(C.bcat) << " : 0;\n";
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
        << "            rp_red_shared_u32(res_hist + " << A.res_off << " + " << cat(A.cat[other])
        << (A.res_lanes ? " * 32 + lane" : "") << ", static_cast<uint32_t>(w));\n"
        << "          } else {\n"
        << "            rp_direct_add(p, p.dir[" << d << "], static_cast<int64_t>(" << cat(A.cat[0]) << ") * "
        << A.dom[1] << " + " << cat(A.cat[1]) << ", crow, w, cache);\n"
        << "          }\n        }\n      } else {\n        " << gl << "\n      }\n";
    } else if (count_pair && A.res_off < 0 && !A.runs) {
      o << "      if (live) {\n        const int a = " << cat(A.cat[0]) << ", b = " << cat(A.cat[1]) << ";\n";
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
  gen_grouped(o, rp, direct, [](int i) { return "crow[" + std::to_string(i) + "]"; });
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

LeanShape lean_shape(const RootParams& rp, bool direct_z) {
  LeanShape L;
  L.mpx = rp.gram_n > 4 ? (rp.gram_n + 3) / 4 * 4 : 4;
  for (int i = 0; i < kMaxZ; ++i) {
    L.col_of_z[i] = -1;
    L.col_scale[i] = 0.f;
  }
  L.col_of_z[0] = 0;  // the count (z[0] = 1 on a live row)
  L.col_scale[0] = 1.f;
  L.ncol = 1;
  auto add_cols = [&](const RevView& R) {
    for (int s = 0; s < R.n_slot; ++s) {
      const int z = R.slot_z[s];
      if (L.col_of_z[z] >= 0) continue;
      L.col_of_z[z] = L.ncol;
      L.col_scale[L.ncol] = R.slot_scale[s];
      ++L.ncol;
    }
  };
  for (int r = 0; r < rp.n_rv; ++r)  // bulk views first: their slots can be the row's first columns
    if (rp.rv[r].mode == kRvBulk) add_cols(rp.rv[r]);
  for (int r = 0; r < rp.n_rv; ++r)
    if (rp.rv[r].mode != kRvBulk) add_cols(rp.rv[r]);
  L.zi_ld = (L.ncol + 1) & ~1;
  for (int r = 0; r < rp.n_rv; ++r) {
    const RevView& R = rp.rv[r];
    L.stage_at[r] = -1;
    if (R.mode == kRvBulk) {
      bool prefix = R.stride <= L.zi_ld;
      for (int s = 0; s < R.n_slot && prefix; ++s) prefix = L.col_of_z[R.slot_z[s]] == 1 + s;
      if (prefix) {
        L.stage_at[r] = -2;
      } else {
        L.stage_at[r] = L.stage_w;
        L.stage_w += R.stride;
      }
    } else if (R.mode == kRvResident) {
      L.racc = (1 + R.n_slot + 31) / 32;
    }
  }
  L.zf_ld = direct_z ? rp.m : 0;
  L.cat_w = rp.n_direct > 0 ? std::max(1, rp.n_rowcat) : 0;
  uint32_t off = static_cast<uint32_t>(kLeanT * L.zi_ld * 8);
  L.xg_off = off;
  off += static_cast<uint32_t>(kLeanT * L.mpx * 4);
  L.zf_off = off;
  off += static_cast<uint32_t>(kLeanT * L.zf_ld * 4);
  off = (off + 15u) & ~15u;
  L.stage_off = off;
  off += static_cast<uint32_t>(kLeanT * L.stage_w * 8);
  L.cat_off = off;
  off += static_cast<uint32_t>(kLeanT * L.cat_w * 4);
  // the counters live across tiles: after the row Gram's fold staging, which
  // reuses the start of the per-tile scratch
  L.cache_off = std::max<uint32_t>((off + 15u) & ~15u, static_cast<uint32_t>(kLeanFoldStage));
  L.smem = L.cache_off + static_cast<size_t>(rp.cache_cells + rp.res_cells) * 4;
  return L;
}

std::string jit_lean_source(const RootParams& rp, const std::vector<DirectAgg>& direct, int min_ctas) {
  bool direct_z = false;
  for (int d = 0; d < rp.n_direct; ++d) direct_z = direct_z || direct[d].z >= 0;
  const LeanShape L = lean_shape(rp, direct_z);
  std::ostringstream o;
  o << "// plan-specialised key-level root scan (generated)\n#include \"lmf_root_lean.cuh\"\nnamespace lmf {\n";
  // record word -> column of the fixed-point tile, for the views summed in
  // warps (word 0, the count, is column 0)
  int res_rv = -1;
  for (int r = 0; r < rp.n_rv; ++r) {
    const RevView& R = rp.rv[r];
    if (R.mode == kRvResident) res_rv = r;
    if (R.mode == kRvBulk) continue;
    const int nw = 1 + R.n_slot, n = (nw + 31) / 32 * 32;
    o << "__device__ const int8_t kLc" << r << "[" << n << "] = {";
    for (int s = 0; s < n; ++s) o << (s == 0 || s >= nw ? 0 : L.col_of_z[R.slot_z[s - 1]]) << (s + 1 < n ? "," : "");
    o << "};\n";
  }
  // what the row pass needs from the records: every z index of a column, of
  // the row Gram or of a per-row table; every category a view or table reads
  std::vector<char> need_z(kMaxZ, 0), need_c(kMaxCat, 0);
  auto fixed = [&](int z) { return z > 0 && z < kMaxZ && rp.fix_of_z[z] >= 0; };
  for (int z = 1; z < rp.m; ++z)
    if ((L.col_of_z[z] >= 0 && !fixed(z)) || (z >= rp.gram_off && z < rp.gram_off + rp.gram_n) || L.zf_ld > 0)
      need_z[z] = 1;
  for (int v = 0; v < rp.n_cv; ++v) need_c[rp.cv[v].bcat] = 1;
  for (int d = 0; d < rp.n_direct; ++d)
    for (int q = 0; q < direct[d].n_gb; ++q) need_c[direct[d].cat[q]] = 1;
  if (rp.n_direct > 0)
    for (int i = 0; i < rp.n_rowcat; ++i) need_c[i] = 1;
  o << "struct JitLeanPass {\n"
    << "  static constexpr int kZiLd = " << L.zi_ld << ", kMpx = " << L.mpx << ", kZfLd = " << L.zf_ld
    << ", kStageW = " << L.stage_w << ", kCatW = " << L.cat_w << ", kRacc = " << L.racc << ";\n"
    << "  static constexpr bool kResident = " << ((res_rv >= 0 || rp.res_cells > 0) ? "true" : "false") << ";\n"
    << "  static constexpr uint32_t kXgOff = " << L.xg_off << "u, kZfOff = " << L.zf_off << "u, kStageOff = "
    << L.stage_off << "u, kCatOff = " << L.cat_off << "u, kCacheOff = " << L.cache_off << "u;\n"
    ;
  // the root row's own columns (foreign keys, features, root categories),
  // loaded one tile ahead of their use
  const int n_rc = rp.n_rcat;
  o << "  struct Row {\n    int32_t fk[" << std::max(1, rp.n_grp) << "];\n    float x[" << std::max(1, rp.n_x)
    << "];\n    int32_t rc[" << std::max(1, n_rc) << "];\n  };\n"
    << "  static __device__ __forceinline__ void load(const RootParams& p, int64_t row, Row& r) {\n"
    << "    if (row >= p.N) return;\n";
  // the root's columns are read once per launch: streaming loads (evict first)
  for (int i = 0; i < rp.n_x; ++i) {
    if (rp.x[i].dtype == 2)
      o << "    r.x[" << i << "] = static_cast<float>(__ldcs(static_cast<const double*>(p.x[" << i << "].p) + row));\n";
    else
      o << "    r.x[" << i << "] = __ldcs(static_cast<const float*>(p.x[" << i << "].p) + row);\n";
  }
  for (int g = 0; g < rp.n_grp; ++g) o << "    r.fk[" << g << "] = __ldcs(p.grp[" << g << "].fk + row);\n";
  for (int i = 0; i < n_rc; ++i) o << "    r.rc[" << i << "] = __ldcs(p.rcat[" << i << "] + row);\n";
  o << "  }\n"
    << "  static __device__ __forceinline__ long long run(const RootParams& p, int64_t row, const Row& r, long long* zi,\n"
       "      float* xg, float* zrow, int32_t* crow, uint32_t* cache, uint32_t* res_hist, long long res_key,\n"
       "      long long* racc, unsigned long long* stage) {\n"
       "    const int lane = threadIdx.x & 31;\n"
       "    long long w = 0;\n";
  for (int g = 0; g < rp.n_grp; ++g) o << "    int32_t fk" << g << " = -1;\n";
  for (int i = 1; i < rp.m; ++i) o << "    float z" << i << " = 0.f;\n";
  for (int i = 0; i < rp.n_rowcat; ++i) o << "    int32_t c" << i << " = 0;\n";
  // the row's earlier bulk reductions read its fixed-point row: wait for them
  // before anything writes it
  bool any_bulk = false;
  for (int r = 0; r < rp.n_rv; ++r) any_bulk = any_bulk || rp.rv[r].mode == kRvBulk;
  if (any_bulk) o << "    lean_bulk_wait_read();\n";
  o << "    if (row < p.N) {\n      w = 1;\n";
  for (int i = 0; i < rp.n_x; ++i) o << "      z" << 1 + i << " = r.x[" << i << "];\n";
  for (int g = 0; g < rp.n_grp; ++g) {
    const GroupDesc& G = rp.grp[g];
    const int nw = G.n_cnt + G.n_mu + G.n_cat;
    o << "      {\n        const int32_t fk = r.fk[" << g << "];\n"
      << "        fk" << g << " = fk;\n"
      << "        if (fk < 0 || fk >= " << G.K << ") {\n          w = 0;\n        } else {\n"
      << "          const uint4* rec = reinterpret_cast<const uint4*>(p.grp[" << g
      << "].rec + static_cast<int64_t>(fk) * " << G.stride << ");\n";
    for (int q = 0; q < (nw + 3) / 4; ++q) {
      bool any = false;
      for (int e = 0; e < 4; ++e) {
        const int wd = 4 * q + e;
        if (wd < G.n_cnt) any = true;
        else if (wd < G.n_cnt + G.n_mu) any = any || need_z[rp.grp_zoff[g] + wd - G.n_cnt];
        else if (wd < nw) any = any || need_c[rp.grp_catoff[g] + wd - G.n_cnt - G.n_mu];
      }
      if (!any) continue;
      o << "          {\n          const uint4 v = __ldg(rec + " << q << ");\n";
      const char* comp[4] = {"v.x", "v.y", "v.z", "v.w"};
      for (int e = 0; e < 4; ++e) {
        const int wd = 4 * q + e;
        if (wd < G.n_cnt) {
          o << "          w *= static_cast<long long>(" << comp[e] << ");\n";
        } else if (wd < G.n_cnt + G.n_mu) {
          const int z = rp.grp_zoff[g] + wd - G.n_cnt;
          if (need_z[z]) o << "          z" << z << " = __uint_as_float(" << comp[e] << ");\n";
        } else if (wd < nw) {
          const int c = rp.grp_catoff[g] + wd - G.n_cnt - G.n_mu;
          if (need_c[c]) o << "          c" << c << " = static_cast<int32_t>(" << comp[e] << ");\n";
        }
      }
      o << "          }\n";
    }
    // the fixed-point images of the group's means the views sum
    std::vector<int> fzs;
    for (int z = rp.grp_zoff[g]; z < rp.grp_zoff[g] + G.n_mu; ++z)
      if (fixed(z)) fzs.push_back(z);
    if (!fzs.empty()) {
      int fs = 0;
      for (int z : fzs) fs = std::max(fs, rp.fix_of_z[z] + 1);
      fs = (fs + 1) & ~1;
      o << "          const uint4* fx = reinterpret_cast<const uint4*>(p.grp[" << g
        << "].fix + static_cast<int64_t>(fk) * " << fs << ");\n";
      for (int q = 0; q < fs / 2; ++q) {
        std::vector<int> in_q;
        for (int z : fzs)
          if (rp.fix_of_z[z] / 2 == q) in_q.push_back(z);
        if (in_q.empty()) continue;
        o << "          {\n          const uint4 f = __ldg(fx + " << q << ");\n";
        for (int z : in_q)  // straight into the row's fixed-point tile row (no register held)
          o << "          reinterpret_cast<unsigned long long*>(zi)[" << L.col_of_z[z] << "] = (static_cast<unsigned long long>("
            << (rp.fix_of_z[z] % 2 ? "f.w" : "f.y") << ") << 32) | " << (rp.fix_of_z[z] % 2 ? "f.z" : "f.x") << ";\n";
        o << "          }\n";
      }
    }
    o << "        }\n      }\n";
  }
  for (int i = 0; i < rp.n_rcat; ++i) {
    const int c = rp.n_rowcat - rp.n_rcat + i;
    o << "      {\n        int32_t v = r.rc[" << i << "];\n"
      << "        if (v < 0 || v >= " << rp.rcat_dom[i] << ") {\n"
      << "          atomicOr(p.status, kStatusCatRange);\n          v = 0;\n        }\n"
      << "        c" << c << " = v;\n      }\n";
  }
  o << "    }\n    const bool live = w != 0;\n";
  for (int i = 1; i < rp.m; ++i) o << "    z" << i << " = live ? z" << i << " : 0.f;\n";
  // the fixed-point row: column 0 the count, then each value at its scale
  // (exact: a power-of-two scaling rounded to an integer)
  std::vector<int> z_of_col(L.ncol, 0);
  for (int z = 0; z < kMaxZ; ++z)
    if (L.col_of_z[z] >= 0) z_of_col[L.col_of_z[z]] = z;
  auto col_fixed = [&](int c) { return c > 0 && c < L.ncol && fixed(z_of_col[c]); };
  auto col_expr = [&](int c) -> std::string {
    if (c == 0) return "(live ? 1ull : 0ull)";
    if (c >= L.ncol) return "0ull";
    const int z = z_of_col[c];
    int e2 = 0;
    std::frexp(L.col_scale[c], &e2);  // the scale is 2^(e2 - 1)
    return "static_cast<unsigned long long>(lean_fx(z" + std::to_string(z) + ", " + std::to_string(e2 - 1) + "))";
  };
  // (the fixed-point images of means were stored as they arrived; a row that
  // does not join clears them)
  for (int c = 0; c < L.zi_ld; c += 2) {
    if (!col_fixed(c) && !col_fixed(c + 1)) {
      o << "    reinterpret_cast<ulonglong2*>(zi)[" << c / 2 << "] = make_ulonglong2(" << col_expr(c) << ", "
        << col_expr(c + 1) << ");\n";
      continue;
    }
    for (int e = c; e < c + 2; ++e)
      if (!col_fixed(e)) o << "    reinterpret_cast<unsigned long long*>(zi)[" << e << "] = " << col_expr(e) << ";\n";
  }
  {
    bool anyf = false;
    for (int c = 0; c < L.zi_ld; ++c) anyf = anyf || col_fixed(c);
    if (anyf) {
      o << "    if (!live) {\n";
      for (int c = 0; c < L.zi_ld; ++c)
        if (col_fixed(c)) o << "      reinterpret_cast<unsigned long long*>(zi)[" << c << "] = 0ull;\n";
      o << "    }\n";
    }
  }
  auto zv = [&](int i) { return i < rp.m ? "z" + std::to_string(i) : std::string("0.f"); };
  for (int c = 0; c < L.mpx; c += 4)
    o << "    *reinterpret_cast<float4*>(xg + " << c << ") = make_float4(" << zv(rp.gram_off + c) << ", "
      << zv(rp.gram_off + c + 1) << ", " << zv(rp.gram_off + c + 2) << ", " << zv(rp.gram_off + c + 3) << ");\n";
  if (L.zf_ld > 0) {
    o << "    zrow[0] = live ? 1.f : 0.f;\n";
    for (int i = 1; i < rp.m; ++i) o << "    zrow[" << i << "] = z" << i << ";\n";
  }
  if (rp.n_direct > 0)
    for (int i = 0; i < rp.n_rowcat; ++i) o << "    crow[" << i << "] = c" << i << ";\n";
  // bulk reverse views: one bulk reduction of the row's record
  for (int r = 0; r < rp.n_rv; ++r) {
    const RevView& R = rp.rv[r];
    if (R.mode != kRvBulk) continue;
    const int nw = 1 + R.n_slot;
    o << "    if (live) {  // reverse view " << r << ": the row's record, one bulk reduction\n";
    std::string src = "zi";
    if (L.stage_at[r] != -2) {
      src = "st";
      o << "      unsigned long long* st = stage + " << L.stage_at[r] << ";\n";
      auto word = [&](int wd) -> std::string {
        if (wd == 0) return "1ull";
        if (wd >= nw) return "0ull";
        return "static_cast<unsigned long long>(zi[" + std::to_string(L.col_of_z[R.slot_z[wd - 1]]) + "])";
      };
      for (int wd = 0; wd < R.stride; wd += 2)
        o << "      reinterpret_cast<ulonglong2*>(st)[" << wd / 2 << "] = make_ulonglong2(" << word(wd) << ", "
          << word(wd + 1) << ");\n";
    }
    o << "      lean_bulk_add(reinterpret_cast<unsigned long long*>(p.rv[" << r << "].hist) + static_cast<int64_t>(fk"
      << R.grp << ") * " << R.stride << ", reinterpret_cast<const unsigned long long*>(" << src << "), "
      << R.stride * 8 << ");\n    }\n";
  }
  if (rp.res_cells > 0)
    o << "    const long long fres = (live && res_key >= 0) ? static_cast<long long>(fk" << rp.res_grp << ") : -2ll;\n";
  else
    o << "    const long long fres = -2ll;\n";
  o << "    __syncwarp();  // the warp's rows are in shared memory\n";
  gen_grouped(o, rp, direct, [](int i) { return "c" + std::to_string(i); });
  // reverse views summed in warps.  One view in runs whose record is the
  // first columns of the tile row (at most 32 words) is reduced in place, after
  // every other reader of the tile: each run's sums are written into the run's
  // last row and that row's thread adds the record with one bulk reduction
  int inplace = -1;
  for (int r = 0; r < rp.n_rv && inplace < 0; ++r) {
    const RevView& R = rp.rv[r];
    if (R.mode != kRvRuns || 1 + R.n_slot > 32 || R.stride > L.zi_ld) continue;
    bool prefix = true;
    for (int sl = 0; sl < R.n_slot && prefix; ++sl) prefix = L.col_of_z[R.slot_z[sl]] == 1 + sl;
    if (prefix) inplace = r;
  }
  for (int r = 0; r < rp.n_rv; ++r) {
    const RevView& R = rp.rv[r];
    const int nw = 1 + R.n_slot;
    if (R.mode == kRvBulk || r == inplace) continue;
    o << "    {  // reverse view " << r << (R.mode == kRvResident ? " (resident key)" : " (runs)") << "\n"
      << "      const long long fk = live ? static_cast<long long>(fk" << R.grp << ") : -1ll;\n"
      << "      const WarpRuns q = warp_runs(fk);\n"
      << "      unsigned long long* rec0 = reinterpret_cast<unsigned long long*>(p.rv[" << r << "].hist);\n"
      << "      const long long* ziw = zi - lane * kZiLd;\n";
    for (int c = 0; c * 32 < nw; ++c) {
      o << "      {\n        const int wd = " << 32 * c << " + lane;\n";
      if (R.mode == kRvResident)
        o << "        lean_rv_resident(q, fk, res_key, ziw, kZiLd, kLc" << r << "[wd], wd < " << nw << ", racc[" << c
          << "], rec0, " << R.stride << ", wd);\n";
      else
        o << "        lean_rv_runs(q, fk, ziw, kZiLd, kLc" << r << "[wd], wd < " << nw << ", rec0, " << R.stride
          << ", wd);\n";
      o << "      }\n";
    }
    o << "    }\n";
  }
  if (inplace >= 0) {
    const RevView& R = rp.rv[inplace];
    o << "    {  // reverse view " << inplace << " (runs, reduced in place)\n"
      << "      const long long fk = live ? static_cast<long long>(fk" << R.grp << ") : -1ll;\n"
      << "      const WarpRuns q = warp_runs(fk);\n"
      << "      lean_bulk_wait_read();  // this row's earlier bulk reductions have read the tile row\n"
      << "      __syncwarp();\n"
      << "      lean_rv_inplace(q, zi - lane * kZiLd, kZiLd, lane, lane < " << 1 + R.n_slot << ");\n"
      << "      __syncwarp();\n"
      << "      if (fk >= 0 && (lane == 31 || ((q.heads >> (lane + 1)) & 1u)))\n"
      << "        lean_bulk_add(reinterpret_cast<unsigned long long*>(p.rv[" << inplace << "].hist) + fk * " << R.stride
      << ", reinterpret_cast<const unsigned long long*>(zi), " << R.stride * 8 << ");\n"
      << "    }\n";
  }
  o << "    (void)lane;\n    (void)fres;\n    (void)stage;\n    (void)racc;\n    (void)cache;\n    (void)crow;\n"
       "    (void)zrow;\n    return w;\n  }\n";
  o << "  static __device__ __forceinline__ void flush_resident(const RootParams& p, long long* racc, long long key) {\n";
  if (res_rv >= 0) {
    const RevView& R = rp.rv[res_rv];
    const int nw = 1 + R.n_slot;
    o << "    const int lane = threadIdx.x & 31;\n"
      << "    unsigned long long* rec0 = reinterpret_cast<unsigned long long*>(p.rv[" << res_rv << "].hist);\n"
      << "#pragma unroll\n    for (int c = 0; c < kRacc; ++c) {\n      const int wd = c * 32 + lane;\n"
      << "      if (key >= 0 && wd < " << nw << " && racc[c] != 0)\n"
      << "        rp_red_u64(rec0 + key * " << R.stride << " + wd, static_cast<unsigned long long>(racc[c]));\n"
      << "      racc[c] = 0;\n    }\n";
  } else {
    o << "    (void)p;\n    (void)racc;\n    (void)key;\n";
  }
  o << "  }\n};\n}  // namespace lmf\n"
    << "extern \"C\" __global__ void __launch_bounds__(256, " << min_ctas
    << ") lmf_root_lean_jit(const __grid_constant__ lmf::RootParams p, int64_t n_tiles) {\n"
    << "  lmf::root_lean_body<lmf::JitLeanPass>(p, n_tiles);\n}\n";
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
  if (const char* dir = std::getenv("LMF_JIT_DUMP")) {  // keep the generated source for inspection
    const std::string path = std::string(dir) + "/" + name + "_" + std::to_string(std::hash<std::string>{}(src)) + ".cu";
    if (FILE* f = std::fopen(path.c_str(), "w")) {
      std::fwrite(src.data(), 1, src.size(), f);
      std::fclose(f);
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

int jit_kernels_parallel(const std::vector<std::pair<std::string, const char*>>& jobs, int threads, int device) {
  // distinct jobs only: two threads compiling one source would both load it
  std::vector<size_t> todo;
  {
    std::set<std::string> seen;
    std::lock_guard<std::mutex> g(g_cache_mu);
    for (size_t i = 0; i < jobs.size(); ++i) {
      const std::string key = std::string(jobs[i].second) + '\n' + jobs[i].first;
      if (g_cache.count(key) || !seen.insert(key).second) continue;
      todo.push_back(i);
    }
  }
  std::atomic<size_t> next{0};
  std::atomic<int> done{0};
  auto work = [&]() {
    cudaSetDevice(device);
    for (size_t t; (t = next.fetch_add(1)) < todo.size();) {
      cudaKernel_t k = nullptr;
      std::string log;
      if (jit_kernel(jobs[todo[t]].first, jobs[todo[t]].second, &k, &log)) done.fetch_add(1);
    }
  };
  const int nt = std::max(1, std::min<int>(threads, static_cast<int>(todo.size())));
  std::vector<std::thread> pool;
  for (int i = 1; i < nt; ++i) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  return done.load();
}

}  // namespace lmf
