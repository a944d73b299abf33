// Host-only check of the plan-time code generator (no GPU needed): builds
// plans of several shapes by hand, generates the plain and the tensor-core
// root-scan sources for each (and a tree pass), and compiles them for sm_103a
// with NVRTC.
// Used by tests/test_jit_codegen.py.  Exit status 0 when every source
// compiles; one line per compiled source on stdout.
#include "lmf_jit.cu"
#include "lmf_jit_tree.cu"

#include <cstdio>
#include <string>
#include <vector>

using namespace lmf;

namespace {

bool compile(const std::string& src, const char* what) {
  const Nvrtc& n = nvrtc();
  nvrtcProgram prog = nullptr;
  const int nh = static_cast<int>(sizeof(kJitHeaderNames) / sizeof(kJitHeaderNames[0]));
  if (n.create(&prog, src.c_str(), "check.cu", nh, kJitHeaderSrc, kJitHeaderNames) != NVRTC_SUCCESS) return false;
  const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "--device-as-default-execution-space"};
  const nvrtcResult rc = n.compile(prog, 3, opts);
  size_t cs = 0;
  if (rc == NVRTC_SUCCESS) n.cubin_size(prog, &cs);
  if (rc != NVRTC_SUCCESS || cs == 0) {
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) n.get_log(prog, &log[0]);
    std::printf("FAIL %s: %s\n%s\n", what, n.err(rc), log.c_str());
    n.destroy(&prog);
    return false;
  }
  n.destroy(&prog);
  std::printf("ok %s (%zu bytes of cubin)\n", what, cs);
  return true;
}

// a snowflake-like root: 8 features, three probe groups with means and categories
RootParams base(bool unit_w) {
  RootParams rp{};
  rp.N = 100000;
  rp.n_x = 8;
  for (int i = 0; i < rp.n_x; ++i) rp.x[i].dtype = 1;
  const int nmu[3] = {12, 5, 5}, ncat[3] = {4, 3, 3};
  int zoff = 1 + rp.n_x, coff = 0;
  rp.n_grp = 3;
  for (int g = 0; g < 3; ++g) {
    GroupDesc& G = rp.grp[g];
    G.K = 1000 * (g + 1);
    G.n_cnt = 1;
    G.n_mu = nmu[g];
    G.n_cat = ncat[g];
    G.stride = (G.n_cnt + G.n_mu + G.n_cat + 3) / 4 * 4;
    rp.grp_zoff[g] = zoff;
    rp.grp_catoff[g] = coff;
    zoff += nmu[g];
    coff += ncat[g];
  }
  rp.m = zoff;
  rp.n_rowcat = coff;
  rp.n_rv = 3;
  for (int r = 0; r < 3; ++r) {
    rp.rv[r].grp = r;
    rp.rv[r].n_slot = 19 + 3 * r;
    for (int s = 0; s < rp.rv[r].n_slot; ++s) {
      rp.rv[r].slot_z[s] = static_cast<int16_t>(s % rp.m);
      rp.rv[r].slot_scale[s] = 1048576.f;
    }
  }
  rp.unit_w = unit_w ? 1 : 0;
  rp.hot_h = 8;
  for (int i = 0; i < kMaxCat; ++i) rp.hot_lut_off[i] = i * 64;
  return rp;
}

DirectAgg pair(int a, int b, int dom_a, int dom_b) {
  DirectAgg d{};
  d.n_gb = 2;
  d.cat[0] = a;
  d.cat[1] = b;
  d.dom[0] = dom_a;
  d.dom[1] = dom_b;
  d.z = -1;
  d.cache_off = -1;
  d.res_off = -1;
  return d;
}

}  // namespace

int main() {
  if (!jit_available()) {
    std::printf("FAIL NVRTC not available\n");
    return 1;
  }
  int bad = 0;
  auto check = [&](const RootParams& rp, int mp, const std::vector<DirectAgg>& dir, const char* name, bool tc) {
    bad += !compile(jit_plain_source(rp, mp, dir, 3), (std::string(name) + " plain").c_str());
    if (tc) bad += !compile(jit_tc_source(rp, dir), (std::string(name) + " tc").c_str());
  };

  {  // sorted snowflake: resident key, hot cache, lane-private and shared resident tables, runs
    RootParams rp = base(true);
    rp.res_grp = 2;
    rp.res_cells = 2000;
    rp.cache_cells = 128;
    rp.fold = 8;
    std::vector<DirectAgg> dir;
    for (int d = 0; d < 6; ++d) {
      DirectAgg a = pair(d % 4, 4 + d % 6, 20, 30);
      a.cache_off = d < 2 ? 64 * d : -1;
      if (d >= 2) {
        a.res_off = 100 * d;
        a.res_q = 1;
        a.res_word = 18;
        a.res_n = 20;
        a.res_lanes = d == 3;
      }
      a.runs = d == 5;
      dir.push_back(a);
    }
    DirectAgg s{};  // SUM(z) grouped by a root-side category, with runs
    s.n_gb = 1;
    s.cat[0] = 1;
    s.dom[0] = 5;
    s.z = 3;
    s.scale = 1024.f;
    s.cache_off = -1;
    s.res_off = -1;
    s.runs = 1;
    dir.push_back(s);
    rp.n_cv = 3;
    for (int v = 0; v < 3; ++v) {
      CatView& C = rp.cv[v];
      C.grp = v;
      C.bcat = 5 + v;
      C.dom = 17 + v;
      C.res_off = v == 2 ? 1500 : -1;
      C.runs = v == 1;
    }
    rp.n_direct = static_cast<int>(dir.size());
    check(rp, 32, dir, "snowflake", true);
  }
  {  // fanning-out joins: w above 1, omega accumulators, no resident key
    RootParams rp = base(false);
    rp.n_om = 2;
    std::vector<DirectAgg> dir = {pair(0, 5, 7, 9)};
    rp.n_direct = 1;
    check(rp, 32, dir, "fanout", false);
  }
  {  // more per-row tables than ride in the parameters; FP64 features; root categories
    RootParams rp = base(true);
    rp.x[0].dtype = 2;
    rp.x[5].dtype = 2;
    rp.n_rcat = 2;
    rp.rcat_dom[0] = 7;
    rp.rcat_dom[1] = 3;
    rp.n_rowcat += 2;
    std::vector<DirectAgg> dir;
    for (int d = 0; d < 110; ++d) {
      DirectAgg a = pair(d % 10, 10 + (d % 2), 11, 7);
      if (d % 3 == 0) {
        a.z = 2 + d % 5;
        a.scale = 4096.f;
      }
      dir.push_back(a);
    }
    rp.n_direct = static_cast<int>(dir.size());
    check(rp, 32, dir, "many-tables", true);
  }
  {  // wide z (two 32-feature blocks): plain form only
    RootParams rp = base(true);
    rp.n_x = 30;
    for (int i = 0; i < rp.n_x; ++i) rp.x[i].dtype = 1;
    int zoff = 1 + rp.n_x;
    for (int g = 0; g < rp.n_grp; ++g) {
      rp.grp_zoff[g] = zoff;
      zoff += rp.grp[g].n_mu;
    }
    rp.m = zoff;
    for (int r = 0; r < rp.n_rv; ++r)
      for (int s = 0; s < rp.rv[r].n_slot; ++s) rp.rv[r].slot_z[s] = static_cast<int16_t>((s * 3) % rp.m);
    check(rp, 64, {}, "wide", false);
  }
  {  // key-level form of the sorted snowflake: a bulk, a runs and a resident reverse view
    RootParams rp = base(true);
    rp.lean = 1;
    rp.gram_off = 1;
    rp.gram_n = rp.n_x;
    rp.res_grp = 2;
    rp.res_cells = 1800;
    const int nslot[3] = {8, 20, 25}, mode[3] = {kRvBulk, kRvRuns, kRvResident};
    for (int r = 0; r < 3; ++r) {
      RevView& R = rp.rv[r];
      R.n_slot = nslot[r];
      for (int s = 0; s < R.n_slot; ++s) R.slot_z[s] = static_cast<int16_t>(1 + s);
      R.stride = (1 + R.n_slot + 1) & ~1;
      R.hstride = R.rstride = R.stride;
      R.mode = mode[r];
    }
    rp.res_rv = 2;
    // the means of groups 0 and 1 come as fixed-point images from their fix records
    for (int z = 0; z < kMaxZ; ++z) rp.fix_of_z[z] = -1;
    for (int g = 0; g < 2; ++g)
      for (int j = 0; j < rp.grp[g].n_mu; ++j) rp.fix_of_z[rp.grp_zoff[g] + j] = static_cast<int16_t>(j);
    rp.n_cv = 4;
    for (int v = 0; v < 4; ++v) {
      CatView& C = rp.cv[v];
      C.grp = v < 2 ? 1 : 2;
      C.bcat = v;
      C.dom = 50 + v;
      C.res_off = v < 2 ? -1 : 400 * v;
    }
    bad += !compile(jit_lean_source(rp, {}, 3), "key-level snowflake");
    // random order: every view summed per run, root categories and per-row tables with features,
    // every value converted in the row pass
    for (int z = 0; z < kMaxZ; ++z) rp.fix_of_z[z] = -1;
    rp.res_cells = 0;
    rp.res_rv = -1;
    for (int r = 0; r < 3; ++r) rp.rv[r].mode = kRvRuns;
    rp.n_cv = 0;
    rp.n_rcat = 1;
    rp.rcat_dom[0] = 9;
    rp.n_rowcat += 1;
    std::vector<DirectAgg> dir = {pair(0, rp.n_rowcat - 1, 11, 9)};
    DirectAgg s{};
    s.n_gb = 1;
    s.cat[0] = rp.n_rowcat - 1;
    s.dom[0] = 9;
    s.z = 4;
    s.scale = 1024.f;
    s.cache_off = -1;
    s.res_off = -1;
    dir.push_back(s);
    rp.n_direct = static_cast<int>(dir.size());
    bad += !compile(jit_lean_source(rp, dir, 2), "key-level random");
  }
  {  // the tree pass of a snowflake root: two groups of nodes, a decision tree over their predicates
    RootParams rp = base(true);
    rp.x[2].dtype = 2;
    TreeJitSpec t;
    t.mp = 32;
    t.preds = {{}, {{3, 0, 0.5f}}, {{3, 1, 0.5f}}, {{3, 1, 0.5f}, {12, 0, -1.25e-3f}}, {{3, 1, 0.5f}, {12, 1, -1.25e-3f}}};
    // group 0: the root node alone; group 1: z3 <= 0.5 -> node 1, else one of nodes 2..4
    t.droot = {0, 1};
    t.dt = {{0, 1, 0.f, 0, 1}, {3, 0, 0.5f, 2, 3}, {0, 1, 0.f, 1, 1}, {0, 1, 0.f, 2, 3}};
    t.cand = {0, 1, 3, 4, 2};
    bad += !compile(jit_tree_source(rp, t), "tree pass");
    // a decision tree too large to spell out: the node search over the device tables
    t.dt.resize(5000, TreeJitSpec::Entry{0, 1, 0.f, 0, 1});
    const std::string big = jit_tree_source(rp, t);
    if (big.find("tree_node_of(d, g, zrow)") == std::string::npos) {
      std::printf("FAIL large tree not searched through the tables\n");
      ++bad;
    }
    bad += !compile(big, "tree pass (table search)");
  }
  {  // a root without probe groups: features only
    RootParams rp{};
    rp.N = 1000;
    rp.n_x = 5;
    rp.m = 6;
    rp.unit_w = 1;
    for (int i = 0; i < rp.n_x; ++i) rp.x[i].dtype = 1;
    check(rp, 16, {}, "root-only", false);
  }
  return bad ? 1 : 0;
}
