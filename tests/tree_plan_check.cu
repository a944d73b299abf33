// Host-only check of the tree planner (no GPU needed): the decomposition of a
// batch of threshold-filtered aggregates into nodes, split attributes and the
// decision tree that finds a row's node.  Used by tests/test_tree_plan.py.
// Exit status 0 when every check holds; one line per check on stdout.
//
// With `--emit DIR` it instead writes, for plans of several shapes, the tree
// pass source generated for the plan (case_K.cu) and a set of points with the
// node each group's brute-force search gives them (case_K.txt: "G P NZ", then
// per point NZ float bit patterns in hex and G node ids, 65535 for none), so
// that the test can compile the generated node search on the host and
// compare; and the source generated for the root layouts of tree_row_cases.h
// (row_case_K.cu), whose row pass tests/tree_row_host.cu checks.
#include "lmf_tree.cu"
#include "lmf_jit_tree.cu"
#include "tree_row_cases.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace lmf;

namespace {

int bad = 0;

void expect(bool ok, const char* what) {
  std::printf("%s %s\n", ok ? "ok" : "FAIL", what);
  bad += !ok;
}

// one level of a complete binary tree of depth `depth` in heap order: internal
// entry k splits on feature f(k % nf) at threshold 0.125 k, its children are
// 2k+1 (<=) and 2k+2 (>); every leaf becomes a node with three thresholds of
// one split attribute, SUM(y) each (the aggregates of a tree level, Sec. 5)
std::vector<TreeAggIn> level(int depth, int nf, std::map<std::string, int>* zidx) {
  for (int i = 0; i < nf; ++i) (*zidx)["f" + std::to_string(i)] = 1 + i;
  (*zidx)["y"] = nf + 1;
  const int n_int = (1 << depth) - 1;
  std::vector<TreeAggIn> in;
  for (int leaf = 0; leaf <= n_int; ++leaf) {
    std::vector<TreeFactorIn> path;
    for (int i = n_int + leaf; i > 0;) {
      const int k = (i - 1) / 2;
      path.push_back({"f" + std::to_string(k % nf), i == 2 * k + 1 ? LMF_LE : LMF_GT, 0, 0.125 * k});
      i = k;
    }
    for (int j = 0; j < 3; ++j) {
      TreeAggIn a;
      a.factors = path;
      a.factors.push_back({"f" + std::to_string(nf - 1 - leaf % 7), LMF_LE, 0, 10.0 + j});
      a.factors.push_back({"y", LMF_POW, 1, 0.0});
      in.push_back(a);
    }
  }
  return in;
}

// the node a point z reaches through the decision tree of group g (host copy
// of the device search)
int dt_node(const TreePlanImpl& T, int g, const std::vector<float>& z) {
  int i = T.droot[g];
  while (!T.dt[i].leaf) i = z[T.dt[i].z] <= T.dt[i].thr ? T.dt[i].left : T.dt[i].right;
  const TreeDt& e = T.dt[i];
  for (int c = e.left; c < e.left + e.right; ++c) {
    const int n = T.dcand[c];
    bool ok = true;
    for (const TreePred& p : T.nodes[n]) ok = ok && (p.op == 0 ? z[p.z] <= p.thr : z[p.z] > p.thr);
    if (ok) return n;
  }
  return -1;
}

// random conjunctions of 1-3 predicates over four features, thresholds from
// a small grid (so that nodes share predicates and overlap), each node with
// three thresholds of a fifth attribute as its split
std::vector<TreeAggIn> random_nodes(int n_nodes, uint64_t seed, std::map<std::string, int>* zidx) {
  for (int i = 0; i < 5; ++i) (*zidx)["f" + std::to_string(i)] = 1 + i;
  (*zidx)["y"] = 6;
  uint64_t x = seed;
  auto next = [&]() {
    x = x * 6364136223846793005ull + 1442695040888963407ull;
    return static_cast<int>(x >> 33);
  };
  const double grid[5] = {-1.0, -0.5, 0.0, 0.5, 1.0};
  std::vector<TreeAggIn> in;
  for (int k = 0; k < n_nodes; ++k) {
    std::vector<TreeFactorIn> node;
    const int np = 1 + next() % 3;
    for (int j = 0; j < np; ++j)
      node.push_back({"f" + std::to_string(next() % 4), next() % 2 ? LMF_LE : LMF_GT, 0, grid[next() % 5]});
    for (int j = 0; j < 3; ++j) {
      TreeAggIn a;
      a.factors = node;
      a.factors.push_back({"f4", LMF_LE, 0, 10.0 + j});
      a.factors.push_back({"y", LMF_POW, 1, 0.0});
      in.push_back(a);
    }
  }
  return in;
}

bool emit_case(const std::string& dir, int k, const std::vector<TreeAggIn>& in, const std::map<std::string, int>& zidx) {
  TreePlan tp;
  std::string msg;
  if (tree_plan(in, zidx, &tp, &msg) != LMF_OK) {
    std::printf("FAIL plan of case %d: %s\n", k, msg.c_str());
    return false;
  }
  const TreePlanImpl& T = *tp.impl;
  TreeJitSpec spec;
  tree_jit_spec(&tp, &spec);
  RootParams rp{};
  const std::string src = jit_tree_source(rp, spec);
  FILE* f = std::fopen((dir + "/case_" + std::to_string(k) + ".cu").c_str(), "w");
  if (!f) return false;
  std::fwrite(src.data(), 1, src.size(), f);
  std::fclose(f);
  // points: thresholds, their neighbours and uniform values on every coordinate
  std::vector<float> special;
  for (const auto& v : T.nodes)
    for (const TreePred& p : v) {
      special.push_back(p.thr);
      special.push_back(std::nextafter(p.thr, -INFINITY));
      special.push_back(std::nextafter(p.thr, INFINITY));
    }
  const int nz = static_cast<int>(zidx.size()) + 1, G = static_cast<int>(T.groups.size()), P = 4000;
  f = std::fopen((dir + "/case_" + std::to_string(k) + ".txt").c_str(), "w");
  if (!f) return false;
  std::fprintf(f, "%d %d %d\n", G, P, nz);
  uint64_t x = 977 + k;
  for (int t = 0; t < P; ++t) {
    std::vector<float> z(nz);
    for (auto& v : z) {
      x = x * 6364136223846793005ull + 1442695040888963407ull;
      const uint32_t r = static_cast<uint32_t>(x >> 32);
      v = (r & 1) && !special.empty() ? special[(r >> 1) % special.size()]
                                      : static_cast<float>((r >> 8) % 4096) / 1024.f - 2.f;
      uint32_t u;
      std::memcpy(&u, &v, 4);
      std::fprintf(f, "%08x ", u);
    }
    for (int g = 0; g < G; ++g) {
      int want = kNoNode, hits = 0;
      for (int n : T.groups[g]) {
        bool ok = true;
        for (const TreePred& p : T.nodes[n]) ok = ok && (p.op == 0 ? z[p.z] <= p.thr : z[p.z] > p.thr);
        if (ok) {
          want = n;
          ++hits;
        }
      }
      if (hits > 1) {
        std::printf("FAIL case %d: two nodes of group %d hold at one point\n", k, g);
        return false;
      }
      std::fprintf(f, "%d ", want);
    }
    std::fprintf(f, "\n");
  }
  std::fclose(f);
  std::printf("emitted case %d: %zu nodes, %d groups, %zu decision-tree entries\n", k, T.nodes.size(), G, T.dt.size());
  return true;
}

}  // namespace

// the cells of a g x g grid of bins on (f0, f1), edges 0.25 i - 5: mutually
// exclusive nodes whose predicates name different thresholds of one attribute
// (a cell with f0 <= a_3 does not mention a_20), three thresholds of a split
// attribute per cell
std::vector<TreeAggIn> grid(int g, std::map<std::string, int>* zidx) {
  for (int i = 0; i < 4; ++i) (*zidx)["f" + std::to_string(i)] = 1 + i;
  (*zidx)["y"] = 5;
  auto edge = [](int i) { return 0.25 * i - 5.0; };
  std::vector<TreeAggIn> in;
  for (int i = 0; i < g; ++i)
    for (int j = 0; j < g; ++j) {
      std::vector<TreeFactorIn> cell;
      if (i > 0) cell.push_back({"f0", LMF_GT, 0, edge(i)});
      if (i + 1 < g) cell.push_back({"f0", LMF_LE, 0, edge(i + 1)});
      if (j > 0) cell.push_back({"f1", LMF_GT, 0, edge(j)});
      if (j + 1 < g) cell.push_back({"f1", LMF_LE, 0, edge(j + 1)});
      for (int t = 0; t < 3; ++t) {
        TreeAggIn a;
        a.factors = cell;
        a.factors.push_back({"f2", LMF_LE, 0, 10.0 + t});
        a.factors.push_back({"y", LMF_POW, 1, 0.0});
        in.push_back(a);
      }
    }
  return in;
}

// every point finds through group g's decision tree the node a brute-force
// search over the group finds (points on, beside and between thresholds)
bool all_points_find_their_node(const TreePlanImpl& T, int nz, int points) {
  std::vector<float> special;
  for (const auto& v : T.nodes)
    for (const TreePred& p : v) {
      special.push_back(p.thr);
      special.push_back(std::nextafter(p.thr, -INFINITY));
      special.push_back(std::nextafter(p.thr, INFINITY));
    }
  uint64_t x = 4242;
  for (int t = 0; t < points; ++t) {
    std::vector<float> z(nz);
    for (auto& v : z) {
      x = x * 6364136223846793005ull + 1442695040888963407ull;
      const uint32_t r = static_cast<uint32_t>(x >> 32);
      v = (r & 1) && !special.empty() ? special[(r >> 1) % special.size()]
                                      : static_cast<float>((r >> 8) % 8192) / 512.f - 8.f;
    }
    for (int g = 0; g < (int)T.groups.size(); ++g) {
      int want = -1;
      for (int n : T.groups[g]) {
        bool ok = true;
        for (const TreePred& p : T.nodes[n]) ok = ok && (p.op == 0 ? z[p.z] <= p.thr : z[p.z] > p.thr);
        if (ok) want = n;
      }
      if (dt_node(T, g, z) != want) return false;
    }
  }
  return true;
}

int main(int argc, char** argv) {
  if (argc == 3 && std::string(argv[1]) == "--emit") {
    bool ok = true;
    {  // one complete level of depth 6: one group
      std::map<std::string, int> zidx;
      ok = ok && emit_case(argv[2], 0, level(6, 20, &zidx), zidx);
    }
    {  // the leaves of depths 2 and 3 of one tree: nested nodes, several groups
      std::map<std::string, int> zidx;
      std::vector<TreeAggIn> in = level(2, 20, &zidx);
      const std::vector<TreeAggIn> l3 = level(3, 20, &zidx);
      in.insert(in.end(), l3.begin(), l3.end());
      ok = ok && emit_case(argv[2], 1, in, zidx);
    }
    for (int k = 2; k < 6; ++k) {  // random overlapping conjunctions
      std::map<std::string, int> zidx;
      ok = ok && emit_case(argv[2], k, random_nodes(12 * k, 31 * k + 7, &zidx), zidx);
    }
    {  // a 30 x 30 grid of bins
      std::map<std::string, int> zidx;
      ok = ok && emit_case(argv[2], 6, grid(30, &zidx), zidx);
    }
    for (int k = 0; k < kTreeRowCases; ++k) {  // the row pass for the layouts of tree_row_cases.h
      const RootParams rp = tree_row_case(k);
      TreeJitSpec t;
      t.mp = (rp.m + 15) / 16 * 16;
      t.droot = {0};
      t.dt = {{0, 1, 0.f, 0, 0}};
      const std::string src = jit_tree_source(rp, t);
      FILE* f = std::fopen((std::string(argv[2]) + "/row_case_" + std::to_string(k) + ".cu").c_str(), "w");
      ok = ok && f != nullptr;
      if (f) {
        std::fwrite(src.data(), 1, src.size(), f);
        std::fclose(f);
      }
    }
    return ok ? 0 : 1;
  }
  for (int depth : {3, 6}) {
    std::map<std::string, int> zidx;
    const std::vector<TreeAggIn> in = level(depth, 20, &zidx);
    TreePlan tp;
    std::string msg;
    const lmf_status s = tree_plan(in, zidx, &tp, &msg);
    const std::string d = " (depth " + std::to_string(depth) + ")";
    expect(s == LMF_OK, ("plan" + d + " " + msg).c_str());
    if (s != LMF_OK) continue;
    const TreePlanImpl& T = *tp.impl;
    const size_t leaves = size_t(1) << depth;
    expect(T.nodes.size() == leaves, ("one node per leaf" + d).c_str());
    expect(T.groups.size() == 1, ("the leaves are one group of exclusive nodes" + d).c_str());
    // the leaves split into halves on their common ancestors' predicates: a
    // decision tree with one leaf per satisfiable node (a path that bounds one
    // feature twice can leave an empty interval; no row reaches such a node)
    std::vector<int> live;
    for (int nd = 0; nd < (int)T.nodes.size(); ++nd) {
      bool ok = true;
      for (const TreePred& p : T.nodes[nd]) {
        float lo, hi;
        node_interval(T.nodes[nd], p.z, &lo, &hi);
        ok = ok && lo < hi;
      }
      if (ok) live.push_back(nd);
    }
    std::vector<int32_t> cands(T.dcand.begin(), T.dcand.end());
    std::sort(cands.begin(), cands.end());
    expect(!live.empty() && T.dt.size() == 2 * live.size() - 1 && cands == std::vector<int32_t>(live.begin(), live.end()),
           ("decision tree of the level's size, every satisfiable node in one leaf" + d).c_str());
    int deepest = 0;
    std::vector<std::pair<int, int>> stack{{T.droot[0], 0}};
    while (!stack.empty()) {
      const auto [i, dd] = stack.back();
      stack.pop_back();
      deepest = std::max(deepest, dd);
      if (!T.dt[i].leaf) {
        stack.push_back({T.dt[i].left, dd + 1});
        stack.push_back({T.dt[i].right, dd + 1});
      }
    }
    expect(deepest <= depth, ("decision tree within the level's depth" + d).c_str());
    // every point reaches the one node whose predicates it satisfies
    uint64_t x = 12345;
    bool all = true;
    for (int t = 0; t < 20000 && all; ++t) {
      std::vector<float> z(zidx.size() + 1, 0.f);
      for (auto& v : z) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        v = static_cast<float>((x >> 40) % 1024) / 1024.f * 10.f - 1.f;
      }
      int want = -1, count = 0;
      for (int n = 0; n < (int)T.nodes.size(); ++n) {
        bool ok = true;
        for (const TreePred& p : T.nodes[n]) ok = ok && (p.op == 0 ? z[p.z] <= p.thr : z[p.z] > p.thr);
        if (ok) {
          want = n;
          ++count;
        }
      }
      all = count <= 1 && dt_node(T, 0, z) == want;
    }
    expect(all, ("every point finds its node" + d).c_str());
  }
  {  // a 40 x 40 grid of bins: one group, a tree of about log2(1600) levels
    std::map<std::string, int> zidx;
    const std::vector<TreeAggIn> in = grid(40, &zidx);
    TreePlan tp;
    std::string msg;
    const lmf_status s = tree_plan(in, zidx, &tp, &msg);
    expect(s == LMF_OK, ("plan (grid) " + msg).c_str());
    if (s == LMF_OK) {
      const TreePlanImpl& T = *tp.impl;
      expect(T.nodes.size() == 1600 && T.groups.size() == 1, "grid cells are one group of exclusive nodes");
      int deepest = 0;
      std::vector<std::pair<int, int>> stack{{T.droot[0], 0}};
      size_t leaves = 0, most = 0;
      while (!stack.empty()) {
        const auto [i, dd] = stack.back();
        stack.pop_back();
        deepest = std::max(deepest, dd);
        if (!T.dt[i].leaf) {
          stack.push_back({T.dt[i].left, dd + 1});
          stack.push_back({T.dt[i].right, dd + 1});
        } else {
          ++leaves;
          most = std::max(most, static_cast<size_t>(T.dt[i].right));
        }
      }
      std::printf("grid: %zu entries, %zu leaves, depth %d, at most %zu candidates per leaf\n", T.dt.size(), leaves,
                  deepest, most);
      expect(deepest <= 12 && most == 1 && T.dcand.size() == 1600, "grid decision tree of depth <= 12, one node per leaf");
      expect(all_points_find_their_node(T, 6, 20000), "every point finds its grid cell");
    }
  }
  {  // random batches: every aggregate's node, split threshold and moment are its own factors
    bool faithful = true;
    for (int trial = 0; trial < 20 && faithful; ++trial) {
      std::map<std::string, int> zidx;
      for (int i = 0; i < 6; ++i) zidx["f" + std::to_string(i)] = 1 + i;
      zidx["y"] = 7;
      uint64_t x = 1000 + trial;
      auto next = [&]() {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        return static_cast<uint32_t>(x >> 33);
      };
      const double grid_t[7] = {-1.5, -0.25, 0.0, 0.1, 0.75, 2.0, 1e-3};
      std::vector<TreeAggIn> in(1500);
      for (auto& a : in) {
        const int nt = 1 + next() % 5;
        for (int k = 0; k < nt; ++k) {
          const double t = next() % 4 ? grid_t[next() % 7] : (static_cast<double>(next()) / 4294967296.0 - 0.25) * 3.0;
          a.factors.push_back({"f" + std::to_string(next() % 6), next() % 2 ? LMF_LE : LMF_GT, 0, t});
        }
        switch (next() % 4) {
          case 1: a.factors.push_back({"y", LMF_POW, 1, 0.0}); break;
          case 2: a.factors.push_back({"y", LMF_POW, 2, 0.0}); break;
          case 3:
            a.factors.push_back({"f0", LMF_POW, 1, 0.0});
            a.factors.push_back({"y", LMF_POW, 1, 0.0});
            break;
          default: break;
        }
        // factors in any order
        for (size_t k = a.factors.size(); k > 1; --k) std::swap(a.factors[k - 1], a.factors[next() % k]);
      }
      TreePlan tp;
      std::string msg;
      if (tree_plan(in, zidx, &tp, &msg) != LMF_OK || tp.impl->outs.size() != in.size()) {
        faithful = false;
        break;
      }
      const TreePlanImpl& T = *tp.impl;
      for (size_t i = 0; i < in.size() && faithful; ++i) {
        const auto& o = T.outs[i];
        std::set<std::tuple<int, int, float>> want, got;
        std::vector<int> mono_want;
        for (const auto& f : in[i].factors) {
          if (f.kind == LMF_POW) {
            for (int e = 0; e < f.power; ++e) mono_want.push_back(zidx.at(f.attr));
          } else {
            want.insert({zidx.at(f.attr), f.kind == LMF_LE ? 0 : 1, round_down_f32(f.thr)});
          }
        }
        for (const TreePred& p : T.nodes[o.node]) got.insert({p.z, p.op, p.thr});
        got.insert({T.split_z[o.split], o.op, T.thr[o.split][o.j]});
        std::vector<int> mono_got;
        if (T.mom_z[o.mom].first >= 0) mono_got.push_back(T.mom_z[o.mom].first);
        if (T.mom_z[o.mom].second >= 0) mono_got.push_back(T.mom_z[o.mom].second);
        std::sort(mono_want.begin(), mono_want.end());
        std::sort(mono_got.begin(), mono_got.end());
        faithful = want == got && mono_want == mono_got;
        if (!faithful) std::printf("aggregate %zu of trial %d decomposed wrongly\n", i, trial);
      }
      faithful = faithful && all_points_find_their_node(T, 8, 2000);
    }
    expect(faithful, "random batches decompose into their own factors, every point finds its nodes");
  }
  {  // random overlapping conjunctions: several groups, every point finds its node
    std::map<std::string, int> zidx;
    TreePlan tp;
    std::string msg;
    const lmf_status s = tree_plan(random_nodes(300, 99, &zidx), zidx, &tp, &msg);
    expect(s == LMF_OK && all_points_find_their_node(*tp.impl, 7, 20000), "random conjunctions find their nodes");
  }
  return bad ? 1 : 0;
}
