// Host-only check of the tree planner (no GPU needed): the decomposition of a
// batch of threshold-filtered aggregates into nodes, split attributes and the
// decision tree that finds a row's node.  Used by tests/test_tree_plan.py.
// Exit status 0 when every check holds; one line per check on stdout.
#include "lmf_tree.cu"

#include <cstdio>
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

}  // namespace

int main() {
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
    // decision tree with one internal entry per internal tree node
    expect(T.dt.size() == 2 * leaves - 1 && T.dcand.size() == leaves, ("decision tree of the level's size" + d).c_str());
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
    expect(deepest == depth, ("decision tree of the level's depth" + d).c_str());
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
  return bad ? 1 : 0;
}
