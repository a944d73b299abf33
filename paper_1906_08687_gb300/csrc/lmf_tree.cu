// lmf_tree.cu -- threshold-filtered aggregates (regression-tree node batches).
//
// An aggregate SUM(m * 1[p_1] * ... * 1[p_k]) (Sec. 1.1: products of Kronecker
// deltas; Sec. 2, Eq. regression-tree) is read as
//     node (the conjunction of all but one predicate) x split (the remaining
//     predicate x <= t or x > t on attribute f) x moment m (degree <= 2),
// choosing as split the predicate whose removal leaves the conjunction shared
// by the most aggregates of the batch (for a tree level: the candidate
// condition, while the ancestors' conditions form the node).  Any choice gives
// the same product, so the choice only affects speed.  With the sorted thresholds T_f of attribute f
// and the bucket b(x) = #{t in T_f : t < x},
//     x <= T_f[j]  <=>  b(x) <= j,
// so every (node, f, j, m) aggregate is a prefix (or, for >, suffix) sum of
// one histogram H[node][f][b][m].  Thresholds are rounded down to FP32, which
// keeps x <= t exact for FP32 data.
//
// Kernels:
//   k_tree_fused persistent, one pass over the root: for every row it builds z
//                from the views, finds the row's node in every group of
//                mutually exclusive nodes by descending a decision tree over
//                the nodes' predicates, computes the row's fixed-point moments
//                and its bucket for every split attribute (binary search over
//                the thresholds, held in shared memory), and adds the moments
//                to the histogram in global memory as exact integers
//                (order-free): the row's record, staged once in shared memory,
//                to each split's 32-byte cell by one bulk reduction
//                (cp.reduce.async.bulk .add.u64), or by 64-bit reductions when
//                a cell holds more than four moments.  When every active row
//                of a warp falls into one cell -- the rule for a split on a
//                dimension attribute over a root sorted on its join keys --
//                the warp sums its moments first (three 32-bit warp
//                reductions per 64-bit value) and one lane issues the
//                reduction; splits on the resident key's dimension are summed
//                per (node, key) in shared memory and added once per key.
//                Nothing per row leaves the SM.  Its body is
//                tree_body (lmf_tree_dev.cuh); lmf_tree_jit, compiled for the
//                plan at plan time (lmf_jit_tree.cu), runs the same body with
//                the row pass and the node search generated for the plan, and
//                replaces k_tree_fused when it was compiled.
//   k_tree_out   every aggregate as a prefix / suffix sum over the buckets.
#include "lmf_tree.h"
#include "lmf_tree_dev.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>
#include <tuple>

namespace lmf {

struct TreeOut {
  int32_t node, split, j, op, mom, is_count;
  int64_t dst;
  double inv_scale;
};

struct TreeShape {
  int cps;                     // CTAs per SM of the persistent pass
};

struct TreePlanImpl {
  // host plan
  std::vector<std::vector<TreePred>> nodes;
  std::vector<std::vector<int>> groups;
  std::vector<int16_t> split_z;
  std::vector<std::string> split_name;
  std::vector<std::vector<float>> thr;
  std::vector<std::pair<std::string, std::string>> moms;  // attribute names ("" absent)
  std::vector<std::pair<int, int>> mom_z;
  struct OutH {
    int node, split, j, op, mom;
  };
  std::vector<OutH> outs;
  std::vector<int32_t> droot;    // decision tree per group (host copy)
  std::vector<TreeDt> dt;
  std::vector<int32_t> dcand;
  int max_bins = 1;
  int mp = 16;
  // device
  size_t H_off = 0;
  size_t tab_off = 0, tab_bytes = 0, outs_off = 0;
  TreeDev dev{};
  const TreeOut* d_outs = nullptr;
  int n_outs = 0;
  long long* res_i64 = nullptr;
  double* res_f64 = nullptr;
  int num_sms = 0;
  TreeShape shape{2};
  bool tuned = false;
  cudaKernel_t jit = nullptr;    // the pass compiled for the plan (null: k_tree_fused)
};

TreePlan::~TreePlan() { delete impl; }

namespace {

float round_down_f32(double t) {
  float f = static_cast<float>(t);
  if (static_cast<double>(f) > t) f = std::nextafter(f, -INFINITY);
  return f;
}

bool disjoint(const std::vector<TreePred>& a, const std::vector<TreePred>& b) {
  for (const auto& p : a)
    for (const auto& q : b) {
      if (p.z != q.z || p.op == q.op) continue;
      const TreePred& le = p.op == 0 ? p : q;
      const TreePred& gt = p.op == 0 ? q : p;
      if (gt.thr >= le.thr) return true;  // x <= t1 and x > t2 >= t1 cannot both hold
    }
  return false;
}

// Decision tree over a set of mutually exclusive nodes: an internal entry
// splits on one threshold (z, thr) taken from the nodes' predicates.  On z a
// node allows the interval (lo, hi] that its predicates leave (lo the largest
// threshold of a "z > t", hi the smallest of a "z <= t"); it goes left when
// the interval reaches below thr (lo < thr), right when it reaches above
// (hi > thr), both ways when it straddles thr, and nowhere when it is empty.
// The split whose larger side is smallest is taken (ties: the fewer nodes on
// both sides together), so that the nodes of a tree level, which split into
// halves on the predicate of their common ancestor, give a tree of the level's
// depth, and the cells of a grid of bins on a few attributes a tree of about
// log2 of their number.  A set that no split divides, or a tree that reached
// kMaxDt entries, kMaxCand candidates or kMaxWork predicate visits, ends in a
// leaf (its nodes are checked in full).  Once a cap is reached only the
// pending right subtrees of the current path (at most one per level) still
// add leaves, so the tables stay within the caps plus 25 sets.
constexpr size_t kMaxDt = size_t(1) << 16;
constexpr size_t kMaxCand = size_t(1) << 20;
constexpr size_t kMaxWork = size_t(1) << 26;

// the interval (lo, hi] that node `preds` allows on z; (+inf, -inf] when empty
void node_interval(const std::vector<TreePred>& preds, int z, float* lo, float* hi) {
  float a = -INFINITY, b = INFINITY;
  for (const TreePred& p : preds)
    if (p.z == z) {
      if (p.op == 0) b = std::min(b, p.thr);
      else a = std::max(a, p.thr);
    }
  if (!(a < b)) {
    a = INFINITY;
    b = -INFINITY;
  }
  *lo = a;
  *hi = b;
}

int build_dt(const std::vector<std::vector<TreePred>>& nodes, const std::vector<int>& set, int depth,
             std::vector<TreeDt>* dt, std::vector<int32_t>* cand, size_t* work) {
  const int at = (int)dt->size();
  dt->push_back(TreeDt{});
  auto leaf = [&]() {
    (*dt)[at] = TreeDt{0, 1, 0.f, (int32_t)cand->size(), (int32_t)set.size()};
    cand->insert(cand->end(), set.begin(), set.end());
    return at;
  };
  if (set.size() <= 1 || depth >= 24 || dt->size() >= kMaxDt || cand->size() >= kMaxCand || *work >= kMaxWork)
    return leaf();
  const int n = (int)set.size();
  // candidate thresholds per attribute
  std::map<int, std::vector<float>> thrs;
  for (int i : set)
    for (const TreePred& p : nodes[i])
      if (p.thr == p.thr) thrs[p.z].push_back(p.thr);  // (a NaN threshold orders nothing)
  int best_max = n, best_sum = 2 * n;
  std::pair<int, float> best{-1, 0.f};
  std::vector<float> lo(n), hi(n);
  for (auto& kv : thrs) {
    const int z = kv.first;
    for (int k = 0; k < n; ++k) node_interval(nodes[set[k]], z, &lo[k], &hi[k]);
    *work += static_cast<size_t>(n) * (nodes[set[0]].size() + 1);
    std::sort(lo.begin(), lo.end());
    std::sort(hi.begin(), hi.end());
    std::vector<float>& ts = kv.second;
    std::sort(ts.begin(), ts.end());
    ts.erase(std::unique(ts.begin(), ts.end()), ts.end());
    for (float t : ts) {
      const int l = (int)(std::lower_bound(lo.begin(), lo.end(), t) - lo.begin());  // lo < t
      const int r = (int)(hi.end() - std::upper_bound(hi.begin(), hi.end(), t));   // hi > t
      if (l >= n || r >= n) continue;  // one side keeps every node: no progress
      const int mx = std::max(l, r), sum = l + r;
      if (mx < best_max || (mx == best_max && sum < best_sum)) {
        best_max = mx;
        best_sum = sum;
        best = {z, t};
      }
    }
  }
  if (best.first < 0) return leaf();
  std::vector<int> L, R;
  for (int i : set) {
    float a, b;
    node_interval(nodes[i], best.first, &a, &b);
    if (a < best.second) L.push_back(i);
    if (b > best.second) R.push_back(i);
  }
  const int l = build_dt(nodes, L, depth + 1, dt, cand, work);
  const int r = build_dt(nodes, R, depth + 1, dt, cand, work);
  (*dt)[at] = TreeDt{(int16_t)best.first, 0, best.second, l, r};
  return at;
}

}  // namespace

lmf_status tree_plan(const std::vector<TreeAggIn>& in, const std::map<std::string, int>& zidx, TreePlan* tp,
                     std::string* msg) {
  tp->impl = new TreePlanImpl();
  TreePlanImpl& T = *tp->impl;
  // Split choice.  Removing predicate k of aggregate a leaves the candidate node
  // N(a, k).  Every aggregate takes the split whose node is a candidate of the
  // most aggregates (its "support"), so that aggregates sharing a conjunction
  // share a node even when a candidate threshold equals one of the
  // conjunction's own thresholds; ties go to the least frequent predicate.
  using Key = std::tuple<std::string, int, double>;
  std::map<Key, int> pid;
  std::vector<int> freq;
  std::vector<std::vector<int>> apred(in.size());
  for (size_t i = 0; i < in.size(); ++i)
    for (auto& f : in[i].factors)
      if (f.kind != LMF_POW) {
        auto it = pid.emplace(Key(f.attr, f.kind, f.thr), (int)pid.size()).first;
        if ((int)freq.size() <= it->second) freq.push_back(0);
        freq[it->second]++;
        apred[i].push_back(it->second);
      }
  auto cand_node = [&](size_t i, size_t k) {
    std::vector<int> n;
    for (size_t j = 0; j < apred[i].size(); ++j)
      if (j != k) n.push_back(apred[i][j]);
    std::sort(n.begin(), n.end());
    n.erase(std::unique(n.begin(), n.end()), n.end());
    return n;
  };
  std::map<std::vector<int>, int> support;
  for (size_t i = 0; i < in.size(); ++i) {
    std::set<std::vector<int>> seen;
    for (size_t k = 0; k < apred[i].size(); ++k) seen.insert(cand_node(i, k));
    for (auto& n : seen) support[n]++;
  }
  std::vector<int> split_pos(in.size(), -1);  // position among the aggregate's predicates
  for (size_t i = 0; i < in.size(); ++i) {
    int best = -1, bs = -1, bf = 1 << 30;
    for (size_t k = 0; k < apred[i].size(); ++k) {
      const int s = support[cand_node(i, k)];
      const int f = freq[apred[i][k]];
      if (s > bs || (s == bs && f <= bf)) {
        bs = s;
        bf = f;
        best = (int)k;
      }
    }
    split_pos[i] = best;
  }
  std::map<std::vector<std::tuple<int, int, float>>, int> node_id;
  std::map<std::string, int> split_id;
  std::vector<std::set<float>> split_thr;
  std::map<std::pair<std::string, std::string>, int> mom_id;
  struct Pending {
    int node, split, op, mom;
    float t;
  };
  std::vector<Pending> pend;
  for (size_t i = 0; i < in.size(); ++i) {
    const auto& a = in[i];
    int best = -1;
    std::vector<std::string> mono;
    for (size_t k = 0, np = 0; k < a.factors.size(); ++k) {
      const auto& f = a.factors[k];
      if (f.kind == LMF_POW) {
        for (int e = 0; e < f.power; ++e) mono.push_back(f.attr);
        continue;
      }
      if ((int)np++ == split_pos[i]) best = (int)k;
    }
    if (best < 0 || mono.size() > 2) {
      *msg = "filtered aggregate without a threshold factor or with a monomial of degree > 2";
      return LMF_ERR_UNSUPPORTED;
    }
    std::vector<std::tuple<int, int, float>> node;
    for (size_t k = 0; k < a.factors.size(); ++k) {
      const auto& f = a.factors[k];
      if (f.kind == LMF_POW || (int)k == best) continue;
      node.emplace_back(zidx.at(f.attr), f.kind == LMF_LE ? 0 : 1, round_down_f32(f.thr));
    }
    std::sort(node.begin(), node.end());
    node.erase(std::unique(node.begin(), node.end()), node.end());
    auto nit = node_id.find(node);
    int nid;
    if (nit == node_id.end()) {
      nid = (int)T.nodes.size();
      node_id[node] = nid;
      std::vector<TreePred> preds;
      for (auto& p : node) preds.push_back({(int16_t)std::get<0>(p), (int16_t)std::get<1>(p), std::get<2>(p)});
      T.nodes.push_back(preds);
    } else {
      nid = nit->second;
    }
    const auto& sf = a.factors[best];
    auto sit = split_id.find(sf.attr);
    int sid;
    if (sit == split_id.end()) {
      sid = (int)T.split_z.size();
      split_id[sf.attr] = sid;
      T.split_z.push_back((int16_t)zidx.at(sf.attr));
      T.split_name.push_back(sf.attr);
      split_thr.emplace_back();
    } else {
      sid = sit->second;
    }
    const float t = round_down_f32(sf.thr);
    split_thr[sid].insert(t);
    std::pair<std::string, std::string> mk{mono.size() > 0 ? mono[0] : "", mono.size() > 1 ? mono[1] : ""};
    auto mit = mom_id.find(mk);
    int mid;
    if (mit == mom_id.end()) {
      mid = (int)T.moms.size();
      if (mid >= kTreeMaxMom) {
        *msg = "more than 8 distinct monomials among filtered aggregates";
        return LMF_ERR_UNSUPPORTED;
      }
      mom_id[mk] = mid;
      T.moms.push_back(mk);
      T.mom_z.push_back({mk.first.empty() ? -1 : zidx.at(mk.first), mk.second.empty() ? -1 : zidx.at(mk.second)});
    } else {
      mid = mit->second;
    }
    pend.push_back({nid, sid, sf.kind == LMF_LE ? 0 : 1, mid, t});
  }
  if (T.nodes.size() >= kNoNode) {
    *msg = "too many distinct nodes";
    return LMF_ERR_UNSUPPORTED;
  }
  for (auto& s : split_thr) {
    if (s.size() > 254) {
      *msg = "more than 254 thresholds on one attribute";
      return LMF_ERR_UNSUPPORTED;
    }
    T.thr.emplace_back(s.begin(), s.end());
    T.max_bins = std::max<int>(T.max_bins, (int)s.size() + 1);
  }
  for (auto& p : pend) {
    const auto& v = T.thr[p.split];
    const int j = (int)(std::lower_bound(v.begin(), v.end(), p.t) - v.begin());
    T.outs.push_back({p.node, p.split, j, p.op, p.mom});
  }
  // groups of mutually exclusive nodes (greedy)
  for (int n = 0; n < (int)T.nodes.size(); ++n) {
    bool placed = false;
    for (auto& g : T.groups) {
      bool ok = true;
      for (int o : g)
        if (!disjoint(T.nodes[n], T.nodes[o])) {
          ok = false;
          break;
        }
      if (ok) {
        g.push_back(n);
        placed = true;
        break;
      }
    }
    if (!placed) T.groups.push_back({n});
  }
  size_t dt_work = 0;
  for (auto& g : T.groups) T.droot.push_back(build_dt(T.nodes, g, 0, &T.dt, &T.dcand, &dt_work));
  int mz = 0;
  for (auto& kv : zidx) mz = std::max(mz, kv.second + 1);
  T.mp = 16;
  while (T.mp < mz) T.mp += 16;
  T.dev.n_nodes = (int)T.nodes.size();
  T.dev.n_groups = (int)T.groups.size();
  T.dev.n_split = (int)T.split_z.size();
  T.dev.max_bins = T.max_bins;
  T.dev.n_mom = (int)T.moms.size();
  T.dev.mom_stride = T.dev.n_mom <= 4 ? 4 : T.dev.n_mom;
  T.shape.cps = 2;
  return LMF_OK;
}

void tree_alloc_zeroed(TreePlan* tp, int64_t /*N*/, const std::function<size_t(size_t)>& take) {
  TreePlanImpl& T = *tp->impl;
  T.H_off = take(static_cast<size_t>(T.dev.n_nodes) * T.dev.n_split * T.max_bins * T.dev.mom_stride * 8);
}

void tree_alloc(TreePlan* tp, int64_t /*N*/, const std::function<size_t(size_t)>& take) {
  TreePlanImpl& T = *tp->impl;
  size_t npred = 0, nthr = 0;
  for (auto& v : T.nodes) npred += v.size();
  for (auto& v : T.thr) nthr += v.size();
  T.tab_bytes = (T.nodes.size() + 1) * 4 + (npred + 1) * sizeof(TreePred) + (T.groups.size() + 1) * 4 +
                (T.nodes.size() + 1) * 4 + (T.split_z.size() + 1) * 2 + (T.split_z.size() + 1) * 4 +
                (nthr + 1) * 4 + (T.droot.size() + 1) * 4 + (T.dt.size() + 1) * sizeof(TreeDt) +
                (T.dcand.size() + 1) * 4 + 128;
  T.tab_off = take(T.tab_bytes);
  T.outs_off = take(sizeof(TreeOut) * (T.outs.size() + 1));
}

lmf_status tree_finish(TreePlan* tp, char* base, long long* res_i64, double* res_f64,
                       const std::vector<int64_t>& agg_off, const std::vector<int>& filt_idx,
                       const std::vector<int32_t>& agg_dtype, uint32_t* status, int64_t N, int num_sms,
                       const std::map<std::string, double>& bound, double W, const RootParams& rp, int res_q) {
  TreePlanImpl& T = *tp->impl;
  T.num_sms = num_sms;
  TreeDev& D = T.dev;
  D.res_q = -1;
  D.res_mask = 0ull;
  if (res_q >= 0 && res_q < rp.n_grp && D.n_nodes <= kTreeResNodes && D.n_mom <= 4 && D.n_split <= 64) {
    const int z0 = rp.grp_zoff[res_q], z1 = z0 + rp.grp[res_q].n_mu;
    for (int f = 0; f < D.n_split; ++f)
      if (T.split_z[f] >= z0 && T.split_z[f] < z1) D.res_mask |= 1ull << f;
    if (D.res_mask) D.res_q = res_q;
  }
  D.N = N;
  D.status = status;
  D.H = reinterpret_cast<long long*>(base + T.H_off);
  // moments: fixed-point scale from the value bounds, 0 for the count
  std::vector<double> scale(T.moms.size());
  for (size_t m = 0; m < T.moms.size(); ++m) {
    D.mom_a[m] = (int16_t)T.mom_z[m].first;
    D.mom_b[m] = (int16_t)T.mom_z[m].second;
    if (T.moms[m].first.empty()) {
      scale[m] = 0.0;
    } else {
      double b = bound.at(T.moms[m].first);
      if (!T.moms[m].second.empty()) b *= bound.at(T.moms[m].second);
      const double tot = W * b;
      int e = (tot > 0 && std::isfinite(tot)) ? 62 - (int)std::ceil(std::log2(tot)) : 40;
      e = std::max(-1000, std::min(1000, e));
      scale[m] = std::ldexp(1.0, e);
    }
    D.mom_scale[m] = scale[m];
  }
  // plan tables
  std::vector<char> tab(T.tab_bytes, 0);
  size_t off = 0;
  auto put = [&](const void* src, size_t bytes, size_t align) {
    off = (off + align - 1) / align * align;
    size_t at = off;
    if (bytes) std::memcpy(tab.data() + off, src, bytes);
    off += bytes;
    return at;
  };
  std::vector<int32_t> pred_off{0};
  std::vector<TreePred> preds;
  for (auto& v : T.nodes) {
    preds.insert(preds.end(), v.begin(), v.end());
    pred_off.push_back((int32_t)preds.size());
  }
  std::vector<int32_t> group_off{0}, group_nodes;
  for (auto& g : T.groups) {
    group_nodes.insert(group_nodes.end(), g.begin(), g.end());
    group_off.push_back((int32_t)group_nodes.size());
  }
  std::vector<int32_t> thr_off{0};
  std::vector<float> thr;
  for (auto& v : T.thr) {
    thr.insert(thr.end(), v.begin(), v.end());
    thr_off.push_back((int32_t)thr.size());
  }
  const size_t o_pred_off = put(pred_off.data(), pred_off.size() * 4, 8);
  const size_t o_preds = put(preds.data(), preds.size() * sizeof(TreePred), 8);
  const size_t o_group_off = put(group_off.data(), group_off.size() * 4, 8);
  const size_t o_group_nodes = put(group_nodes.data(), group_nodes.size() * 4, 8);
  const size_t o_split_z = put(T.split_z.data(), T.split_z.size() * 2, 8);
  const size_t o_thr_off = put(thr_off.data(), thr_off.size() * 4, 8);
  const size_t o_thr = put(thr.data(), thr.size() * 4, 8);
  const size_t o_droot = put(T.droot.data(), T.droot.size() * 4, 8);
  const size_t o_dt = put(T.dt.data(), T.dt.size() * sizeof(TreeDt), 8);
  const size_t o_dcand = put(T.dcand.data(), T.dcand.size() * 4, 8);
  if (off > T.tab_bytes) return LMF_ERR_ARG;
  char* dtab = base + T.tab_off;
  D.pred_off = reinterpret_cast<const int32_t*>(dtab + o_pred_off);
  D.preds = reinterpret_cast<const TreePred*>(dtab + o_preds);
  D.group_off = reinterpret_cast<const int32_t*>(dtab + o_group_off);
  D.group_nodes = reinterpret_cast<const int32_t*>(dtab + o_group_nodes);
  D.split_z = reinterpret_cast<const int16_t*>(dtab + o_split_z);
  D.thr_off = reinterpret_cast<const int32_t*>(dtab + o_thr_off);
  D.thr = reinterpret_cast<const float*>(dtab + o_thr);
  D.droot = reinterpret_cast<const int32_t*>(dtab + o_droot);
  D.dt = reinterpret_cast<const TreeDt*>(dtab + o_dt);
  D.dcand = reinterpret_cast<const int32_t*>(dtab + o_dcand);
  if (cudaMemcpy(dtab, tab.data(), T.tab_bytes, cudaMemcpyHostToDevice) != cudaSuccess) return LMF_ERR_CUDA;
  // outputs
  std::vector<TreeOut> outs;
  for (size_t k = 0; k < T.outs.size(); ++k) {
    const auto& o = T.outs[k];
    const int a = filt_idx[k];
    TreeOut t;
    t.node = o.node;
    t.split = o.split;
    t.j = o.j;
    t.op = o.op;
    t.mom = o.mom;
    t.is_count = agg_dtype[a] == LMF_I64 ? 1 : 0;
    t.dst = agg_off[a];
    t.inv_scale = scale[o.mom] > 0 ? 1.0 / scale[o.mom] : 1.0;
    outs.push_back(t);
  }
  T.n_outs = (int)outs.size();
  if (!outs.empty() &&
      cudaMemcpy(base + T.outs_off, outs.data(), sizeof(TreeOut) * outs.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return LMF_ERR_CUDA;
  T.d_outs = reinterpret_cast<const TreeOut*>(base + T.outs_off);
  T.res_i64 = res_i64;
  T.res_f64 = res_f64;
  return LMF_OK;
}

// ---------------------------------------------------------------------------
// kernels

template <int MP>
__global__ void __launch_bounds__(kTreeThreads, 2) k_tree_fused(const __grid_constant__ RootParams p,
                                                                const __grid_constant__ TreeDev d) {
  tree_body<InterpTreeRow<MP>, MP>(p, d);
}

__global__ void k_tree_out(const __grid_constant__ TreeDev d, const TreeOut* outs, int n, long long* res_i64,
                           double* res_f64) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const TreeOut o = outs[k];
  const int nb = d.thr_off[o.split + 1] - d.thr_off[o.split] + 1;
  const long long* h = d.H + ((int64_t)o.node * d.n_split + o.split) * d.max_bins * d.mom_stride + o.mom;
  long long s = 0;
  if (o.op == 0) {
    for (int b = 0; b <= o.j; ++b) s += h[(int64_t)b * d.mom_stride];
  } else {
    for (int b = o.j + 1; b < nb; ++b) s += h[(int64_t)b * d.mom_stride];
  }
  if (o.is_count) res_i64[o.dst] = s;
  else res_f64[o.dst] = static_cast<double>(s) * o.inv_scale;
}

namespace {

size_t fused_smem(const TreePlanImpl& T, const RootParams& rp) {
  size_t nthr = 0;
  for (auto& v : T.thr) nthr += v.size();
  const size_t thr = nthr * 4 <= static_cast<size_t>(kTreeThrSmem) ? ((nthr + 3) & ~static_cast<size_t>(3)) * 4 : 0;
  const size_t z = static_cast<size_t>(kTreeThreads) * (T.mp + 1) * 4;
  const size_t cat = static_cast<size_t>(kTreeThreads) * (rp.n_rowcat > 0 ? rp.n_rowcat : 1) * 4;
  return thr + z + cat;
}

cudaError_t launch_fused_jit(const TreePlanImpl& T, const RootParams& rp, const TreeShape& sh, cudaStream_t s) {
  const size_t sm = fused_smem(T, rp);
  const void* fn = reinterpret_cast<const void*>(T.jit);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int fit = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, kTreeThreads, sm) != cudaSuccess) {
    cudaGetLastError();  // the query is only advisory: the launch bounds guarantee two
    fit = 2;
  }
  const int cps = std::max(1, std::min(sh.cps, std::max(1, fit)));
  const int64_t need = (T.dev.N + kTreeThreads - 1) / kTreeThreads;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, static_cast<int64_t>(T.num_sms) * cps));
  void* args[] = {const_cast<RootParams*>(&rp), const_cast<TreeDev*>(&T.dev)};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(kTreeThreads), args, sm, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int MP>
cudaError_t launch_fused_mp(const TreePlanImpl& T, const RootParams& rp, const TreeShape& sh, cudaStream_t s) {
  const size_t sm = fused_smem(T, rp);
  cudaError_t e = cudaFuncSetAttribute(k_tree_fused<MP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int fit = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_tree_fused<MP>, kTreeThreads, sm);
  if (e != cudaSuccess) return e;
  const int cps = std::max(1, std::min(sh.cps, fit));
  const int64_t need = (T.dev.N + kTreeThreads - 1) / kTreeThreads;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, static_cast<int64_t>(T.num_sms) * cps));
  k_tree_fused<MP><<<grid, kTreeThreads, sm, s>>>(rp, T.dev);
  return cudaGetLastError();
}

cudaError_t launch_fused(const TreePlanImpl& T, const RootParams& rp, const TreeShape& sh, cudaStream_t s) {
  if (T.jit) return launch_fused_jit(T, rp, sh, s);
  switch (T.mp) {
    case 16: return launch_fused_mp<16>(T, rp, sh, s);
    case 32: return launch_fused_mp<32>(T, rp, sh, s);
    case 48: return launch_fused_mp<48>(T, rp, sh, s);
    default: return launch_fused_mp<64>(T, rp, sh, s);
  }
}

}  // namespace

cudaError_t tree_launch(TreePlan* tp, const RootParams& rp, cudaStream_t s, int* nk) {
  TreePlanImpl& T = *tp->impl;
  cudaError_t e = launch_fused(T, rp, T.shape, s);
  if (e != cudaSuccess) return e;
  if (T.n_outs > 0) {
    k_tree_out<<<(T.n_outs + 255) / 256, 256, 0, s>>>(T.dev, T.d_outs, T.n_outs, T.res_i64, T.res_f64);
  }
  *nk += 2;
  return cudaGetLastError();
}

void tree_jit_spec(const TreePlan* tp, TreeJitSpec* out) {
  const TreePlanImpl& T = *tp->impl;
  out->mp = T.mp;
  out->droot.assign(T.droot.begin(), T.droot.end());
  out->dt.clear();
  for (const TreeDt& e : T.dt) out->dt.push_back({e.z, e.leaf, e.thr, e.left, e.right});
  out->cand.assign(T.dcand.begin(), T.dcand.end());
  out->preds.clear();
  for (const auto& v : T.nodes) {
    std::vector<TreeJitSpec::Pred> ps;
    for (const TreePred& pr : v) ps.push_back({pr.z, pr.op, pr.thr});
    out->preds.push_back(ps);
  }
}

void tree_set_jit(TreePlan* tp, cudaKernel_t k) { tp->impl->jit = k; }

bool tree_needs_tuning(const TreePlan* tp) { return tp && tp->impl && !tp->impl->tuned; }

cudaError_t tree_autotune(TreePlan* tp, const RootParams& rp, cudaStream_t s) {
  TreePlanImpl& T = *tp->impl;
  (void)rp;
  // CTAs per SM of the persistent pass (capped by what fits)
  std::vector<TreeShape> cand{{2}, {3}, {4}, {6}};
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  TreeShape pick = T.shape;
  const size_t hbytes = static_cast<size_t>(T.dev.n_nodes) * T.dev.n_split * T.max_bins * T.dev.mom_stride * 8;
  for (const auto& c : cand) {
    cudaMemsetAsync(T.dev.H, 0, hbytes, s);
    cudaEventRecord(a, s);
    cudaError_t e = launch_fused(T, rp, c, s);
    cudaEventRecord(b, s);
    if (e != cudaSuccess) continue;
    if (cudaEventSynchronize(b) != cudaSuccess) break;
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  T.shape = pick;
  T.tuned = true;
  return cudaGetLastError();
}

void tree_shape(const TreePlan* tp, int* out5) {
  const TreePlanImpl& T = *tp->impl;
  out5[0] = 1;                    // one pass over the root, every node and split
  out5[1] = T.dev.n_split;
  out5[2] = T.dev.n_nodes;
  out5[3] = T.shape.cps;
  out5[4] = 0;
}

}  // namespace lmf

namespace lmf {
void tree_counts(const TreePlan* tp, int32_t* nodes, int32_t* groups) {
  *nodes = tp->impl->dev.n_nodes;
  *groups = tp->impl->dev.n_groups;
}
}  // namespace lmf
