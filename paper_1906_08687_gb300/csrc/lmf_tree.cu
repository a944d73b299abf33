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
//                to the histogram in global memory with 64-bit integer
//                reductions (exact, order-free).  When every active row of a
//                warp falls into one cell -- the rule for a split on a
//                dimension attribute over a root sorted on its join keys --
//                the warp sums its moments first (three 32-bit warp
//                reductions per 64-bit value) and one lane issues the
//                reduction.  Nothing per row leaves the SM.
//   k_tree_out   every aggregate as a prefix / suffix sum over the buckets.
#include "lmf_tree.h"
#include "lmf_rowpass.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>
#include <tuple>

namespace lmf {

constexpr int kTreeMaxMom = 8;
constexpr int kTreeResNodes = 256;  // nodes whose resident-key sums fit the shared table
constexpr uint16_t kNoNode = 0xFFFF;

struct TreePred {
  int16_t z;
  int16_t op;     // 0: x <= thr, 1: x > thr
  float thr;
};

struct TreeOut {
  int32_t node, split, j, op, mom, is_count;
  int64_t dst;
  double inv_scale;
};

struct TreeDev {
  int32_t n_nodes, n_groups, n_split, max_bins, n_mom;
  int32_t mom_stride;          // words per histogram cell: 4 (one 32-byte sector) when n_mom <= 4
  const int32_t* pred_off;     // [n_nodes + 1]
  const TreePred* preds;
  const int32_t* group_off;    // [n_groups + 1] into group_nodes
  const int32_t* group_nodes;
  const int16_t* split_z;      // [n_split]
  const int32_t* thr_off;      // [n_split + 1]
  const float* thr;
  int16_t mom_a[kTreeMaxMom], mom_b[kTreeMaxMom];  // z indices, -1: absent
  double mom_scale[kTreeMaxMom];                   // 0: the count moment (w itself)
  // decision tree over the nodes' predicates, per group: internal entries
  // send a row left when z[dz] <= dthr; a leaf lists candidate nodes
  // [dleft, dleft + dright) of dcand, each checked on all of its predicates
  const int32_t* droot;        // [n_groups]
  const struct TreeDt* dt;
  const int32_t* dcand;
  // splits on an attribute of the resident key's dimension (the root's first
  // sort key, Sec. 3.5): bit f of res_mask; their cells are summed per
  // (node, key) in shared memory and added once per key (res_q: the probe group, -1: none)
  int32_t res_q;
  unsigned long long res_mask;
  long long* H;                // [n_nodes][n_split][max_bins][mom_stride]
  int64_t N;
  uint32_t* status;
};

struct TreeDt {
  int16_t z;
  int16_t leaf;                // 1: left/right are the candidate range [left, left + right)
  float thr;
  int32_t left, right;
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
// splits on one predicate (z, thr) of the nodes; a node that requires z <= thr
// goes only left, one that requires z > thr only right, the others both ways.
// The predicate that leaves the smaller side largest is taken; a set that no
// predicate splits is a leaf (its nodes are checked in full).
int build_dt(const std::vector<std::vector<TreePred>>& nodes, const std::vector<int>& set, int depth,
             std::vector<TreeDt>* dt, std::vector<int32_t>* cand) {
  const int at = (int)dt->size();
  dt->push_back(TreeDt{});
  auto leaf = [&]() {
    (*dt)[at] = TreeDt{0, 1, 0.f, (int32_t)cand->size(), (int32_t)set.size()};
    cand->insert(cand->end(), set.begin(), set.end());
    return at;
  };
  if (set.size() <= 1 || depth >= 24) return leaf();
  std::map<std::pair<int, float>, std::pair<int, int>> cnt;  // (z, thr) -> (nodes only left, only right)
  for (int n : set)
    for (const TreePred& p : nodes[n]) {
      auto& c = cnt[{p.z, p.thr}];
      (p.op == 0 ? c.first : c.second)++;
    }
  int best_min = 0;
  std::pair<int, float> best{-1, 0.f};
  for (auto& kv : cnt) {
    const int n = (int)set.size();
    const int l = n - kv.second.second, r = n - kv.second.first;  // sizes of the two sides
    if (l >= n || r >= n) continue;
    const int mn = std::min(l, r);
    if (mn > best_min) {
      best_min = mn;
      best = kv.first;
    }
  }
  if (best.first < 0) return leaf();
  std::vector<int> L, R;
  for (int n : set) {
    bool le = false, gt = false;
    for (const TreePred& p : nodes[n])
      if (p.z == best.first && p.thr == best.second) (p.op == 0 ? le : gt) = true;
    if (!gt) L.push_back(n);
    if (!le) R.push_back(n);
  }
  const int l = build_dt(nodes, L, depth + 1, dt, cand);
  const int r = build_dt(nodes, R, depth + 1, dt, cand);
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
  for (auto& g : T.groups) T.droot.push_back(build_dt(T.nodes, g, 0, &T.dt, &T.dcand));
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

// exact sum over the lanes of `mask` of a 64-bit integer (two's complement,
// mod 2^64): three 32-bit warp reductions of its 16 + 16 + 32-bit pieces,
// none of which can overflow over 32 lanes; every lane of mask gets the sum
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned mask, unsigned long long v) {
  const unsigned s0 = __reduce_add_sync(mask, static_cast<unsigned>(v & 0xffffu));
  const unsigned s1 = __reduce_add_sync(mask, static_cast<unsigned>((v >> 16) & 0xffffu));
  const unsigned s2 = __reduce_add_sync(mask, static_cast<unsigned>(v >> 32));
  return (static_cast<unsigned long long>(s2) << 32) + (static_cast<unsigned long long>(s1) << 16) + s0;
}

__device__ __forceinline__ void red_add_u64(long long* dst, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(dst), static_cast<unsigned long long>(v));
}

// the row's node in group g: descend the decision tree, then check the
// candidates of the leaf on all of their predicates; kNoNode when none holds
__device__ __forceinline__ int tree_node_of(const TreeDev& d, int g, const float* zrow) {
  int i = d.droot[g];
  TreeDt e = d.dt[i];
  while (!e.leaf) {
    i = zrow[e.z] <= e.thr ? e.left : e.right;
    e = d.dt[i];
  }
  for (int c = e.left; c < e.left + e.right; ++c) {
    const int n = d.dcand[c];
    bool ok = true;
    for (int k = d.pred_off[n]; k < d.pred_off[n + 1] && ok; ++k) {
      const TreePred pr = d.preds[k];
      const float x = zrow[pr.z];
      ok = pr.op == 0 ? (x <= pr.thr) : (x > pr.thr);
    }
    if (ok) return n;
  }
  return kNoNode;
}

constexpr int kTreeThreads = 256;
constexpr int kTreeThrSmem = 48 * 1024;   // thresholds staged in shared memory up to this size

template <int MP>
__global__ void __launch_bounds__(kTreeThreads, 2) k_tree_fused(const __grid_constant__ RootParams p,
                                                                const __grid_constant__ TreeDev d) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int nthr = d.thr_off[d.n_split];
  const bool thr_smem = static_cast<size_t>(nthr) * 4 <= static_cast<size_t>(kTreeThrSmem);
  float* thr_s = reinterpret_cast<float*>(sm);                  // all thresholds, split after split
  float* Z = reinterpret_cast<float*>(sm + (thr_smem ? ((nthr + 3) & ~3) : 0));
  int32_t* C = reinterpret_cast<int32_t*>(Z + kTreeThreads * (MP + 1));
  const int ncat = p.n_rowcat > 0 ? p.n_rowcat : 1;
  // the row's moments, one 32-byte record, the source of its bulk reductions
  __shared__ __align__(16) unsigned long long stage[kTreeThreads][4];
  const bool bulk = d.mom_stride == 4;
  if (thr_smem)
    for (int j = threadIdx.x; j < nthr; j += blockDim.x) thr_s[j] = d.thr[j];
  const float* thr = thr_smem ? thr_s : d.thr;
  float* zrow = Z + threadIdx.x * (MP + 1);  // odd stride: no bank conflicts
  int32_t* crow = C + threadIdx.x * ncat;
  const int lane = threadIdx.x & 31;
  // the resident key's sums per node, added to the histogram once per key
  __shared__ unsigned long long racc[kTreeResNodes][4];
  const bool resident = d.res_q >= 0;
  const GroupDesc& RG = p.grp[resident ? d.res_q : 0];
  long long res_key = -1;
  for (int i = threadIdx.x; i < kTreeResNodes * 4; i += blockDim.x) (&racc[0][0])[i] = 0ull;
  // adds the resident key's sums to their cells (one per node and resident
  // split) and clears them; every thread of the CTA calls this
  auto res_flush = [&]() {
    __syncthreads();
    int nres = 0;
    int fres[64];
    for (int f = 0; f < d.n_split && f < 64; ++f)
      if ((d.res_mask >> f) & 1ull) fres[nres++] = f;
    if (res_key >= 0)
      for (int e = threadIdx.x; e < d.n_nodes * nres; e += blockDim.x) {
        const int n = e / nres, f = fres[e % nres];
        if (racc[n][0] == 0ull && racc[n][1] == 0ull && racc[n][2] == 0ull && racc[n][3] == 0ull) continue;
        const int zf = d.split_z[f];
        const float x = __uint_as_float(RG.rec[res_key * RG.stride + RG.n_cnt + (zf - p.grp_zoff[d.res_q])]);
        const int t0 = d.thr_off[f];
        int l = 0, h = d.thr_off[f + 1] - t0;
        while (l < h) {
          const int mid = (l + h) >> 1;
          if (thr[t0 + mid] < x) l = mid + 1;
          else h = mid;
        }
        const int64_t cell = ((static_cast<int64_t>(n) * d.n_split + f) * d.max_bins + l) * d.mom_stride;
        for (int m = 0; m < d.n_mom; ++m)
          if (racc[n][m] != 0ull) red_add_u64(d.H + cell + m, static_cast<long long>(racc[n][m]));
      }
    __syncthreads();
    for (int i = threadIdx.x; i < kTreeResNodes * 4; i += blockDim.x) (&racc[0][0])[i] = 0ull;
    __syncthreads();
  };
  __syncthreads();
  // each CTA a contiguous range of rows (the resident key changes rarely
  // inside it); every lane of a warp runs every iteration (warp reductions
  // below), rows past the range are inactive
  const int64_t r_begin = static_cast<int64_t>(blockIdx.x) * d.N / gridDim.x;
  const int64_t r_end = (static_cast<int64_t>(blockIdx.x) + 1) * d.N / gridDim.x;
  for (int64_t base = r_begin; base < r_end; base += blockDim.x) {
    if (resident) {  // CTA-uniform: the key of the chunk's first row
      const int32_t k0 = RG.fk[base];
      const long long nk = (k0 >= 0 && k0 < RG.K) ? k0 : -1;
      if (nk != res_key) {
        res_flush();
        res_key = nk;
      }
    }
    const int64_t row = base + threadIdx.x;
    long long w = 0;
    if (row < r_end) w = root_row_z<MP>(p, row, zrow, crow);
    // the row's cells of resident splits go to the shared sums
    const bool row_res = resident && w != 0 && res_key >= 0 && static_cast<long long>(RG.fk[row]) == res_key;
    long long mv[kTreeMaxMom];
    bool have = false;
    for (int g = 0; g < d.n_groups; ++g) {
      const int n = w != 0 ? tree_node_of(d, g, zrow) : static_cast<int>(kNoNode);
      const bool on_g = n != static_cast<int>(kNoNode);
      const unsigned on_mask = __ballot_sync(0xffffffffu, on_g);
      if (on_mask == 0u) continue;  // warp-uniform
      if (on_g && !have) {  // the row's fixed-point moments, once
#pragma unroll
        for (int m = 0; m < kTreeMaxMom; ++m) {
          if (m >= d.n_mom) break;
          long long v = w;
          if (d.mom_scale[m] > 0.0) {
            double x = static_cast<double>(w);
            if (d.mom_a[m] >= 0) x *= static_cast<double>(zrow[d.mom_a[m]]);
            if (d.mom_b[m] >= 0) x *= static_cast<double>(zrow[d.mom_b[m]]);
            v = llrint(x * d.mom_scale[m]);
          }
          mv[m] = v;
        }
        have = true;
        if (bulk) {  // the previous row's reductions have read the record: refill it
          asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
#pragma unroll
          for (int m = 0; m < 4; ++m) stage[threadIdx.x][m] = m < d.n_mom ? static_cast<unsigned long long>(mv[m]) : 0ull;
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
      }
      if (on_g && row_res)
        for (int m = 0; m < d.n_mom && m < 4; ++m)
          if (mv[m] != 0) atomicAdd(&racc[n][m], static_cast<unsigned long long>(mv[m]));
      for (int f = 0; f < d.n_split; ++f) {
        // a resident split of a row with the resident key is in the shared sums
        const bool on = on_g && !(row_res && f < 64 && ((d.res_mask >> f) & 1ull));
        int64_t cell = 0;
        if (on) {
          const float x = zrow[d.split_z[f]];
          const int t0 = d.thr_off[f];
          int l = 0, h = d.thr_off[f + 1] - t0;
          while (l < h) {  // number of thresholds < x
            const int mid = (l + h) >> 1;
            if (thr[t0 + mid] < x) l = mid + 1;
            else h = mid;
          }
          cell = ((static_cast<int64_t>(n) * d.n_split + f) * d.max_bins + l) * d.mom_stride;
        }
        const unsigned f_mask = __ballot_sync(0xffffffffu, on);
        if (f_mask == 0u) continue;  // warp-uniform
        const int f_lead = __ffs(f_mask) - 1;
        const int64_t c0 = __shfl_sync(0xffffffffu, cell, f_lead);
        if (__all_sync(0xffffffffu, !on || cell == c0)) {  // one cell for the whole warp
#pragma unroll
          for (int m = 0; m < kTreeMaxMom; ++m) {
            if (m >= d.n_mom) break;
            const unsigned long long sum = warp_sum_u64(0xffffffffu, on ? static_cast<unsigned long long>(mv[m]) : 0ull);
            if (lane == f_lead && sum != 0ull) red_add_u64(d.H + c0 + m, static_cast<long long>(sum));
          }
        } else if (on && bulk) {  // the row's record added to its 32-byte cell in one reduction
          asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], 32;" ::"l"(d.H + cell),
                       "r"(static_cast<uint32_t>(__cvta_generic_to_shared(&stage[threadIdx.x][0])))
                       : "memory");
        } else if (on) {
#pragma unroll
          for (int m = 0; m < kTreeMaxMom; ++m) {
            if (m >= d.n_mom) break;
            if (mv[m] != 0) red_add_u64(d.H + cell + m, mv[m]);
          }
        }
      }
      if (bulk) asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
  if (resident) res_flush();
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
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
