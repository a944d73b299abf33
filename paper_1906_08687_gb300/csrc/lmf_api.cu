// lmf_api.cu -- the C ABI (include/lmf.h) and the host planner.
//
// Planning follows the paper's logical layers in a GPU form:
//   join tree (Sec. 3.1)            -> lmf_declare_join validates the tree, indexes child keys
//   aggregate pushdown (Sec. 3.2)   -> every child relation gets one view carrying its
//                                      subtree count, the means of the subtree features the
//                                      batch needs and the categories it groups by
//   view merging (Sec. 3.4)         -> views of children joined on the same parent key share
//                                      one record array (a probe group); one view per edge
//                                      serves every aggregate that needs it
//   view groups / ordering (Sec. 3.4) -> child views are built deepest first
//   multi-output plan (Sec. 3.5)    -> one root scan produces the Gram, the counts, the
//                                      reverse views and the per-row grouped tables at once
#include "lmf.h"
#include "lmf_internal.h"
#include "lmf_jit.h"
#include "lmf_keymap.h"
#include "lmf_tree.h"
#include "lmf_gram_tc.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <set>
#include <string>
#include <vector>

using namespace lmf;

namespace {

struct ColumnH {
  std::string name;
  int dtype, role, dom, on_host;
  const void* data;      // user pointer
  void* dev = nullptr;   // device copy of a host column
  const void* mapped = nullptr;  // LMF_HOST_MAPPED: the device's address of the host data
  void* remap = nullptr;  // engine-owned renumbered copy of a sparse join key (lmf_keymap.cu)
  const void* dptr() const {
    if (remap) return remap;
    return on_host == LMF_HOST_COPY ? dev : on_host == LMF_HOST_MAPPED ? mapped : data;
  }
  size_t esize() const { return dtype == LMF_F64 ? 8 : 4; }
};

struct RelationH {
  std::string name;
  int64_t nrows = 0;
  std::vector<ColumnH> cols;
  int parent = -1;
  std::string key;            // join attribute towards the parent
  std::vector<int> children;
  int K = 0;                  // child key space 0..K-1
  int max_mult = 0;           // largest number of rows sharing a key
  // the parent's foreign-key column of this edge (used when a plan reverses it)
  int fk_K = 0, fk_mult = 0;
  bool fk_ok = true;
  int find(const std::string& n) const {
    for (size_t i = 0; i < cols.size(); ++i)
      if (cols[i].name == n) return (int)i;
    return -1;
  }
};

struct FactorH {
  std::string attr;
  int kind, power;
  double thr;
};
struct AggH {
  std::vector<std::string> gb;
  std::vector<FactorH> f;
};

// ---- plan ------------------------------------------------------------------
// a device allocation freed when its scope ends, error returns included
struct DevScratch {
  void* p = nullptr;
  DevScratch() = default;
  DevScratch(const DevScratch&) = delete;
  DevScratch& operator=(const DevScratch&) = delete;
  ~DevScratch() {
    if (p) cudaFree(p);
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

struct Arena {
  char* base = nullptr;
  size_t size = 0, used = 0;
  size_t take(size_t n) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + n;
    return off;
  }
};

struct GroupH {                  // a probe group of relation `owner`
  int owner;
  std::string fk;                // FK column in owner
  std::vector<int> children;     // child relations
  int K = 0, stride = 0, n_cnt = 0, n_mu = 0, n_cat = 0;
  size_t rec_off = 0;            // arena offset of the record array
  std::vector<int> child_mu_off, child_cat_off;
};

struct RelPlan {
  std::vector<int> own_feat;     // column indices of needed own continuous columns
  std::vector<int> own_cat;      // column indices of needed own categorical columns
  std::vector<int> groups;       // indices into Plan::groups (this relation's children)
  int d = 0;                     // subtree feature count (section mean words)
  int ncat = 0;                  // subtree category count
  bool unique = true;            // every subtree count is 0 or 1
  double maxcnt = 1;             // bound on the subtree count of one key
  std::vector<std::string> feat_names;   // subtree features in section order
  std::vector<std::string> cat_names;    // subtree categories in section order
  std::vector<double> feat_bound;        // max |x| per subtree feature
  // general path buffers
  size_t cnt64_off = 0, S_off = 0, Q_off = 0, sc_off = 0;
  float s_scale[kMaxOwn + kMaxZ];
  double q_scale = 1;
  int group = -1, slot = -1;     // the parent's group holding this relation, child index in it
};

struct Plan {
  lmf_plan_opts opts{};
  std::vector<GroupH> groups;
  std::vector<RelPlan> rp;
  std::vector<int> post;         // non-root relations, children before parents
  Arena arena;
  size_t zero_off = 0, zero_len = 0;
  // root
  RootParams rootp{};
  int mp = 16, grid = 1;
  int64_t n_tiles = 0;
  size_t smem = 0;
  size_t part_off = 0, cntp_off = 0, G_off = 0, count_off = 0, status_off = 0;
  std::map<std::string, int> zidx;          // feature -> z index
  std::map<std::string, int> rowcat;        // category -> row category index
  std::map<std::string, std::pair<int, int>> catword;  // category -> (root group, word)
  std::map<std::string, int> feat_group;    // feature -> root group owning it (-1 root)
  std::vector<RvTask> rv_tasks;
  std::vector<CatViewTask> cv_tasks;
  TaskRanges rv_ranges{}, cv_ranges{};
  std::vector<GroupGram> ggram;
  size_t ggram_off = 0, ggram_part_off = 0;
  static constexpr int kGgChunks = 2048;  // key ranges (one warp each) of the key-level Gram
  // key-level plan (lmf_root_lean.cuh): the row Gram covers the root's
  // features only, every block with a view mean comes from CrossGram /
  // GroupGram over the reverse views
  bool lean = false;
  int lean_mpx = 4;
  std::vector<CrossGram> cgram;
  std::vector<CrossPair> cpairs;
  std::vector<FixMeans> fixm;    // per root group with fixed-point mean images
  // work items of the key-level tasks and the final placement, in `aux`
  std::vector<RvItem> rv_items;
  std::vector<CvPairItem> cv_pair_items;
  std::vector<CvMeanItem> cv_mean_items;
  std::vector<OutItem> out_items;
  int rv_item_cells = 0, cv_pair_cells = 0;
  // category indexes of the COUNT tables read off category views
  std::vector<CatIndex> cat_idx;
  size_t cat_idx_off = 0;
  int64_t cat_idx_maxK = 0;
  bool rv_wide = false;          // some reverse-view task is too wide for a block's table
  void* aux = nullptr;
  size_t aux_rv = 0, aux_cvp = 0, aux_cvm = 0, aux_out = 0;
  size_t cgram_off = 0, cpair_off = 0, cgram_part_off = 0;
  size_t cvtask_off = 0;
  int64_t cv_max_cells = 0;
  std::vector<DirectAgg> direct;
  std::vector<CorrTask> corr;
  std::vector<OutMap> maps;
  size_t rvtask_off = 0, direct_off = 0, corr_off = 0, maps_off = 0;
  int max_group_K = 0;
  // filtered aggregates (tree-node batches)
  std::unique_ptr<TreePlan> tree;
  // tensor-core Gram
  std::unique_ptr<GramTcPlan> tc;
  // root scan compiled for this plan (null: the interpreted kernel)
  cudaKernel_t jit_plain = nullptr, jit_tc = nullptr, jit_lean = nullptr;
  bool dry = false;             // built for its features only: not runnable
  double run_log2 = 0;          // mean over probe groups of log2(rows per run of equal keys)
  // results
  int64_t n_i64 = 0, n_f64 = 0;
  size_t res_i64_off = 0, res_f64_off = 0;
  std::vector<int32_t> agg_dtype;
  std::vector<int64_t> agg_off, agg_n;
  // graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t graph_stream = nullptr;
  int n_kernels = 0;
  bool unique_all = true;
  int n_views = 0, n_gram = 0, n_grouped = 0, n_filtered = 0;
  // orientation of the join tree from the plan's root
  int root = 0;
  bool merge = true;
  std::vector<int> par, K, mult;
  std::vector<std::string> key;
  std::vector<std::vector<int>> kids;
  bool root_scan = true;         // some aggregate needs the Gram / counts / grouped tables
  template <class T>
  T* at(size_t off) const { return reinterpret_cast<T*>(arena.base + off); }
  // device resources of the plan; a plan that fails half-way releases what it
  // had allocated when it is dropped
  // per-query roots (LMF_ROOT_PER_QUERY): the hidden batches, each planned at
  // its own root, whose results this plan's arrays collect
  std::vector<int> subs;
  std::vector<ResultCopy> copies;
  size_t copies_off = 0;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (graph_stream) cudaStreamDestroy(graph_stream);
    if (arena.base) cudaFree(arena.base);
    if (aux) cudaFree(aux);
    aux = nullptr;
    exec = nullptr;
    graph = nullptr;
    graph_stream = nullptr;
    arena.base = nullptr;
  }
  Plan() = default;
  Plan(const Plan&) = delete;
  Plan& operator=(const Plan&) = delete;
  ~Plan() { release(); }
};

struct BatchH {
  std::vector<AggH> aggs;
  std::unique_ptr<Plan> plan;
  cudaStream_t last_stream = nullptr;
};

}  // namespace

struct lmf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  std::vector<RelationH> rels;
  bool joined = false;
  int root = -1;
  std::vector<std::unique_ptr<BatchH>> batches;
  std::string err;
  // dry planning (plan choice): plans are built for their features only, the
  // plan-time compile is skipped and its sources are collected here instead
  bool dry = false;
  std::vector<std::pair<std::string, const char*>> dry_sources;
};

namespace {

lmf_status fail(lmf_ctx* c, lmf_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

#define CUDA_TRY(ctx, expr)                                                              \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? LMF_ERR_OOM : LMF_ERR_CUDA,      \
                  "%s: %s", #expr, cudaGetErrorString(e_));                              \
  } while (0)

void free_plan(Plan* p) {
  if (p) p->release();
}

// min and max of an int32 device column (n > 0) through the scratch pair mm
lmf_status key_range(lmf_ctx* c, const int32_t* col, int64_t n, int* mm, int out[2]) {
  int h_mm[2] = {0x7fffffff, -0x7fffffff - 1};
  CUDA_TRY(c, cudaMemcpy(mm, h_mm, sizeof(h_mm), cudaMemcpyHostToDevice));
  CUDA_TRY(c, launch_key_stats(col, n, nullptr, 0, mm, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(h_mm, mm, sizeof(h_mm), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  out[0] = h_mm[0];
  out[1] = h_mm[1];
  return LMF_OK;
}

// Join attribute `a` has child keys too sparse for direct addressing: every
// column of that name on either side of an edge keyed on it gets an
// engine-owned copy holding the rank of its values among the distinct child
// keys (lmf_keymap.cu), so the key index stays a direct-addressed array.
lmf_status renumber_attribute(lmf_ctx* c, const std::string& a, int* mm) {
  std::vector<std::pair<int, int>> cols;  // (relation, column): child sides first
  auto add = [&](int r, int col) {
    for (auto& x : cols)
      if (x.first == r && x.second == col) return;
    cols.push_back({r, col});
  };
  const int nrel = (int)c->rels.size();
  for (int ch = 0; ch < nrel; ++ch)
    if (c->rels[ch].parent >= 0 && c->rels[ch].key == a) add(ch, c->rels[ch].find(a));
  const int n_child = (int)cols.size();
  for (int ch = 0; ch < nrel; ++ch)
    if (c->rels[ch].parent >= 0 && c->rels[ch].key == a) {
      const int p = c->rels[ch].parent;
      add(p, c->rels[p].find(a));
    }
  int max_key = -1;
  for (int i = 0; i < n_child; ++i) {
    const RelationH& R = c->rels[cols[i].first];
    if (R.nrows == 0) continue;
    int mmv[2];
    lmf_status st = key_range(c, static_cast<const int32_t*>(R.cols[cols[i].second].dptr()), R.nrows, mm, mmv);
    if (st) return st;
    if (mmv[0] < 0) return fail(c, LMF_ERR_KEY, "relation %s: negative key %d", R.name.c_str(), mmv[0]);
    max_key = std::max(max_key, mmv[1]);
  }
  if (max_key < 0) return LMF_OK;  // no child rows
  std::vector<const int32_t*> in;
  std::vector<int64_t> rows;
  std::vector<int32_t*> out;
  struct Owned {
    std::vector<int32_t*>* v;
    bool keep = false;
    ~Owned() {
      if (!keep)
        for (int32_t* p : *v)
          if (p) cudaFree(p);
    }
  } owned{&out};
  for (auto& [r, col] : cols) {
    const RelationH& R = c->rels[r];
    int32_t* d = nullptr;
    if (R.nrows > 0) CUDA_TRY(c, cudaMalloc(&d, sizeof(int32_t) * (size_t)R.nrows));
    in.push_back(static_cast<const int32_t*>(R.cols[col].dptr()));
    rows.push_back(R.nrows);
    out.push_back(d);
  }
  int64_t n_keys = 0;
  CUDA_TRY(c, keymap_renumber(in.data(), rows.data(), (int)cols.size(), n_child, max_key, out.data(), &n_keys,
                              c->stream));
  for (size_t i = 0; i < cols.size(); ++i) c->rels[cols[i].first].cols[cols[i].second].remap = out[i];
  owned.keep = true;
  return LMF_OK;
}

// which relation holds attribute `a` (non-key attributes are unique)
int owner_of(const lmf_ctx* c, const std::string& a, int* col) {
  for (size_t r = 0; r < c->rels.size(); ++r) {
    int i = c->rels[r].find(a);
    if (i >= 0 && c->rels[r].cols[i].role != LMF_KEY) {
      *col = i;
      return (int)r;
    }
  }
  return -1;
}

int fixp_exp(double bound) {  // exponent e with bound * 2^e <= 2^62
  if (!(bound > 0) || !std::isfinite(bound)) return 40;
  int e = 62 - (int)std::ceil(std::log2(bound));
  return std::max(-120, std::min(120, e));
}

}  // namespace

// ============================================================================
extern "C" {

const char* lmf_status_string(lmf_status s) {
  switch (s) {
    case LMF_OK: return "ok";
    case LMF_ERR_ARG: return "bad argument";
    case LMF_ERR_NOT_TREE: return "edges do not form a join tree";
    case LMF_ERR_DTYPE: return "column dtype or role does not fit its use";
    case LMF_ERR_KEY: return "key or category out of range";
    case LMF_ERR_OOM: return "device out of memory";
    case LMF_ERR_CUDA: return "CUDA error";
    case LMF_ERR_TIMEOUT: return "device wait timed out";
    case LMF_ERR_OVERFLOW: return "exact count overflow";
    case LMF_ERR_STATE: return "call out of order";
    case LMF_ERR_UNSUPPORTED: return "unsupported aggregate shape";
    default: return "unknown status";
  }
}

const char* lmf_error_message(lmf_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

lmf_status lmf_create(int device, lmf_ctx** out) {
  if (!out) return LMF_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return LMF_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return LMF_ERR_CUDA;
  auto* c = new lmf_ctx();
  c->device = device;
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return LMF_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  *out = c;
  return LMF_OK;
}

lmf_status lmf_destroy(lmf_ctx* c) {
  if (!c) return LMF_ERR_ARG;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  for (auto& b : c->batches)
    if (b && b->plan) free_plan(b->plan.get());
  for (auto& r : c->rels)
    for (auto& col : r.cols) {
      if (col.dev) cudaFree(col.dev);
      if (col.remap) cudaFree(col.remap);
    }
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return LMF_OK;
}

lmf_status lmf_register_relation(lmf_ctx* c, const char* name, int64_t nrows, const lmf_column* cols,
                                 int ncols, int* rel_id) {
  if (!c || !name || nrows < 0 || ncols < 0 || (ncols > 0 && !cols) || !rel_id)
    return fail(c, LMF_ERR_ARG, "register_relation: bad argument");
  if (c->joined) return fail(c, LMF_ERR_STATE, "register_relation after declare_join");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, LMF_ERR_CUDA, "cudaSetDevice");
  RelationH r;
  r.name = name;
  r.nrows = nrows;
  // on any failure below, the staging copies made so far are freed
  struct Staged {
    RelationH* r;
    bool keep = false;
    ~Staged() {
      if (!keep)
        for (auto& col : r->cols)
          if (col.dev) cudaFree(col.dev);
    }
  } staged{&r};
  for (int i = 0; i < ncols; ++i) {
    const lmf_column& s = cols[i];
    if (!s.name || (!s.data && nrows > 0)) return fail(c, LMF_ERR_ARG, "column %d: null name/data", i);
    if (r.find(s.name) >= 0) return fail(c, LMF_ERR_ARG, "duplicate column %s", s.name);
    bool ok = (s.role == LMF_KEY || s.role == LMF_CAT) ? s.dtype == LMF_I32
              : s.role == LMF_CONT                     ? (s.dtype == LMF_F32 || s.dtype == LMF_F64)
                                                       : false;
    if (!ok) return fail(c, LMF_ERR_DTYPE, "column %s: dtype %d does not fit role %d", s.name, s.dtype, s.role);
    if (s.role == LMF_CAT && s.cat_domain <= 0)
      return fail(c, LMF_ERR_ARG, "column %s: cat_domain must be positive", s.name);
    if (s.on_host < LMF_DEVICE || s.on_host > LMF_HOST_MAPPED)
      return fail(c, LMF_ERR_ARG, "column %s: on_host %d", s.name, s.on_host);
    ColumnH h{s.name, s.dtype, s.role, s.cat_domain, s.on_host, s.data};
    if (h.on_host == LMF_HOST_MAPPED && nrows > 0) {
      cudaPointerAttributes at{};
      if (cudaPointerGetAttributes(&at, s.data) != cudaSuccess || at.type != cudaMemoryTypeHost ||
          at.devicePointer == nullptr) {
        cudaGetLastError();
        return fail(c, LMF_ERR_ARG, "column %s: LMF_HOST_MAPPED needs page-locked, device-mapped host memory", s.name);
      }
      h.mapped = at.devicePointer;
    }
    if (h.on_host == LMF_HOST_COPY && nrows > 0) {
      if (cudaMalloc(&h.dev, (size_t)nrows * h.esize()) != cudaSuccess)
        return fail(c, LMF_ERR_OOM, "staging buffer for %s", s.name);
      r.cols.push_back(h);
      const cudaError_t e = cudaMemcpy(h.dev, h.data, (size_t)nrows * h.esize(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return fail(c, LMF_ERR_CUDA, "column %s: host copy: %s", s.name, cudaGetErrorString(e));
      continue;
    }
    r.cols.push_back(h);
  }
  for (auto& other : c->rels) {
    if (other.name == r.name) return fail(c, LMF_ERR_ARG, "duplicate relation %s", name);
    for (auto& col : r.cols)
      if (col.role != LMF_KEY && other.find(col.name) >= 0)
        return fail(c, LMF_ERR_UNSUPPORTED, "non-key attribute %s occurs in %s and %s", col.name.c_str(),
                    other.name.c_str(), name);
  }
  *rel_id = (int)c->rels.size();
  staged.keep = true;
  c->rels.push_back(std::move(r));
  return LMF_OK;
}

lmf_status lmf_declare_join(lmf_ctx* c, int n_edges, const int* parent_rel, const int* child_rel,
                            const char* const* key_attr) {
  if (!c) return LMF_ERR_ARG;
  if (c->joined) return fail(c, LMF_ERR_STATE, "declare_join called twice");
  const int n = (int)c->rels.size();
  if (n == 0) return fail(c, LMF_ERR_STATE, "no relations");
  if (n_edges != n - 1) return fail(c, LMF_ERR_NOT_TREE, "%d relations need %d edges", n, n - 1);
  if (n_edges > 0 && (!parent_rel || !child_rel || !key_attr)) return fail(c, LMF_ERR_ARG, "null edges");
  cudaSetDevice(c->device);
  for (auto& r : c->rels) {
    r.parent = -1;
    r.children.clear();
  }
  for (int e = 0; e < n_edges; ++e) {
    int p = parent_rel[e], ch = child_rel[e];
    if (p < 0 || p >= n || ch < 0 || ch >= n || p == ch || !key_attr[e])
      return fail(c, LMF_ERR_ARG, "edge %d: bad relation id", e);
    if (c->rels[ch].parent != -1) return fail(c, LMF_ERR_NOT_TREE, "relation %d has two parents", ch);
    c->rels[ch].parent = p;
    c->rels[ch].key = key_attr[e];
    c->rels[p].children.push_back(ch);
  }
  int root = -1;
  for (int r = 0; r < n; ++r)
    if (c->rels[r].parent == -1) {
      if (root != -1) return fail(c, LMF_ERR_NOT_TREE, "more than one root");
      root = r;
    }
  if (root < 0) return fail(c, LMF_ERR_NOT_TREE, "no root (cycle)");
  // reachability from the root (no cycles)
  std::vector<int> seen(n, 0), stack{root};
  int cnt = 0;
  while (!stack.empty()) {
    int r = stack.back();
    stack.pop_back();
    if (seen[r]++) return fail(c, LMF_ERR_NOT_TREE, "cycle");
    ++cnt;
    for (int ch : c->rels[r].children) stack.push_back(ch);
  }
  if (cnt != n) return fail(c, LMF_ERR_NOT_TREE, "edges do not connect all relations");
  // edge keys: int32 key columns on both sides; no other shared attribute
  for (int ch = 0; ch < n; ++ch) {
    RelationH& R = c->rels[ch];
    if (R.parent < 0) continue;
    RelationH& P = c->rels[R.parent];
    int kc = R.find(R.key), kp = P.find(R.key);
    if (kc < 0 || kp < 0) return fail(c, LMF_ERR_ARG, "edge %s-%s: key %s missing", P.name.c_str(), R.name.c_str(), R.key.c_str());
    if (R.cols[kc].role != LMF_KEY || P.cols[kp].role != LMF_KEY)
      return fail(c, LMF_ERR_DTYPE, "edge key %s must have role LMF_KEY on both sides", R.key.c_str());
    for (auto& col : R.cols)
      if (col.name != R.key && P.find(col.name) >= 0)
        return fail(c, LMF_ERR_UNSUPPORTED, "%s and %s share %s besides their edge key", P.name.c_str(),
                    R.name.c_str(), col.name.c_str());
  }
  // running intersection for key names shared by non-adjacent relations: every
  // relation on the path must carry the name
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b)
      for (auto& col : c->rels[a].cols) {
        if (c->rels[b].find(col.name) < 0) continue;
        // path a -> lca -> b
        std::vector<int> pa, pb;
        for (int x = a; x >= 0; x = c->rels[x].parent) pa.push_back(x);
        for (int x = b; x >= 0; x = c->rels[x].parent) pb.push_back(x);
        std::set<int> sa(pa.begin(), pa.end());
        int lca = b;
        for (int x : pb)
          if (sa.count(x)) {
            lca = x;
            break;
          }
        for (int x = a; x != lca; x = c->rels[x].parent)
          if (c->rels[x].find(col.name) < 0) return fail(c, LMF_ERR_NOT_TREE, "attribute %s breaks running intersection", col.name.c_str());
        for (int x = b; x != lca; x = c->rels[x].parent)
          if (c->rels[x].find(col.name) < 0) return fail(c, LMF_ERR_NOT_TREE, "attribute %s breaks running intersection", col.name.c_str());
        if (c->rels[lca].find(col.name) < 0) return fail(c, LMF_ERR_NOT_TREE, "attribute %s breaks running intersection", col.name.c_str());
      }
  // key index of every child: range and multiplicity (A1)
  DevScratch mm_buf;
  CUDA_TRY(c, cudaMalloc(&mm_buf.p, 2 * sizeof(int)));
  int* mm = mm_buf.as<int>();
  std::set<std::string> renumbered;  // attributes whose keys were renumbered
  for (int ch = 0; ch < n; ++ch) {
    RelationH& R = c->rels[ch];
    if (R.parent < 0) continue;
    const ColumnH& kc = R.cols[R.find(R.key)];
    if (R.nrows == 0) {
      R.K = 0;
      R.max_mult = 0;
      continue;
    }
    int h_mm[2] = {0x7fffffff, -0x7fffffff - 1};
    CUDA_TRY(c, cudaMemcpy(mm, h_mm, sizeof(h_mm), cudaMemcpyHostToDevice));
    CUDA_TRY(c, launch_key_stats(static_cast<const int32_t*>(kc.dptr()), R.nrows, nullptr, 0, mm, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(h_mm, mm, sizeof(h_mm), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (h_mm[0] < 0) return fail(c, LMF_ERR_KEY, "relation %s: negative key %d", R.name.c_str(), h_mm[0]);
    if ((int64_t)h_mm[1] >= 4 * R.nrows + 4096 && !renumbered.count(R.key)) {
      // too sparse for direct addressing: renumber the attribute and start
      // the index again (children indexed so far may share it)
      lmf_status st = renumber_attribute(c, R.key, mm);
      if (st) return st;
      renumbered.insert(R.key);
      ch = -1;
      continue;
    }
    R.K = h_mm[1] + 1;
    DevScratch hist_buf;
    CUDA_TRY(c, cudaMalloc(&hist_buf.p, sizeof(unsigned int) * R.K));
    unsigned int* hist = hist_buf.as<unsigned int>();
    CUDA_TRY(c, cudaMemsetAsync(hist, 0, sizeof(unsigned int) * R.K, c->stream));
    CUDA_TRY(c, launch_key_stats(static_cast<const int32_t*>(kc.dptr()), R.nrows, hist, R.K, nullptr, c->stream));
    std::vector<unsigned int> h(R.K);
    CUDA_TRY(c, cudaMemcpyAsync(h.data(), hist, sizeof(unsigned int) * R.K, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    R.max_mult = (int)*std::max_element(h.begin(), h.end());
  }
  // the parent's side of every edge (its foreign-key column), which becomes the
  // child key when a plan roots the tree below that edge; negative values never
  // join, sparse columns make the edge irreversible
  for (int ch = 0; ch < n; ++ch) {
    RelationH& R = c->rels[ch];
    if (R.parent < 0) continue;
    const RelationH& P = c->rels[R.parent];
    R.fk_K = 0;
    R.fk_mult = 0;
    R.fk_ok = true;
    if (P.nrows == 0) continue;
    const ColumnH& fc = P.cols[P.find(R.key)];
    int h_mm[2] = {0x7fffffff, -0x7fffffff - 1};
    CUDA_TRY(c, cudaMemcpy(mm, h_mm, sizeof(h_mm), cudaMemcpyHostToDevice));
    CUDA_TRY(c, launch_key_stats(static_cast<const int32_t*>(fc.dptr()), P.nrows, nullptr, 0, mm, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(h_mm, mm, sizeof(h_mm), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (h_mm[1] < 0) continue;
    if ((int64_t)h_mm[1] >= 4 * P.nrows + 4096) {
      R.fk_ok = false;
      continue;
    }
    R.fk_K = h_mm[1] + 1;
    DevScratch hist_buf;
    CUDA_TRY(c, cudaMalloc(&hist_buf.p, sizeof(unsigned int) * R.fk_K));
    unsigned int* hist = hist_buf.as<unsigned int>();
    CUDA_TRY(c, cudaMemsetAsync(hist, 0, sizeof(unsigned int) * R.fk_K, c->stream));
    CUDA_TRY(c, launch_key_stats(static_cast<const int32_t*>(fc.dptr()), P.nrows, hist, R.fk_K, nullptr, c->stream));
    std::vector<unsigned int> h(R.fk_K);
    CUDA_TRY(c, cudaMemcpyAsync(h.data(), hist, sizeof(unsigned int) * R.fk_K, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    R.fk_mult = (int)*std::max_element(h.begin(), h.end());
  }
  c->root = root;
  c->joined = true;
  return LMF_OK;
}

lmf_status lmf_declare_batch(lmf_ctx* c, const lmf_agg_spec* aggs, int n, int* batch_id) {
  if (!c || n < 0 || (n > 0 && !aggs) || !batch_id) return fail(c, LMF_ERR_ARG, "declare_batch: bad argument");
  if (!c->joined) return fail(c, LMF_ERR_STATE, "declare_batch before declare_join");
  auto b = std::make_unique<BatchH>();
  for (int a = 0; a < n; ++a) {
    const lmf_agg_spec& s = aggs[a];
    if (s.n_group_by < 0 || s.n_group_by > LMF_MAX_GROUP_BY || s.n_factors < 0 ||
        s.n_factors > LMF_MAX_FACTORS || (s.n_factors > 0 && !s.factors))
      return fail(c, LMF_ERR_ARG, "aggregate %d: bad sizes", a);
    AggH h;
    for (int g = 0; g < s.n_group_by; ++g) {
      if (!s.group_by[g]) return fail(c, LMF_ERR_ARG, "aggregate %d: null group-by", a);
      int col, r = owner_of(c, s.group_by[g], &col);
      if (r < 0) return fail(c, LMF_ERR_ARG, "aggregate %d: unknown attribute %s", a, s.group_by[g]);
      if (c->rels[r].cols[col].role != LMF_CAT)
        return fail(c, LMF_ERR_DTYPE, "aggregate %d: group-by %s is not categorical", a, s.group_by[g]);
      h.gb.push_back(s.group_by[g]);
    }
    for (int f = 0; f < s.n_factors; ++f) {
      const lmf_factor& x = s.factors[f];
      if (!x.attr) return fail(c, LMF_ERR_ARG, "aggregate %d: null factor attribute", a);
      int col, r = owner_of(c, x.attr, &col);
      if (r < 0) return fail(c, LMF_ERR_ARG, "aggregate %d: unknown attribute %s", a, x.attr);
      if (c->rels[r].cols[col].role != LMF_CONT)
        return fail(c, LMF_ERR_DTYPE, "aggregate %d: factor on non-continuous %s", a, x.attr);
      if (x.kind == LMF_POW) {
        if (x.power != 1 && x.power != 2) return fail(c, LMF_ERR_ARG, "aggregate %d: power %d", a, x.power);
      } else if (x.kind != LMF_LE && x.kind != LMF_GT) {
        return fail(c, LMF_ERR_ARG, "aggregate %d: factor kind %d", a, x.kind);
      } else if (std::isnan(x.threshold)) {  // 1[x <= NaN] orders nothing
        return fail(c, LMF_ERR_ARG, "aggregate %d: NaN threshold on %s", a, x.attr);
      }
      h.f.push_back({x.attr, x.kind, x.power, x.threshold});
    }
    b->aggs.push_back(std::move(h));
  }
  *batch_id = (int)c->batches.size();
  c->batches.push_back(std::move(b));
  return LMF_OK;
}

}  // extern "C"

// ============================================================================
// planner
namespace {

struct AggClass {
  int kind;              // 0 gram, 1 grouped, 2 filtered
  std::vector<std::string> mono;   // monomial attributes with multiplicity (degree <= 2)
};

lmf_status classify(lmf_ctx* c, const AggH& a, int idx, AggClass* out) {
  bool filt = false;
  out->mono.clear();
  for (auto& f : a.f) {
    if (f.kind == LMF_POW) {
      for (int e = 0; e < f.power; ++e) out->mono.push_back(f.attr);
    } else {
      filt = true;
    }
  }
  if (filt) {
    if (!a.gb.empty()) return fail(c, LMF_ERR_UNSUPPORTED, "aggregate %d: group-by with threshold factors", idx);
    if (out->mono.size() > 2) return fail(c, LMF_ERR_UNSUPPORTED, "aggregate %d: filtered monomial of degree > 2", idx);
    out->kind = 2;
    return LMF_OK;
  }
  if (!a.gb.empty()) {
    if (out->mono.size() > 1)
      return fail(c, LMF_ERR_UNSUPPORTED, "aggregate %d: grouped monomial of degree > 1", idx);
    out->kind = 1;
    return LMF_OK;
  }
  if (out->mono.size() > 2) return fail(c, LMF_ERR_UNSUPPORTED, "aggregate %d: monomial of degree > 2", idx);
  out->kind = 0;
  return LMF_OK;
}

// post-order layout of the views
void layout_rel(lmf_ctx* c, Plan& P, int r, const std::set<std::string>& need_feat,
                const std::set<std::string>& need_cat) {
  RelationH& R = c->rels[r];
  RelPlan& rp = P.rp[r];
  for (size_t i = 0; i < R.cols.size(); ++i) {
    if (R.cols[i].role == LMF_CONT && need_feat.count(R.cols[i].name)) rp.own_feat.push_back((int)i);
    if (R.cols[i].role == LMF_CAT && need_cat.count(R.cols[i].name)) rp.own_cat.push_back((int)i);
  }
  // groups: children sharing the FK column name
  std::vector<std::string> order;
  std::map<std::string, int> gid;
  for (int ch : P.kids[r]) {
    // merged: one record array per parent key; unmerged: one per child view
    const std::string k = P.merge ? P.key[ch] : P.key[ch] + "#" + c->rels[ch].name;
    if (!gid.count(k)) {
      GroupH g;
      g.owner = r;
      g.fk = P.key[ch];
      gid[k] = (int)P.groups.size();
      rp.groups.push_back((int)P.groups.size());
      P.groups.push_back(g);
    }
    P.groups[gid[k]].children.push_back(ch);
  }
  for (int gi : rp.groups)
    for (int ch : P.groups[gi].children) layout_rel(c, P, ch, need_feat, need_cat);
  // own section
  rp.unique = (r == P.root) || P.mult[r] <= 1;
  rp.maxcnt = (r == P.root) ? 1.0 : std::max(1, P.mult[r]);
  for (int i : rp.own_feat) rp.feat_names.push_back(R.cols[i].name);
  for (int i : rp.own_cat) rp.cat_names.push_back(R.cols[i].name);
  for (int gi : rp.groups) {
    GroupH& g = P.groups[gi];
    g.n_cnt = (int)g.children.size();
    g.n_mu = 0;
    g.n_cat = 0;
    g.K = 0;
    for (size_t q = 0; q < g.children.size(); ++q) {
      int ch = g.children[q];
      RelPlan& cp = P.rp[ch];
      cp.group = gi;
      cp.slot = (int)q;
      g.child_mu_off.push_back(g.n_cnt + g.n_mu);
      g.n_mu += cp.d;
      g.K = std::max(g.K, P.K[ch]);
      rp.unique = rp.unique && cp.unique;
      rp.maxcnt *= cp.maxcnt;
      for (auto& f : cp.feat_names) rp.feat_names.push_back(f);
    }
    for (size_t q = 0; q < g.children.size(); ++q) {
      int ch = g.children[q];
      RelPlan& cp = P.rp[ch];
      g.child_cat_off.push_back(g.n_cnt + g.n_mu + g.n_cat);
      g.n_cat += cp.ncat;
      for (auto& f : cp.cat_names) rp.cat_names.push_back(f);
    }
    g.stride = (g.n_cnt + g.n_mu + g.n_cat + 3) & ~3;
  }
  rp.d = (int)rp.feat_names.size();
  rp.ncat = (int)rp.cat_names.size();
  if (r != P.root) P.post.push_back(r);
}

}  // namespace

namespace {

// Orient the declared tree from `root`: parent, edge key, children, and the
// key space and multiplicity of every relation's key towards its parent (a
// reversed edge uses the old parent's foreign-key column as that key).
lmf_status orient(lmf_ctx* c, Plan& P, int root) {
  const int n = (int)c->rels.size();
  P.root = root;
  P.par.assign(n, -1);
  P.key.assign(n, std::string());
  P.kids.assign(n, std::vector<int>());
  P.K.assign(n, 0);
  P.mult.assign(n, 0);
  struct Adj {
    int to;
    std::string key;
    int K, mult;
    bool ok;
  };
  std::vector<std::vector<Adj>> adj(n);
  for (int r = 0; r < n; ++r)
    for (int ch : c->rels[r].children) {
      const RelationH& R = c->rels[ch];
      adj[r].push_back({ch, R.key, R.K, R.max_mult, true});
      adj[ch].push_back({r, R.key, R.fk_K, R.fk_mult, R.fk_ok});
    }
  std::vector<int> seen(n, 0), queue{root};
  seen[root] = 1;
  for (size_t h = 0; h < queue.size(); ++h) {
    const int u = queue[h];
    for (const Adj& a : adj[u]) {
      if (seen[a.to]) continue;
      if (!a.ok)
        return fail(c, LMF_ERR_UNSUPPORTED, "cannot root at %s: the key column %s of %s is too sparse",
                    c->rels[root].name.c_str(), a.key.c_str(), c->rels[a.to].name.c_str());
      seen[a.to] = 1;
      P.par[a.to] = u;
      P.key[a.to] = a.key;
      P.K[a.to] = a.K;
      P.mult[a.to] = a.mult;
      P.kids[u].push_back(a.to);
      queue.push_back(a.to);
    }
  }
  return LMF_OK;
}

// Root rule of Sec. 3.3 for one batch: every query gives each relation the
// fraction of its group-by attributes held there (an equal share of all
// relations when it has none); the root is the relation with the largest total
// weight, ties going to the largest relation.
int heuristic_root(lmf_ctx* c, const BatchH& B) {
  const int n = (int)c->rels.size();
  std::vector<double> w(n, 0.0);
  for (const auto& a : B.aggs) {
    if (a.gb.empty()) {
      for (int r = 0; r < n; ++r) w[r] += 1.0 / n;
      continue;
    }
    for (const auto& g : a.gb) {
      int col, r = owner_of(c, g, &col);
      if (r >= 0) w[r] += 1.0 / a.gb.size();
    }
  }
  int best = 0;
  for (int r = 1; r < n; ++r) {
    const double d = w[r] - w[best];
    if (d > 1e-12 || (std::fabs(d) <= 1e-12 && c->rels[r].nrows > c->rels[best].nrows)) best = r;
  }
  return best;
}

lmf_status plan_with_root(lmf_ctx* c, int batch_id, const lmf_plan_opts& opts, int root);
lmf_status plan_per_query(lmf_ctx* c, int batch_id, const lmf_plan_opts& opts);

}  // namespace

extern "C" lmf_status lmf_plan(lmf_ctx* c, int batch_id, const lmf_plan_opts* opts) {
  if (!c || batch_id < 0 || batch_id >= (int)c->batches.size()) return fail(c, LMF_ERR_ARG, "plan: bad batch id");
  if (!c->joined) return fail(c, LMF_ERR_STATE, "plan before declare_join");
  lmf_plan_opts o{};
  if (opts) {
    o = *opts;
  } else {
    o.precision = LMF_PREC_SPLIT_BF16;
    o.batching = LMF_BATCH_GRAPH;
  }
  BatchH& B = *c->batches[batch_id];
  switch (o.root_mode) {
    case LMF_ROOT_DECLARED:
      return plan_with_root(c, batch_id, o, c->root);
    case LMF_ROOT_EXPLICIT:
      if (o.root_rel < 0 || o.root_rel >= (int)c->rels.size()) return fail(c, LMF_ERR_ARG, "plan: bad root_rel");
      return plan_with_root(c, batch_id, o, o.root_rel);
    case LMF_ROOT_HEURISTIC: {
      const int r = heuristic_root(c, B);
      lmf_status s = plan_with_root(c, batch_id, o, r);
      // fall back to the declared root when this engine cannot evaluate the
      // batch from the rule's root (e.g. group-by attributes below a fan-out)
      if (s == LMF_ERR_UNSUPPORTED && r != c->root) s = plan_with_root(c, batch_id, o, c->root);
      return s;
    }
    case LMF_ROOT_PER_QUERY:
      return plan_per_query(c, batch_id, o);
    default:
      return fail(c, LMF_ERR_ARG, "plan: root_mode %d", o.root_mode);
  }
}

namespace {

// LMF_LOG=1 in the environment: print every plan, and the stage times of
// profiled runs, to stderr
bool log_enabled() {
  const char* e = std::getenv("LMF_LOG");
  return e && *e && std::strcmp(e, "0") != 0;
}

void log_plan(const lmf_ctx* c, int batch_id, const Plan& P) {
  std::fprintf(stderr,
               "lmf: batch %d planned at root %s: %d views, %d probe groups, z length %d, "
               "%d Gram / %d grouped / %d filtered aggregates\n",
               batch_id, c->rels[P.root].name.c_str(), P.n_views, P.rootp.n_grp, P.rootp.m, P.n_gram,
               P.n_grouped, P.n_filtered);
  for (const GroupH& g : P.groups)
    std::fprintf(stderr, "lmf:   probe group %s.%s: %d keys, %d-byte records (%d counts, %d means, %d categories)\n",
                 c->rels[g.owner].name.c_str(), g.fk.c_str(), g.K, g.stride * 4, g.n_cnt, g.n_mu, g.n_cat);
  std::fprintf(stderr,
               "lmf:   root scan: %s Gram, %s, grid %d, %zu B shared memory per CTA, resident group %d "
               "(%d cells), %d reverse views, %d category views; plan arena %zu bytes\n",
               P.tc ? "split-bf16 tcgen05" : P.lean ? "key-level, root-feature FP32" : "FP32 CUDA-core",
               (P.jit_plain || P.jit_tc || P.jit_lean) ? "compiled" : "interpreted",
               P.grid, P.smem, P.rootp.res_cells > 0 ? P.rootp.res_grp : -1, P.rootp.res_cells, P.rootp.n_rv,
               P.rootp.n_cv, P.arena.size);
}

lmf_status plan_with_root(lmf_ctx* c, int batch_id, const lmf_plan_opts& opts, int root) {
  cudaSetDevice(c->device);
  BatchH& B = *c->batches[batch_id];
  if (B.plan) {
    // the old plan may still run on a caller's stream: wait for the device
    // before its arena and graph go
    cudaDeviceSynchronize();
    B.plan.reset();
    B.last_stream = nullptr;
  }
  auto P = std::make_unique<Plan>();
  P->opts = opts;
  P->merge = opts.no_merge == 0;
  const int nrel = (int)c->rels.size();
  {
    lmf_status s = orient(c, *P, root);
    if (s) return s;
  }
  RelationH& Root = c->rels[root];

  // ---- classify aggregates; needed features and categories
  std::vector<AggClass> cls(B.aggs.size());
  std::set<std::string> need_feat, need_cat;
  for (size_t a = 0; a < B.aggs.size(); ++a) {
    lmf_status s = classify(c, B.aggs[a], (int)a, &cls[a]);
    if (s) return s;
    for (auto& m : cls[a].mono) need_feat.insert(m);
    for (auto& g : B.aggs[a].gb) need_cat.insert(g);
    for (auto& f : B.aggs[a].f) need_feat.insert(f.attr);
  }
  P->rp.resize(nrel);
  layout_rel(c, *P, root, need_feat, need_cat);
  RelPlan& RR = P->rp[root];

  // ---- z layout: [1, root features, root groups' means]
  int m = 1;
  for (int i : RR.own_feat) P->zidx[Root.cols[i].name] = m++;
  int ncat = 0;
  for (size_t q = 0; q < RR.groups.size(); ++q) {
    GroupH& g = P->groups[RR.groups[q]];
    int word = g.n_cnt;
    for (size_t k = 0; k < g.children.size(); ++k) {
      for (auto& f : P->rp[g.children[k]].feat_names) {
        P->zidx[f] = m++;
        P->feat_group[f] = (int)q;
        ++word;
      }
    }
    for (size_t k = 0; k < g.children.size(); ++k)
      for (auto& f : P->rp[g.children[k]].cat_names) {
        P->catword[f] = {(int)q, word++};
        P->rowcat[f] = ncat++;
      }
  }
  for (int i : RR.own_cat) {
    P->rowcat[Root.cols[i].name] = ncat++;
    P->catword[Root.cols[i].name] = {-1, -1};
  }
  for (int i : RR.own_feat) P->feat_group[Root.cols[i].name] = -1;
  if (m > kMaxZ) return fail(c, LMF_ERR_UNSUPPORTED, "batch needs %d features, at most %d", m - 1, kMaxZ - 1);
  if (ncat > kMaxCat) return fail(c, LMF_ERR_UNSUPPORTED, "batch needs %d categories, at most %d", ncat, kMaxCat);
  if (RR.groups.size() > (size_t)kMaxGroups) return fail(c, LMF_ERR_UNSUPPORTED, "too many join keys at the root");
  for (int r = 0; r < nrel; ++r) {
    if ((int)P->rp[r].own_feat.size() > kMaxOwn || (int)P->rp[r].own_cat.size() > kMaxCat ||
        P->rp[r].groups.size() > (size_t)kMaxGroups || P->rp[r].d > kMaxZ)
      return fail(c, LMF_ERR_UNSUPPORTED, "relation %s: too many columns in one view", c->rels[r].name.c_str());
    if (r != root && !P->rp[r].unique && P->rp[r].ncat > 0)
      return fail(c, LMF_ERR_UNSUPPORTED, "group-by attribute below the fanning-out key of %s", c->rels[r].name.c_str());
  }
  for (int r : P->post)
    if (!P->rp[r].unique) P->unique_all = false;

  // ---- value bounds of every needed continuous column (fixed-point scales)
  std::map<std::string, double> bound;
  {
    std::vector<Col> cols;
    std::vector<std::string> names;
    std::vector<int64_t> rows;
    for (int r = 0; r < nrel; ++r)
      for (auto& col : c->rels[r].cols)
        if (col.role == LMF_CONT && need_feat.count(col.name)) {
          cols.push_back({col.dptr(), col.dtype == LMF_F64 ? 2 : 1});
          names.push_back(col.name);
          rows.push_back(c->rels[r].nrows);
        }
    if (!cols.empty()) {
      DevScratch d_buf;
      CUDA_TRY(c, cudaMalloc(&d_buf.p, sizeof(double) * cols.size()));
      double* d = d_buf.as<double>();
      CUDA_TRY(c, cudaMemsetAsync(d, 0, sizeof(double) * cols.size(), c->stream));
      for (size_t i = 0; i < cols.size(); ++i) CUDA_TRY(c, launch_colmaxabs(&cols[i], 1, rows[i], d + i, c->stream));
      std::vector<double> h(cols.size());
      CUDA_TRY(c, cudaMemcpyAsync(h.data(), d, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      for (size_t i = 0; i < h.size(); ++i) bound[names[i]] = h[i];
    }
  }
  const double W = std::max<double>(1.0, (double)Root.nrows) * RR.maxcnt;  // bound on sum of w

  // ---- arena layout
  Arena& A = P->arena;
  A.take(0);
  // zero region first: everything that must start at zero every run
  size_t zero_begin = A.take(0);
  for (auto& g : P->groups) g.rec_off = A.take((size_t)g.K * g.stride * 4);
  for (int r : P->post) {
    RelPlan& rp = P->rp[r];
    if (rp.unique) continue;
    int K = P->groups[rp.group].K;
    int dq = rp.d * (rp.d + 1) / 2;
    rp.cnt64_off = A.take((size_t)K * 8);
    rp.S_off = A.take((size_t)K * rp.d * 8 + 8);
    rp.Q_off = A.take((size_t)K * dq * 8 + 8);
  }
  P->status_off = A.take(16);

  // ---- root parameters
  RootParams& rp = P->rootp;
  rp.N = Root.nrows;
  rp.m = m;
  rp.n_grp = (int)RR.groups.size();
  {
    int zoff = 1 + (int)RR.own_feat.size(), coff = 0;
    for (int q = 0; q < rp.n_grp; ++q) {
      GroupH& g = P->groups[RR.groups[q]];
      rp.grp_zoff[q] = zoff;
      rp.grp_catoff[q] = coff;
      zoff += g.n_mu;
      coff += g.n_cat;
    }
  }
  rp.n_x = (int)RR.own_feat.size();
  for (int i = 0; i < rp.n_x; ++i) {
    const ColumnH& col = Root.cols[RR.own_feat[i]];
    rp.x[i] = {col.dptr(), col.dtype == LMF_F64 ? 2 : 1};
  }
  rp.n_rcat = (int)RR.own_cat.size();
  for (int i = 0; i < rp.n_rcat; ++i) {
    rp.rcat[i] = static_cast<const int32_t*>(Root.cols[RR.own_cat[i]].dptr());
    rp.rcat_dom[i] = Root.cols[RR.own_cat[i]].dom;
  }
  rp.n_rowcat = ncat;

  // ---- key runs: changes between adjacent root rows of every probe group's
  // foreign key.  A key whose runs average 4 rows or more gets its updates
  // summed per run inside a warp; the key with the fewest changes, if its
  // runs average at least kResRun rows (a root sorted on its join attributes,
  // Sec. 3.5), is held per CTA (the resident key)
  constexpr int64_t kResRun = 1024;
  int res_grp = -1;
  std::vector<unsigned long long> changes(rp.n_grp, 0);
  std::vector<int> has_runs(rp.n_grp, 0);
  if (rp.n_grp > 0 && Root.nrows > 1) {
    DevScratch d_buf;
    CUDA_TRY(c, cudaMalloc(&d_buf.p, sizeof(unsigned long long) * rp.n_grp));
    unsigned long long* d = d_buf.as<unsigned long long>();
    CUDA_TRY(c, cudaMemsetAsync(d, 0, sizeof(unsigned long long) * rp.n_grp, c->stream));
    for (int q = 0; q < rp.n_grp; ++q) {
      GroupH& g = P->groups[RR.groups[q]];
      const RelationH& O = c->rels[g.owner];
      CUDA_TRY(c, launch_key_changes(static_cast<const int32_t*>(O.cols[O.find(g.fk)].dptr()), O.nrows, d + q,
                                     c->stream));
    }
    CUDA_TRY(c, cudaMemcpyAsync(changes.data(), d, sizeof(unsigned long long) * rp.n_grp, cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int q = 0; q < rp.n_grp; ++q) {
      P->run_log2 += std::log2((double)Root.nrows / (double)(changes[q] + 1)) / rp.n_grp;
      has_runs[q] = (int64_t)(changes[q] + 1) * 4 <= Root.nrows;
      if (P->unique_all && Root.nrows >= 2 * kResRun && (int64_t)(changes[q] + 1) * kResRun <= Root.nrows &&
          (res_grp < 0 || changes[q] < changes[res_grp]))
        res_grp = q;
    }
  }

  const int sorted_q = res_grp;  // the first sort key's probe group (-1: the root is not sorted so)
  // ---- key-level form (lmf_root_lean.cuh): every child key unique, plain
  // precision, a compiled scan, at least one probe group and one feature, and
  // some foreign key in runs (on a root in no useful order every reverse-view
  // update is a reduction of its own: the row-level form is faster there)
  bool any_runs = false;
  for (int q = 0; q < rp.n_grp; ++q) any_runs = any_runs || has_runs[q];
  P->lean = any_runs && P->unique_all && rp.n_grp >= 1 && m > 1 && Root.nrows > 0 &&
            P->opts.precision == LMF_PREC_PLAIN_FP32 && !(P->opts.flags & (LMF_PLAN_NO_JIT | LMF_PLAN_ROW_GRAM)) &&
            jit_available();
  std::vector<size_t> deferred;   // grouped sums of another group's mean, placed with the carriers

  // ---- grouped aggregates
  std::vector<size_t> rv_hist_off(rp.n_grp, 0), rv_R_off(rp.n_grp, 0);
  std::vector<std::vector<int>> rv_slots(rp.n_grp);     // z index per slot
  std::vector<int> rv_used(rp.n_grp, 0);
  struct GPlan {
    int mode; int grp; int slot; int mu_word; int direct; double scale; int64_t cells; size_t out_off; int cache_off;
    int res_off, res_q, res_word, res_n, res_lanes;
    int cv, cv_aword, cv_afirst, cv_doma;  // COUNT table read off category view cv (-1: none)
    int cv_mode, cv_muword;                // 1: SUM of a mean of the view's keying group grouped by b
  };
  // category views: (keying group, row category of b) -> view
  struct CvPlan { int grp, bcat, bgrp, dom; size_t off; int res_off; };
  std::vector<CvPlan> cvs;
  std::map<std::pair<int, int>, int> cv_index;
  std::vector<GPlan> gplan(B.aggs.size());
  for (size_t a = 0; a < B.aggs.size(); ++a) {
    if (cls[a].kind != 1) continue;
    const AggH& ag = B.aggs[a];
    int64_t cells = 1;
    int gsrc = -2;
    for (auto& g : ag.gb) {
      int col, r = owner_of(c, g, &col);
      cells *= c->rels[r].cols[col].dom;
      int q = P->catword.at(g).first;
      gsrc = (gsrc == -2 || gsrc == q) ? q : -3;
    }
    GPlan gp{};
    gp.cache_off = -1;
    gp.res_off = -1;
    gp.cv = -1;
    gp.cv_mode = 0;
    gp.cv_muword = -1;
    gp.cells = cells;
    gp.direct = (gsrc < 0) ? 1 : 0;   // root categories or several keys: per-row table
    if (gp.direct && cls[a].mono.empty() && ag.gb.size() == 2 && P->unique_all) {
      // a COUNT table over two categories of different keys (or a key and the
      // root): read it off a view keyed by one of the keys that keeps the other
      // category; the resident key if it is one of them (its counters live in
      // shared memory), else the key with fewer values (smaller views, and
      // the grouped sums of the other key's means by this key's categories
      // can read them)
      const int g0 = P->catword.at(ag.gb[0]).first, g1 = P->catword.at(ag.gb[1]).first;
      int x = -1;
      if (g0 >= 0 && (g0 == res_grp || g1 < 0)) x = 0;
      else if (g1 >= 0 && (g1 == res_grp || g0 < 0)) x = 1;
      else if (g0 >= 0 && g1 >= 0)
        x = P->groups[RR.groups[g1]].K < P->groups[RR.groups[g0]].K ? 1 : 0;
      // a view holds K x dom(b) 32-bit counters: keep it within kCvMaxCells
      // (else try the other key, else the per-row table)
      auto cells_of = [&](int xx) -> int64_t {
        const int gx = xx == 0 ? g0 : g1;
        if (gx < 0) return INT64_MAX;
        int col, r = owner_of(c, ag.gb[1 - xx], &col);
        return (int64_t)P->groups[RR.groups[gx]].K * c->rels[r].cols[col].dom;
      };
      constexpr int64_t kCvMaxCells = 8 << 20;
      if (x >= 0 && cells_of(x) > kCvMaxCells) x = cells_of(1 - x) <= kCvMaxCells ? 1 - x : -1;
      if (Root.nrows >= ((int64_t)1 << 32)) x = -1;
      if (x >= 0) {
        const int gx = x == 0 ? g0 : g1;
        const std::string& bname = ag.gb[1 - x];
        const int bcat = P->rowcat.at(bname);
        auto key = std::make_pair(gx, bcat);
        auto it = cv_index.find(key);
        if (it == cv_index.end() && (int)cvs.size() < kMaxCatViews) {
          int col, r = owner_of(c, bname, &col);
          cvs.push_back({gx, bcat, P->catword.at(bname).first, c->rels[r].cols[col].dom, 0, -1});
          it = cv_index.emplace(key, (int)cvs.size() - 1).first;
        }
        if (it != cv_index.end()) {
          int col, r = owner_of(c, ag.gb[x], &col);
          gp.cv = it->second;
          gp.cv_aword = P->catword.at(ag.gb[x]).second;
          gp.cv_afirst = x == 0 ? 1 : 0;
          gp.cv_doma = c->rels[r].cols[col].dom;
          gp.direct = 0;
        }
      }
    }
    std::string f = cls[a].mono.empty() ? "" : cls[a].mono[0];
    gp.scale = f.empty() ? 1.0 : std::ldexp(1.0, fixp_exp(W * bound[f]));
    if (!gp.direct && gp.cv < 0) {
      gp.grp = gsrc;
      rv_used[gsrc] = 1;
      if (f.empty()) {
        gp.mode = 0;
      } else if (P->feat_group.at(f) == gsrc) {
        gp.mode = 2;
        GroupH& g = P->groups[RR.groups[gsrc]];
        gp.mu_word = g.n_cnt + (P->zidx.at(f) - rp.grp_zoff[gsrc]);
      } else if (P->lean && P->feat_group.at(f) >= 0) {
        gp.mode = 1;  // a mean of another group: a slot of this view, or a category view (below)
        gp.slot = -1;
        deferred.push_back(a);
      } else {
        gp.mode = 1;
        auto& sl = rv_slots[gsrc];
        int z = P->zidx.at(f);
        auto it = std::find(sl.begin(), sl.end(), z);
        gp.slot = (int)(it - sl.begin());
        if (it == sl.end()) sl.push_back(z);
      }
    }
    gplan[a] = gp;
    ++P->n_grouped;
  }
  // the Gram block of a group's view means is taken at the key level
  // (GroupGram) wherever the group keeps its key counts; a group whose key
  // comes in runs always does (on a sorted root the row-level FP32 sums would
  // add the same products over and over)
  for (int q = 0; q < rp.n_grp; ++q)
    if (P->groups[RR.groups[q]].n_mu > 0 && has_runs[q]) rv_used[q] = 1;

  // ---- key-level form: where every Gram block with a view mean comes from.
  // (x, m_g): the root feature x as a slot of g's reverse view; (m_g, m_h):
  // the carrier's view holds the other group's means (the carrier is the
  // group whose view adds fewer reductions: a slot of the resident key's view
  // costs nothing per row, one of a view summed in runs one reduction per
  // run, one of a view reduced row by row 8 of the 32 bytes of a sector per
  // row; ties: the resident key, the key with fewer changes, fewer keys);
  // (1, x): the root feature's sum from the view with the fewest keys; (m_g,
  // m_g) and (1, m_g): GroupGram over g's key counts; (x, x): the row Gram.
  struct LeanPair {
    int q, z_slot, mean_i, za, zb;
  };
  std::vector<LeanPair> lean_pairs;
  std::vector<int> rv_mode(rp.n_grp, kRvRuns);
  if (P->lean) {
    auto n_mu_of = [&](int q) { return P->groups[RR.groups[q]].n_mu; };
    auto zgroup = [&](int z) -> int {
      for (int q = 0; q < rp.n_grp; ++q)
        if (z >= rp.grp_zoff[q] && z < rp.grp_zoff[q] + n_mu_of(q)) return q;
      return -1;  // the constant or a root feature
    };
    auto rank = [&](int q) {
      return std::make_tuple(q == res_grp ? 0 : 1, changes[q], P->groups[RR.groups[q]].K, q);
    };
    auto slot_cost = [&](int q) -> double {
      if (q == res_grp) return 0.0;
      return has_runs[q] ? (double)(changes[q] + 1) : (double)Root.nrows / 4.0;
    };
    // per pair of groups: the means of each that some (m_g, m_h) product needs
    std::map<std::pair<int, int>, std::pair<std::set<int>, std::set<int>>> cross_means;
    // means a view gets anyway: grouped sums of another group's mean by one
    // of its categories that no category view answers (resolved below)
    std::vector<std::set<int>> pre_slot(rp.n_grp);
    for (size_t a : deferred) {
      const std::string& f = cls[a].mono[0];
      const int h = P->feat_group.at(f);
      if (B.aggs[a].gb.size() == 1 && cv_index.count({h, P->rowcat.at(B.aggs[a].gb[0])})) continue;
      pre_slot[gplan[a].grp].insert(P->zidx.at(f));
    }
    auto carrier = [&](int g, int h) {
      const auto key = std::make_pair(std::min(g, h), std::max(g, h));
      auto it = cross_means.find(key);
      if (it != cross_means.end()) {
        // carrying in the lower group adds the higher group's means to its
        // view, those it does not hold anyway
        auto added = [&](int q, const std::set<int>& zs) {
          double n = 0;
          for (int z : zs) n += pre_slot[q].count(z) ? 0.0 : 1.0;
          return n;
        };
        const double c_lo = slot_cost(key.first) * added(key.first, it->second.second);
        const double c_hi = slot_cost(key.second) * added(key.second, it->second.first);
        if (c_lo != c_hi) return c_lo < c_hi ? key.first : key.second;
      }
      return rank(g) < rank(h) ? g : h;
    };
    auto add_slot = [&](int q, int z) {
      auto& sl = rv_slots[q];
      auto it = std::find(sl.begin(), sl.end(), z);
      if (it == sl.end()) sl.push_back(z);
    };
    std::set<std::pair<int, int>> need;
    for (size_t a = 0; a < B.aggs.size(); ++a) {
      if (cls[a].kind != 0 || cls[a].mono.empty()) continue;
      int i = cls[a].mono.size() == 2 ? P->zidx.at(cls[a].mono[0]) : 0;
      int j = P->zidx.at(cls[a].mono.back());
      if (i > j) std::swap(i, j);
      need.insert({i, j});
    }
    for (auto& ij : need) {
      const int gi = zgroup(ij.first), gj = zgroup(ij.second);
      if (ij.first == 0 || gi < 0 || gj < 0 || gi == gj) continue;
      auto& e = cross_means[{std::min(gi, gj), std::max(gi, gj)}];
      (gi < gj ? e.first : e.second).insert(ij.first);
      (gi < gj ? e.second : e.first).insert(ij.second);
    }
    int sum_q = 0;
    for (int q = 1; q < rp.n_grp; ++q)
      if (P->groups[RR.groups[q]].K < P->groups[RR.groups[sum_q]].K) sum_q = q;
    for (auto& ij : need) {
      const int i = ij.first, j = ij.second, gi = zgroup(i), gj = zgroup(j);
      if (i == 0) {
        if (gj < 0) lean_pairs.push_back({sum_q, j, -1, 0, j});
        continue;  // (1, m_g): GroupGram
      }
      if (gi < 0 && gj < 0) continue;  // row Gram
      if (gi < 0) {
        lean_pairs.push_back({gj, i, j - rp.grp_zoff[gj], i, j});
        continue;
      }
      if (gi == gj) continue;  // GroupGram
      const int cq = carrier(gi, gj);
      const int carried = cq == gi ? j : i, own = cq == gi ? i : j;
      lean_pairs.push_back({cq, carried, own - rp.grp_zoff[cq], i, j});
    }
    // root features first in every view, then carried means
    for (auto& lp : lean_pairs)
      if (zgroup(lp.z_slot) < 0) add_slot(lp.q, lp.z_slot);
    for (auto& lp : lean_pairs)
      if (zgroup(lp.z_slot) >= 0) add_slot(lp.q, lp.z_slot);
    // grouped sums of another group h's mean, grouped by a category of g: a
    // slot g's view already holds, else a category view keyed by h keeping
    // the category (count x mean over h's keys), else a new slot
    for (size_t a : deferred) {
      GPlan& gp = gplan[a];
      const std::string& f = cls[a].mono[0];
      const int h = P->feat_group.at(f), z = P->zidx.at(f);
      auto& sl = rv_slots[gp.grp];
      auto it = std::find(sl.begin(), sl.end(), z);
      if (it != sl.end()) {
        gp.slot = (int)(it - sl.begin());
        continue;
      }
      auto cv = cv_index.find({h, P->rowcat.at(B.aggs[a].gb[0])});
      if (B.aggs[a].gb.size() == 1 && cv != cv_index.end()) {
        gp.cv = cv->second;
        gp.cv_mode = 1;
        gp.cv_muword = P->groups[RR.groups[h]].n_cnt + (z - rp.grp_zoff[h]);
        continue;
      }
      gp.slot = (int)sl.size();
      sl.push_back(z);
    }
    // every group with means keeps its key counts (GroupGram); update modes:
    // the resident key in registers, keys in runs summed per run, the rest one
    // bulk reduction per row while the staging fits (16 words a row)
    int stage_words = 0;
    for (int q = 0; q < rp.n_grp; ++q) {
      if (n_mu_of(q) > 0 || !rv_slots[q].empty()) rv_used[q] = 1;
      if (!rv_used[q]) continue;
      const int stride = (int)(1 + rv_slots[q].size() + 1) & ~1;
      if (q == res_grp) {
        rv_mode[q] = kRvResident;
      } else if (has_runs[q] || stage_words + stride > 16) {
        rv_mode[q] = kRvRuns;
      } else {
        rv_mode[q] = kRvBulk;
        stage_words += stride;
      }
    }
  }
  for (int q = 0; q < rp.n_grp; ++q) {
    if (!rv_used[q]) continue;
    GroupH& g = P->groups[RR.groups[q]];
    if (P->lean) {  // one record per key: [count, slots], an even number of int64 words
      const size_t stride = (1 + rv_slots[q].size() + 1) & ~(size_t)1;
      rv_hist_off[q] = A.take((size_t)g.K * stride * 8);
      rv_R_off[q] = rv_hist_off[q] + 8;
      continue;
    }
    rv_hist_off[q] = A.take((size_t)g.K * 8);
    rv_R_off[q] = A.take((size_t)g.K * rv_slots[q].size() * 8 + 8);
  }
  // key-level form: the exact fixed-point image of every mean a view sums,
  // once per key (k_fix_means), so that the scan does not convert it per row
  std::vector<std::vector<int>> fix_z(rp.n_grp);
  std::vector<size_t> fix_off(rp.n_grp, 0);
  for (int i = 0; i < kMaxZ; ++i) rp.fix_of_z[i] = -1;
  if (P->lean) {
    // (a count times a mean's image would multiply the image's rounding by the
    // count: key-level tasks round the exact product instead)
    std::set<int> slot_z;
    for (int q = 0; q < rp.n_grp; ++q)
      for (int z : rv_slots[q]) slot_z.insert(z);
    for (int q = 0; q < rp.n_grp; ++q) {
      const GroupH& g = P->groups[RR.groups[q]];
      for (int z : slot_z)
        if (z >= rp.grp_zoff[q] && z < rp.grp_zoff[q] + g.n_mu) {
          rp.fix_of_z[z] = (int16_t)fix_z[q].size();
          fix_z[q].push_back(z);
        }
      if (!fix_z[q].empty()) fix_off[q] = A.take((size_t)g.K * ((fix_z[q].size() + 1) & ~(size_t)1) * 8 + 16);
    }
  }
  for (size_t a = 0; a < B.aggs.size(); ++a)
    if (cls[a].kind == 1) gplan[a].out_off = A.take((size_t)gplan[a].cells * 8);
  for (auto& v : cvs) v.off = A.take((size_t)P->groups[RR.groups[v.grp]].K * v.dom * 4 + 16);
  // the keys of each (keying group, row category of a) listed by a, for the
  // COUNT tables read off category views: counters in the zeroed region
  struct CatIdxPlan { int grp, aword, dom; size_t cnt_off, start_off, perm_off; };
  std::vector<CatIdxPlan> cidx;
  std::map<std::pair<int, int>, int> cidx_of;
  for (size_t a = 0; a < B.aggs.size(); ++a) {
    if (cls[a].kind != 1 || gplan[a].cv < 0 || gplan[a].cv_mode != 0) continue;
    const auto key = std::make_pair(cvs[gplan[a].cv].grp, gplan[a].cv_aword);
    if (cidx_of.count(key)) continue;
    cidx_of[key] = (int)cidx.size();
    cidx.push_back({key.first, key.second, gplan[a].cv_doma, A.take((size_t)(gplan[a].cv_doma + 1) * 4), 0, 0});
  }
  // omega accumulators of fanning-out root children
  std::vector<std::pair<int, size_t>> omega;  // child relation, offset
  for (int q = 0; q < rp.n_grp; ++q)
    for (int ch : P->groups[RR.groups[q]].children)
      if (!P->rp[ch].unique) omega.push_back({ch, A.take((size_t)P->groups[RR.groups[q]].K * 8)});
  // tree-node (filtered) batches
  std::vector<int> filt_idx;
  for (size_t a = 0; a < B.aggs.size(); ++a)
    if (cls[a].kind == 2) filt_idx.push_back((int)a);
  if (!filt_idx.empty()) {
    // thresholds and squares are not linear in the attribute: they need the
    // attribute's value in every joined tuple, i.e. a relation reached from the
    // root through unique keys only (its value is then a function of the root row)
    for (int a : filt_idx)
      for (auto& f : B.aggs[a].f) {
        int col, r = owner_of(c, f.attr, &col);
        for (int x = r; x != root; x = P->par[x])
          if (P->mult[x] > 1)
            return fail(c, LMF_ERR_UNSUPPORTED,
                        "aggregate %d: threshold or power factor on %s below the fanning-out key of %s", a,
                        f.attr.c_str(), c->rels[x].name.c_str());
      }
    P->tree = std::make_unique<TreePlan>();
    std::vector<TreeAggIn> in;
    for (int a : filt_idx) {
      TreeAggIn t;
      for (auto& f : B.aggs[a].f) {
        TreeFactorIn x{f.attr, f.kind, f.power, f.thr};
        t.factors.push_back(x);
      }
      in.push_back(t);
    }
    std::string msg;
    lmf_status s = tree_plan(in, P->zidx, P->tree.get(), &msg);
    if (s) return fail(c, s, "%s", msg.c_str());
    P->n_filtered = (int)filt_idx.size();
  }
  if (P->tree) tree_alloc_zeroed(P->tree.get(), Root.nrows, [&](size_t n) { return A.take(n); });
  P->zero_off = zero_begin;
  P->zero_len = A.take(0) - zero_begin;
  for (auto& ci : cidx) {
    ci.start_off = A.take((size_t)(ci.dom + 1) * 4);
    ci.perm_off = A.take((size_t)P->groups[RR.groups[ci.grp]].K * 4 + 4);
  }
  P->cat_idx_off = A.take(sizeof(CatIndex) * (cidx.size() + 1));
  // within-key scatter of fanning-out views: fully rewritten by every run
  for (int r : P->post) {
    RelPlan& cp = P->rp[r];
    if (cp.unique) continue;
    cp.sc_off = A.take((size_t)P->groups[cp.group].K * (cp.d * (cp.d + 1) / 2) * 8 + 8);
  }

  // ---- resident key: the root's foreign key with the fewest changes between
  // adjacent rows, if its runs average at least kResRun rows (a root sorted on
  // its join attributes, Sec. 3.5), carries the COUNT tables that take exactly
  // one category from its group; their counters for the current key live in
  // shared memory (kResBudget of them in all)
  constexpr int kResTableMax = 4096;
  // shared memory left for the per-CTA counters (resident key, hot cells)
  // when two CTAs share an SM; the resident key takes up to three quarters
  int mp0 = 16;
  while (mp0 < m) mp0 += 16;
  const bool tc_planned = P->opts.precision == LMF_PREC_SPLIT_BF16 && gram_tc_supported(m) && P->unique_all;
  size_t base_smem = tc_planned ? gram_tc_smem(ncat, 0, 0) : root_plain_smem(mp0, ncat, 0, 0, P->unique_all);
  int64_t smem_cap = 108 * 1024;
  // reverse-view descriptors (device pointers are valid once the arena is allocated)
  std::vector<int> rv_index(rp.n_grp, -1);
  auto fill_rvs = [&](RootParams& t) -> lmf_status {
    t.n_rv = 0;
    t.res_rv = -1;
    for (int q = 0; q < rp.n_grp; ++q) {
      if (!rv_used[q]) continue;
      if ((int)rv_slots[q].size() > kMaxZ - 1) return fail(c, LMF_ERR_UNSUPPORTED, "too many reverse-view slots");
      RevView& R = t.rv[t.n_rv];
      R.hist = P->at<unsigned long long>(rv_hist_off[q]);
      R.R = P->at<long long>(rv_R_off[q]);
      R.grp = q;
      R.n_slot = (int)rv_slots[q].size();
      for (int s2 = 0; s2 < R.n_slot; ++s2) {
        R.slot_z[s2] = (int16_t)rv_slots[q][s2];
        std::string fname;
        for (auto& kv : P->zidx)
          if (kv.second == rv_slots[q][s2]) fname = kv.first;
        R.slot_scale[s2] = (float)std::ldexp(1.0, fixp_exp(W * bound[fname]));
      }
      if (P->lean) {
        R.stride = (1 + R.n_slot + 1) & ~1;
        R.hstride = R.rstride = R.stride;
        R.mode = rv_mode[q];
        if (R.mode == kRvResident) t.res_rv = t.n_rv;
      } else {
        R.stride = R.n_slot;
        R.hstride = 1;
        R.rstride = R.n_slot;
        R.mode = kRvRuns;
      }
      rv_index[q] = t.n_rv++;
    }
    return LMF_OK;
  };
  int n_direct_planned = 0;
  bool direct_z = false;
  for (size_t a = 0; a < B.aggs.size(); ++a)
    if (cls[a].kind == 1 && gplan[a].direct) {
      ++n_direct_planned;
      direct_z = direct_z || !cls[a].mono.empty();
    }
  if (P->lean) {  // three CTAs per SM: what the z tile and the bulk staging leave of 74 KB
    rp.lean = 1;
    rp.gram_off = 1;
    rp.gram_n = rp.n_x;
    RootParams t = rp;
    t.cache_cells = t.res_cells = 0;
    t.n_direct = n_direct_planned;
    lmf_status st = fill_rvs(t);
    if (st) return st;
    base_smem = lean_shape(t, direct_z).cache_off;
    smem_cap = 74 * 1024;
  }
  const int64_t cell_budget = std::max<int64_t>(0, (smem_cap - (int64_t)base_smem) / 4);
  const int64_t kResBudget = cell_budget * 3 / 4;
  int res_cells = 0;
  int cv_res_cells = 0;
  if (res_grp >= 0) {
    // category views keyed by the resident key: one counter per value of b
    for (auto& v : cvs)
      if (v.grp == res_grp && cv_res_cells + v.dom <= kResBudget) {
        v.res_off = cv_res_cells;
        cv_res_cells += v.dom;
      }
    res_cells = cv_res_cells;
    for (size_t a = 0; a < B.aggs.size(); ++a) {
      if (cls[a].kind != 1 || !gplan[a].direct || !cls[a].mono.empty()) continue;
      const AggH& ag = B.aggs[a];
      int q_res = -1, n_in = 0;
      int64_t n = 1;
      for (size_t q = 0; q < ag.gb.size(); ++q) {
        if (P->catword.at(ag.gb[q]).first == res_grp) {
          q_res = (int)q;
          ++n_in;
        } else {
          int col, r = owner_of(c, ag.gb[q], &col);
          n *= c->rels[r].cols[col].dom;
        }
      }
      if (n_in != 1 || n > kResTableMax || res_cells + n > kResBudget) continue;
      gplan[a].res_off = 0;
      gplan[a].res_q = q_res;
      gplan[a].res_word = P->catword.at(ag.gb[q_res]).second;
      gplan[a].res_n = (int)n;
      gplan[a].res_lanes = 0;
      res_cells += (int)n;
    }
    // tables of at most 32 cells, smallest first, get one counter per lane
    // while the budget lasts (their few hot cells would serialise a warp's
    // shared-memory atomics)
    std::vector<size_t> small;
    for (size_t a = 0; a < B.aggs.size(); ++a)
      if (cls[a].kind == 1 && gplan[a].res_off >= 0 && gplan[a].res_n <= 32) small.push_back(a);
    std::stable_sort(small.begin(), small.end(), [&](size_t x, size_t y) { return gplan[x].res_n < gplan[y].res_n; });
    for (size_t a : small) {
      if (res_cells + 31 * gplan[a].res_n > kResBudget) break;
      gplan[a].res_lanes = 1;
      res_cells += 31 * gplan[a].res_n;
    }
    res_cells = cv_res_cells;
    for (size_t a = 0; a < B.aggs.size(); ++a) {
      if (cls[a].kind != 1 || gplan[a].res_off < 0) continue;
      gplan[a].res_off = res_cells;
      res_cells += gplan[a].res_n * (gplan[a].res_lanes ? 32 : 1);
    }
    if (res_cells == 0 && !P->lean) res_grp = -1;  // (sorted_q keeps it for the tree pass)
  }

  // ---- hot-cell cache: per CTA, the hottest (value, value) cells of every
  // pair-count table are 32-bit counters in shared memory; Zipf-skewed
  // categories otherwise serialise L2 atomics on a few addresses (a table's
  // hottest cell takes 3-19% of all rows in the snowflake workload).  The hot
  // values are the most frequent ones of each category column, counted here.
  constexpr int kHotVals = 8, kCacheBudget = 24 * 1024 / 4;
  std::map<int, std::vector<int32_t>> hot_vals;  // row category -> its hot values
  int cache_cells = 0;
  {
    auto top_of = [&](const int32_t* col, int64_t n, int K, int h, std::vector<int32_t>* out) -> lmf_status {
      if (n <= 0 || K <= 0) return LMF_OK;
      DevScratch d_buf;
      CUDA_TRY(c, cudaMalloc(&d_buf.p, sizeof(unsigned int) * K));
      unsigned int* d = d_buf.as<unsigned int>();
      CUDA_TRY(c, cudaMemsetAsync(d, 0, sizeof(unsigned int) * K, c->stream));
      CUDA_TRY(c, launch_key_stats(col, n, d, K, nullptr, c->stream));
      std::vector<unsigned int> cnt(K);
      CUDA_TRY(c, cudaMemcpyAsync(cnt.data(), d, sizeof(unsigned int) * K, cudaMemcpyDeviceToHost, c->stream));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      std::vector<int32_t> idx(K);
      for (int i = 0; i < K; ++i) idx[i] = i;
      const int take = std::min(h, K);
      std::partial_sort(idx.begin(), idx.begin() + take, idx.end(),
                        [&](int a, int b) { return cnt[a] > cnt[b] || (cnt[a] == cnt[b] && a < b); });
      for (int i = 0; i < take; ++i)
        if (cnt[idx[i]] > 0) out->push_back(idx[i]);
      return LMF_OK;
    };
    // pair COUNT tables with w in {0, 1}: a CTA counts fewer than 2^32 rows
    for (size_t a = 0; a < B.aggs.size(); ++a) {
      if (cls[a].kind != 1 || !gplan[a].direct || B.aggs[a].gb.size() != 2) continue;
      if (!cls[a].mono.empty() || !P->unique_all || gplan[a].res_off >= 0) continue;
      if (cache_cells + kHotVals * kHotVals > kCacheBudget || res_cells + cache_cells + kHotVals * kHotVals > cell_budget)
        break;
      for (auto& gname : B.aggs[a].gb) {
        const int rc = P->rowcat.at(gname);
        if (hot_vals.count(rc)) continue;
        int col, r = owner_of(c, gname, &col);
        const ColumnH& cc = c->rels[r].cols[col];
        lmf_status st = top_of(static_cast<const int32_t*>(cc.dptr()), c->rels[r].nrows, cc.dom, kHotVals, &hot_vals[rc]);
        if (st) return st;
      }
      gplan[a].cache_off = cache_cells;
      cache_cells += kHotVals * kHotVals;
    }
  }
  size_t hot_lut_bytes = 0;
  std::map<int, size_t> hot_lut_at;  // row category -> offset in the lut
  for (auto& kv : hot_vals) {
    int col, r = owner_of(c, [&] {
      for (auto& n : P->rowcat)
        if (n.second == kv.first) return n.first;
      return std::string();
    }(), &col);
    hot_lut_at[kv.first] = hot_lut_bytes;
    hot_lut_bytes += (size_t)c->rels[r].cols[col].dom;
  }
  const size_t hot_lut_off = A.take(hot_lut_bytes + 1);
  const size_t cache_dst_off = A.take((size_t)cache_cells * 8 + 8);

  // root scan shape
  int mp = 16;
  while (mp < m) mp += 16;
  P->mp = mp;
  const int T = root_plain_tile_rows();
  P->n_tiles = (Root.nrows + T - 1) / T;
  P->smem = root_plain_smem(mp, ncat, cache_cells, res_cells, P->unique_all);
  int cps = P->opts.ctas_per_sm > 0 ? P->opts.ctas_per_sm : (P->smem <= 110 * 1024 ? 2 : 1);
  P->grid = (int)std::max<int64_t>(1, std::min<int64_t>(P->n_tiles, (int64_t)c->num_sms * cps));
  // the compiled scan is built for three CTAs per SM (its launch bounds cap the
  // registers) when its shared memory allows a third one
  const bool jit3 = P->opts.ctas_per_sm <= 0 && P->smem <= 74 * 1024;
  const int grid_jit =
      jit3 ? (int)std::max<int64_t>(1, std::min<int64_t>(P->n_tiles, (int64_t)c->num_sms * 3)) : P->grid;
  CUDA_TRY(c, root_plain_prepare(mp, P->smem));
  // the split-bf16 tensor-core Gram needs w in {0, 1} (unique child keys) and
  // z within one 32-feature block; other plans keep the plain FP32 Gram
  bool use_tc = P->opts.precision == LMF_PREC_SPLIT_BF16 && gram_tc_supported(m) && P->unique_all;
  if (P->opts.precision == LMF_PREC_SPLIT_BF16 && !use_tc) P->opts.precision = LMF_PREC_PLAIN_FP32;
  if (use_tc) {
    P->tc = std::make_unique<GramTcPlan>();
    gram_tc_shape(m, Root.nrows, c->num_sms, P->opts.tile_rows, P->tc.get());
    CUDA_TRY(c, gram_tc_configure(P->tc.get(), ncat, P->opts.ctas_per_sm, cache_cells, res_cells));
    P->grid = P->tc->grid;
  }
  if (P->lean) {
    RootParams t = rp;
    t.cache_cells = cache_cells;
    t.res_cells = res_cells;
    t.n_direct = n_direct_planned;
    lmf_status st = fill_rvs(t);
    if (st) return st;
    const LeanShape L = lean_shape(t, direct_z);
    P->lean_mpx = L.mpx;
    P->smem = L.smem;
    // three CTAs per SM (80 registers a thread) when the shared memory allows,
    // else two; ctas_per_sm caps it
    const int fit = L.smem <= 74 * 1024 ? 3 : (L.smem <= 110 * 1024 ? 2 : 1);
    const int lcps = P->opts.ctas_per_sm > 0 ? std::min(P->opts.ctas_per_sm, fit) : fit;
    P->grid = (int)std::max<int64_t>(1, std::min<int64_t>(P->n_tiles, (int64_t)c->num_sms * lcps));
  }
  const int grid_max = std::max(P->grid, grid_jit);
  P->part_off = A.take((size_t)grid_max * std::max(mp, P->lean_mpx) * std::max(mp, P->lean_mpx) * 8);
  P->cntp_off = A.take((size_t)grid_max * 8);
  P->G_off = A.take((size_t)m * m * 8);
  P->count_off = A.take(8);
  if (use_tc) gram_tc_alloc(P->tc.get(), [&](size_t n) { return A.take(n); });
  if (P->tree) tree_alloc(P->tree.get(), Root.nrows, [&](size_t n) { return A.take(n); });

  // results
  P->agg_dtype.resize(B.aggs.size());
  P->agg_off.resize(B.aggs.size());
  P->agg_n.resize(B.aggs.size());
  for (size_t a = 0; a < B.aggs.size(); ++a) {
    bool is_count = cls[a].mono.empty();
    int64_t cells = cls[a].kind == 1 ? gplan[a].cells : 1;
    P->agg_dtype[a] = is_count ? LMF_I64 : LMF_F64;
    P->agg_n[a] = cells;
    if (is_count) {
      P->agg_off[a] = P->n_i64;
      P->n_i64 += cells;
    } else {
      P->agg_off[a] = P->n_f64;
      P->n_f64 += cells;
    }
  }
  P->res_i64_off = A.take((size_t)std::max<int64_t>(1, P->n_i64) * 8);
  P->res_f64_off = A.take((size_t)std::max<int64_t>(1, P->n_f64) * 8);
  // device tables
  size_t n_rvt_est = B.aggs.size() + 1;
  P->rvtask_off = A.take(sizeof(RvTask) * n_rvt_est);
  P->cvtask_off = A.take(sizeof(CatViewTask) * n_rvt_est);
  {
    size_t npart = 0;
    for (int q = 0; q < rp.n_grp; ++q) {
      const int n = P->groups[RR.groups[q]].n_mu;
      if (n > 0) npart += (size_t)((n + 1) * (n + 2) / 2 - 1);
    }
    P->ggram_off = A.take(sizeof(GroupGram) * (rp.n_grp + 1));
    P->ggram_part_off = A.take(sizeof(double) * (npart * Plan::kGgChunks + 1));
    P->cgram_off = A.take(sizeof(CrossGram) * (rp.n_grp + 1));
    P->cpair_off = A.take(sizeof(CrossPair) * (lean_pairs.size() + 1));
    P->cgram_part_off = A.take(sizeof(double) * (lean_pairs.size() * Plan::kGgChunks + 1));
  }
  P->direct_off = A.take(sizeof(DirectAgg) * n_rvt_est);
  P->corr_off = A.take(sizeof(CorrTask) * (omega.size() + 1));
  P->maps_off = A.take(sizeof(OutMap) * (B.aggs.size() + 1));

  // ---- allocate
  A.size = A.used + 256;
  {
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, A.size);
    if (e != cudaSuccess) return fail(c, LMF_ERR_OOM, "plan arena of %zu bytes", A.size);
    A.base = static_cast<char*>(base);
  }

  // ---- fill device descriptors
  auto gdesc = [&](int gi) {
    GroupH& g = P->groups[gi];
    const RelationH& O = c->rels[g.owner];
    GroupDesc d;
    d.fk = static_cast<const int32_t*>(O.cols[O.find(g.fk)].dptr());
    d.rec = P->at<uint32_t>(g.rec_off);
    d.K = g.K;
    d.stride = g.stride;
    d.n_cnt = g.n_cnt;
    d.n_mu = g.n_mu;
    d.n_cat = g.n_cat;
    d.fix = nullptr;
    d.fix_stride = 0;
    return d;
  };
  for (int q = 0; q < rp.n_grp; ++q) {
    rp.grp[q] = gdesc(RR.groups[q]);
    if (fix_z[q].empty()) continue;
    rp.grp[q].fix = P->at<long long>(fix_off[q]);
    rp.grp[q].fix_stride = (int)((fix_z[q].size() + 1) & ~(size_t)1);
    FixMeans f{};
    f.g = rp.grp[q];
    f.n = (int)fix_z[q].size();
    for (int j = 0; j < f.n; ++j) {
      const int z = fix_z[q][j];
      f.mu_word[j] = (int16_t)(rp.grp[q].n_cnt + (z - rp.grp_zoff[q]));
      std::string fname;
      for (auto& kv : P->zidx)
        if (kv.second == z) fname = kv.first;
      f.scale[j] = (float)std::ldexp(1.0, fixp_exp(W * bound[fname]));
    }
    P->fixm.push_back(f);
  }
  rp.gram_part = P->at<double>(P->part_off);
  rp.cnt_part = P->at<long long>(P->cntp_off);
  rp.status = P->at<uint32_t>(P->status_off);
  {
    lmf_status st = fill_rvs(rp);
    if (st) return st;
  }
  {
    int part = 0;
    for (int q = 0; q < rp.n_grp; ++q) {
      const GroupDesc& G = rp.grp[q];
      if (G.n_mu <= 0 || rv_index[q] < 0) continue;
      GroupGram g{};
      g.grp = q;
      g.rv = rv_index[q];
      g.n = G.n_mu;
      g.zoff = rp.grp_zoff[q];
      g.mu_word = G.n_cnt;
      g.npair = (g.n + 1) * (g.n + 2) / 2 - 1;
      g.part_off = part;
      part += g.npair;
      P->ggram.push_back(g);
    }
  }
  if (P->lean) {  // key-level Gram entries, one CrossGram per view that holds slots for them
    int part = 0;
    for (int q = 0; q < rp.n_grp; ++q) {
      CrossGram g{};
      g.rv = rv_index[q];
      g.grp = q;
      g.mu_word = P->groups[RR.groups[q]].n_cnt;
      g.pair_off = (int)P->cpairs.size();
      g.part_off = part;
      for (auto& lp : lean_pairs) {
        if (lp.q != q) continue;
        const auto& sl = rv_slots[q];
        const int slot = (int)(std::find(sl.begin(), sl.end(), lp.z_slot) - sl.begin());
        P->cpairs.push_back(CrossPair{(int16_t)slot, (int16_t)lp.mean_i, (int16_t)lp.za, (int16_t)lp.zb});
      }
      g.npair = (int)P->cpairs.size() - g.pair_off;
      if (g.npair == 0) continue;
      part += g.npair;
      P->cgram.push_back(g);
    }
  }
  // hot-cell tables: category value -> hot index, and the global cell every
  // cache cell flushes to
  std::vector<long long*> cache_dst(cache_cells, P->at<long long>(P->count_off));
  {
    std::vector<int8_t> lut(hot_lut_bytes + 1, -1);
    for (int i = 0; i < kMaxCat; ++i) rp.hot_lut_off[i] = -1;
    for (auto& kv : hot_vals) {
      const size_t at = hot_lut_at[kv.first];
      for (size_t h = 0; h < kv.second.size(); ++h) lut[at + kv.second[h]] = (int8_t)h;
      rp.hot_lut_off[kv.first] = (int32_t)at;
    }
    CUDA_TRY(c, cudaMemcpy(P->arena.base + hot_lut_off, lut.data(), lut.size(), cudaMemcpyHostToDevice));
  }
  rp.hot_lut = P->at<int8_t>(hot_lut_off);
  rp.hot_h = kHotVals;
  rp.cache_cells = cache_cells;
  rp.res_grp = res_grp < 0 ? 0 : res_grp;
  rp.res_cells = res_cells;
  rp.unit_w = P->unique_all ? 1 : 0;
  {
    int n_runs = 0;
    for (int q = 0; q < rp.n_grp; ++q) n_runs += has_runs[q];
    rp.fold = n_runs >= 2 ? 8 : 0;
  }
  rp.cache_dst = P->at<long long*>(cache_dst_off);
  std::vector<RvTask> tasks;
  std::vector<DirectAgg> direct;
  for (size_t a = 0; a < B.aggs.size(); ++a) {
    if (cls[a].kind != 1) continue;
    const GPlan& gp = gplan[a];
    const AggH& ag = B.aggs[a];
    std::string f = cls[a].mono.empty() ? "" : cls[a].mono[0];
    if (gp.cv >= 0) {
      CatViewTask t{};
      t.view = gp.cv;
      t.a_word = gp.cv_aword;
      t.dom_a = gp.cv_doma;
      t.a_first = gp.cv_afirst;
      t.out = P->at<long long>(gp.out_off);
      t.mode = gp.cv_mode;
      t.mu_word = gp.cv_muword;
      t.scale = (float)gp.scale;
      t.fix_idx = -1;  // count x mean: one rounding of the exact product per cell
      t.cat_idx = gp.cv_mode == 0 ? cidx_of.at({cvs[gp.cv].grp, gp.cv_aword}) : -1;
      P->cv_tasks.push_back(t);
      const CvPlan& v = cvs[gp.cv];
      P->cv_max_cells = std::max<int64_t>(P->cv_max_cells, (int64_t)P->groups[RR.groups[v.grp]].K * v.dom);
    } else if (gp.direct) {
      DirectAgg d{};
      d.n_gb = (int)ag.gb.size();
      d.runs = 1;
      for (int q = 0; q < d.n_gb; ++q) {
        int col, r = owner_of(c, ag.gb[q], &col);
        d.cat[q] = P->rowcat.at(ag.gb[q]);
        d.dom[q] = c->rels[r].cols[col].dom;
        const int g = P->catword.at(ag.gb[q]).first;  // -1: a root category
        if (g < 0 || !has_runs[g]) d.runs = 0;
      }
      d.z = f.empty() ? -1 : P->zidx.at(f);
      d.scale = (float)gp.scale;
      d.out = P->at<long long>(gp.out_off);
      d.cache_off = gp.cache_off;
      d.res_off = gp.res_off;
      d.res_q = gp.res_q;
      d.res_word = gp.res_word;
      d.res_n = gp.res_n;
      d.res_lanes = gp.res_lanes;
      if (gp.cache_off >= 0) {
        const auto& va = hot_vals.at(d.cat[0]);
        const auto& vb = hot_vals.at(d.cat[1]);
        for (size_t ha = 0; ha < va.size(); ++ha)
          for (size_t hb = 0; hb < vb.size(); ++hb)
            cache_dst[gp.cache_off + ha * kHotVals + hb] = d.out + (int64_t)va[ha] * d.dom[1] + vb[hb];
      }
      direct.push_back(d);
    } else {
      RvTask t{};
      t.rv = rv_index[gp.grp];
      t.n_gb = (int)ag.gb.size();
      for (int q = 0; q < t.n_gb; ++q) {
        int col, r = owner_of(c, ag.gb[q], &col);
        t.cat_word[q] = P->catword.at(ag.gb[q]).second;
        t.dom[q] = c->rels[r].cols[col].dom;
      }
      t.mode = gp.mode;
      t.slot = gp.slot;
      t.mu_word = gp.mu_word;
      t.scale = (float)gp.scale;
      t.out = P->at<long long>(gp.out_off);
      t.fix_idx = -1;  // hist x mean: one rounding of the exact product per key (FP64)
      t.soff = -1;
      t.cells = gp.cells;
      tasks.push_back(t);
      P->max_group_K = std::max(P->max_group_K, P->groups[RR.groups[gp.grp]].K);
    }
  }
  if (cache_cells > 0)
    CUDA_TRY(c, cudaMemcpy(P->arena.base + cache_dst_off, cache_dst.data(), sizeof(long long*) * cache_cells,
                           cudaMemcpyHostToDevice));
  // tasks grouped by their view: one pass over a view serves all of them
  auto group_by_view = [](auto& v, int n_views, auto view_of, TaskRanges* rg) {
    std::stable_sort(v.begin(), v.end(), [&](const auto& a, const auto& b) { return view_of(a) < view_of(b); });
    rg->n_views = n_views;
    int t = 0;
    for (int i = 0; i <= n_views; ++i) {
      while (t < (int)v.size() && view_of(v[t]) < i) ++t;
      rg->begin[i] = t;
    }
  };
  group_by_view(tasks, rp.n_rv, [](const RvTask& t) { return t.rv; }, &P->rv_ranges);
  std::stable_sort(P->cv_tasks.begin(), P->cv_tasks.end(),
                   [](const CatViewTask& a, const CatViewTask& b) { return a.mode < b.mode; });
  group_by_view(P->cv_tasks, (int)cvs.size(), [](const CatViewTask& t) { return t.view; }, &P->cv_ranges);
  // work items of the key-level tasks: reverse-view tasks in groups that share
  // one shared-memory table per block (kRvTabCells int64), over key chunks;
  // COUNT and SUM(m) by b tables read off category views (below)
  constexpr int kRvTabCells = 5120;
  {
    for (int r = 0; r < rp.n_rv; ++r) {
      const int t0 = P->rv_ranges.begin[r], t1 = P->rv_ranges.begin[r + 1];
      const int64_t K = rp.grp[rp.rv[r].grp].K;
      int g0 = t0, cells = 0;
      auto close = [&](int g1) {
        if (g1 <= g0) return;
        const int64_t ch = 512;  // keys per block; the block's table is added to the outputs once
        for (int64_t k0 = 0; k0 < K; k0 += ch) P->rv_items.push_back(RvItem{r, g0, g1, cells, k0, std::min(K, k0 + ch)});
        P->rv_item_cells = std::max(P->rv_item_cells, cells);
      };
      for (int t = t0; t < t1; ++t) {
        if (tasks[t].cells > kRvTabCells) {  // wide: straight to its output (k_rv_tasks)
          close(t);
          g0 = t + 1;
          cells = 0;
          P->rv_wide = true;
          continue;
        }
        if (cells + tasks[t].cells > kRvTabCells || t - g0 >= 64) {
          close(t);
          g0 = t;
          cells = 0;
        }
        tasks[t].soff = cells;
        cells += (int)tasks[t].cells;
      }
      close(t1);
    }
    // COUNT tables: per task, chunks of 256 positions of its category index
    // (keys grouped by a) x 256 view cells b
    for (size_t t = 0; t < P->cv_tasks.size(); ++t) {
      const CatViewTask& T = P->cv_tasks[t];
      if (T.mode != 0) continue;
      const int db = cvs[T.view].dom;
      const int64_t K = rp.grp[cvs[T.view].grp].K;
      for (int64_t p0 = 0; p0 < K; p0 += 256)
        for (int b0 = 0; b0 < db; b0 += 256)
          P->cv_pair_items.push_back(CvPairItem{(int)t, b0, 0, 0, p0, std::min(K, p0 + 256)});
    }
    // SUM(m) by b tables: per view, its mean tasks in groups of kCvMeanTasks,
    // chunks of 64 keys x 256 view cells b
    for (int v = 0; v < (int)cvs.size(); ++v) {
      int m0 = -1, m1 = -1;
      for (int t = P->cv_ranges.begin[v]; t < P->cv_ranges.begin[v + 1]; ++t)
        if (P->cv_tasks[t].mode == 1) {
          if (m0 < 0) m0 = t;
          m1 = t + 1;
        }
      if (m0 < 0) continue;
      const int64_t K = rp.grp[cvs[v].grp].K;
      for (int t = m0; t < m1; t += kCvMeanTasks)
        for (int64_t k0 = 0; k0 < K; k0 += 64)
          for (int b0 = 0; b0 < cvs[v].dom; b0 += 256)
            P->cv_mean_items.push_back(CvMeanItem{v, t, std::min(m1, t + kCvMeanTasks), b0, k0, std::min(K, k0 + 64)});
    }
  }
  P->rv_tasks = tasks;
  P->direct = direct;
  rp.n_cv = (int)cvs.size();
  for (size_t i = 0; i < cvs.size(); ++i) {
    CatView& C = rp.cv[i];
    C.grp = cvs[i].grp;
    C.bcat = cvs[i].bcat;
    C.dom = cvs[i].dom;
    C.res_off = res_grp >= 0 ? cvs[i].res_off : -1;
    C.runs = has_runs[cvs[i].grp] && cvs[i].bgrp >= 0 && has_runs[cvs[i].bgrp];
    C.V = P->at<uint32_t>(cvs[i].off);
  }
  rp.n_direct = (int)direct.size();
  rp.direct = P->at<DirectAgg>(P->direct_off);
  for (int d = 0; d < rp.n_direct && d < kDirInline; ++d) rp.dir[d] = direct[d];
  rp.n_om = 0;
  std::vector<CorrTask> corr;
  for (auto& o : omega) {
    int ch = o.first;
    RelPlan& cp = P->rp[ch];
    int q = 0;
    for (; q < rp.n_grp; ++q)
      if (RR.groups[q] == cp.group) break;
    OmegaAcc& O = rp.om[rp.n_om++];
    O.grp = q;
    O.cnt_word = cp.slot;
    O.omega = P->at<unsigned long long>(o.second);
    CorrTask t;
    t.omega = O.omega;
    t.sc = P->at<double>(cp.sc_off);
    t.K = P->groups[cp.group].K;
    t.d = cp.d;
    t.zoff = rp.grp_zoff[q] + (P->groups[cp.group].child_mu_off[cp.slot] - P->groups[cp.group].n_cnt);
    corr.push_back(t);
  }
  // out maps
  std::vector<OutMap> maps;
  for (size_t a = 0; a < B.aggs.size(); ++a) {
    OutMap o{};
    o.dst = P->agg_off[a];
    o.n = P->agg_n[a];
    if (cls[a].kind == 0) {
      const auto& mo = cls[a].mono;
      if (mo.empty()) {
        o.kind = 0;
      } else {
        o.kind = 1;
        o.i = mo.size() == 2 ? P->zidx.at(mo[0]) : 0;
        o.j = P->zidx.at(mo.back());
        if (o.i > o.j) std::swap(o.i, o.j);
        ++P->n_gram;
      }
    } else if (cls[a].kind == 1) {
      o.kind = cls[a].mono.empty() ? 2 : 3;
      o.src = P->at<long long>(gplan[a].out_off);
      o.inv_scale = 1.0 / gplan[a].scale;
    } else {
      continue;  // filtered aggregates are placed by the tree kernels
    }
    maps.push_back(o);
  }
  P->maps = maps;
  for (size_t i = 0; i < maps.size(); ++i)
    for (int64_t c0 = 0; c0 < std::max<int64_t>(1, maps[i].n); c0 += 4096)
      P->out_items.push_back(OutItem{(int)i, 0, c0, std::min<int64_t>(std::max<int64_t>(1, maps[i].n), c0 + 4096)});
  {  // one device buffer for the work-item lists
    auto bytes = [](size_t n, size_t sz) { return (n * sz + 255) & ~(size_t)255; };
    P->aux_rv = 0;
    P->aux_cvp = P->aux_rv + bytes(P->rv_items.size(), sizeof(RvItem));
    P->aux_cvm = P->aux_cvp + bytes(P->cv_pair_items.size(), sizeof(CvPairItem));
    P->aux_out = P->aux_cvm + bytes(P->cv_mean_items.size(), sizeof(CvMeanItem));
    const size_t total = P->aux_out + bytes(P->out_items.size(), sizeof(OutItem)) + 256;
    cudaError_t e = cudaMalloc(&P->aux, total);
    if (e != cudaSuccess) return fail(c, LMF_ERR_OOM, "plan work lists of %zu bytes", total);
    char* a = static_cast<char*>(P->aux);
    CUDA_TRY(c, cudaMemcpy(a + P->aux_rv, P->rv_items.data(), sizeof(RvItem) * P->rv_items.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(a + P->aux_cvp, P->cv_pair_items.data(), sizeof(CvPairItem) * P->cv_pair_items.size(),
                           cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(a + P->aux_cvm, P->cv_mean_items.data(), sizeof(CvMeanItem) * P->cv_mean_items.size(),
                           cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(a + P->aux_out, P->out_items.data(), sizeof(OutItem) * P->out_items.size(),
                           cudaMemcpyHostToDevice));
  }
  P->corr = corr;
  CUDA_TRY(c, cudaMemcpy(P->arena.base + P->rvtask_off, tasks.data(), sizeof(RvTask) * tasks.size(), cudaMemcpyHostToDevice));
  for (auto& ci : cidx) {
    CatIndex I{};
    I.grp = ci.grp;
    I.a_word = ci.aword;
    I.dom = ci.dom;
    I.cnt = P->at<uint32_t>(ci.cnt_off);
    I.start = P->at<uint32_t>(ci.start_off);
    I.perm = P->at<int32_t>(ci.perm_off);
    P->cat_idx.push_back(I);
    P->cat_idx_maxK = std::max<int64_t>(P->cat_idx_maxK, rp.grp[ci.grp].K);
  }
  if (!P->cat_idx.empty())
    CUDA_TRY(c, cudaMemcpy(P->arena.base + P->cat_idx_off, P->cat_idx.data(), sizeof(CatIndex) * P->cat_idx.size(),
                           cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(P->arena.base + P->cvtask_off, P->cv_tasks.data(), sizeof(CatViewTask) * P->cv_tasks.size(),
                         cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(P->arena.base + P->ggram_off, P->ggram.data(), sizeof(GroupGram) * P->ggram.size(),
                         cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(P->arena.base + P->cgram_off, P->cgram.data(), sizeof(CrossGram) * P->cgram.size(),
                         cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(P->arena.base + P->cpair_off, P->cpairs.data(), sizeof(CrossPair) * P->cpairs.size(),
                         cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(P->arena.base + P->direct_off, direct.data(), sizeof(DirectAgg) * direct.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(P->arena.base + P->corr_off, corr.data(), sizeof(CorrTask) * corr.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(P->arena.base + P->maps_off, maps.data(), sizeof(OutMap) * maps.size(), cudaMemcpyHostToDevice));

  // general-path scales
  for (int r : P->post) {
    RelPlan& cp = P->rp[r];
    if (cp.unique) continue;
    double Wc = std::max<double>(1.0, (double)c->rels[r].nrows) * cp.maxcnt;
    double bmax = 0;
    for (int i = 0; i < cp.d; ++i) {
      double b = bound[cp.feat_names[i]];
      cp.s_scale[i] = (float)std::ldexp(1.0, fixp_exp(Wc * b));
      bmax = std::max(bmax, b);
    }
    cp.q_scale = std::ldexp(1.0, fixp_exp(Wc * bmax * bmax));
  }
  if (P->tree) {
    lmf_status s = tree_finish(P->tree.get(), P->arena.base, P->at<long long>(P->res_i64_off),
                               P->at<double>(P->res_f64_off), P->agg_off, filt_idx, P->agg_dtype,
                               P->at<uint32_t>(P->status_off), Root.nrows, c->num_sms, bound, W, rp, sorted_q);
    if (s) return fail(c, s, "tree plan: device tables");
    // the tree pass compiled for the plan (row pass and node search specialised;
    // the interpreted kernel stays when NVRTC is missing or the compile fails)
    if (!(P->opts.flags & LMF_PLAN_NO_JIT) && Root.nrows > 0 && jit_available()) {
      TreeJitSpec spec;
      tree_jit_spec(P->tree.get(), &spec);
      const std::string src = jit_tree_source(rp, spec);
      if (c->dry) {
        c->dry_sources.emplace_back(src, "lmf_tree_jit");
      } else {
        std::string log;
        cudaKernel_t k = nullptr;
        if (jit_kernel(src, "lmf_tree_jit", &k, &log))
          tree_set_jit(P->tree.get(), k);
        else
          std::fprintf(stderr, "lmf: plan-time compile of the tree pass failed, interpreted kernel kept: %.400s\n",
                       log.c_str());
      }
    }
  }
  if (use_tc) {
    gram_tc_finish(P->tc.get(), rp, P->arena.base);
  }
  // the compilation step (Sec. 1.2, App. C): the plain root scan with this
  // plan's layout as constants; the interpreted kernel stays when NVRTC is
  // missing or the compile fails (same arithmetic, same results)
  P->dry = c->dry;
  if (c->dry) {  // plan choice: collect the sources the compile step would build
    if (use_tc && !(P->opts.flags & LMF_PLAN_NO_JIT) && Root.nrows > 0 && jit_available())
      c->dry_sources.emplace_back(jit_tc_source(rp, direct), "lmf_root_tc_jit");
    if (P->lean) {
      const int lcps = (int)std::min<int64_t>(3, std::max<int64_t>(1, (int64_t)P->grid / std::max(1, c->num_sms)));
      c->dry_sources.emplace_back(jit_lean_source(rp, direct, lcps), "lmf_root_lean_jit");
    }
    if (!use_tc && !P->lean && !(P->opts.flags & LMF_PLAN_NO_JIT) && Root.nrows > 0 && jit_available())
      c->dry_sources.emplace_back(jit_plain_source(rp, P->mp, direct, jit3 ? 3 : 1), "lmf_root_plain_jit");
  } else if (use_tc && !(P->opts.flags & LMF_PLAN_NO_JIT) && Root.nrows > 0 && jit_available()) {
    std::string log;
    cudaKernel_t k = nullptr;
    if (jit_kernel(jit_tc_source(rp, direct), "lmf_root_tc_jit", &k, &log)) {
      CUDA_TRY(c, cudaFuncSetAttribute(reinterpret_cast<const void*>(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(P->tc->smem)));
      P->jit_tc = k;
    } else {
      std::fprintf(stderr, "lmf: plan-time compile failed, interpreted root scan kept: %.400s\n", log.c_str());
    }
  }
  if (P->lean && !c->dry) {  // the key-level scan exists only compiled: without it, plan the row-level form
    std::string log;
    cudaKernel_t k = nullptr;
    const int lcps = (int)std::min<int64_t>(3, std::max<int64_t>(1, (int64_t)P->grid / std::max(1, c->num_sms)));
    if (!jit_kernel(jit_lean_source(rp, direct, lcps), "lmf_root_lean_jit", &k, &log)) {
      std::fprintf(stderr, "lmf: plan-time compile of the key-level scan failed, row-level form planned: %.400s\n",
                   log.c_str());
      lmf_plan_opts o2 = opts;
      o2.flags |= LMF_PLAN_ROW_GRAM;
      P.reset();
      return plan_with_root(c, batch_id, o2, root);
    }
    CUDA_TRY(c, cudaFuncSetAttribute(reinterpret_cast<const void*>(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(P->smem)));
    P->jit_lean = k;
  }
  if (!c->dry && !use_tc && !P->lean && !(P->opts.flags & LMF_PLAN_NO_JIT) && Root.nrows > 0 && jit_available()) {
    std::string log;
    cudaKernel_t k = nullptr;
    if (jit_kernel(jit_plain_source(rp, P->mp, direct, jit3 ? 3 : 1), "lmf_root_plain_jit", &k, &log)) {
      CUDA_TRY(c, cudaFuncSetAttribute(reinterpret_cast<const void*>(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(P->smem)));
      P->jit_plain = k;
      P->grid = grid_jit;
    } else {
      std::fprintf(stderr, "lmf: plan-time compile failed, interpreted root scan kept: %.400s\n", log.c_str());
    }
  }
  P->n_views = (int)P->post.size();
  P->root_scan = !P->maps.empty();
  if (log_enabled()) log_plan(c, batch_id, *P);
  B.plan = std::move(P);
  return LMF_OK;
}

}  // namespace

namespace {

// Per-query roots (Sec. 3.3: every query evaluated at a root of its own, with
// the directional views towards that root).  The whole batch at the declared
// root when it plans there; otherwise its aggregates are grouped by the root
// they are tried at first -- the relation holding the first group-by,
// threshold or power attribute (where a group-by category is a column of the
// root itself), the declared root for plain linear sums -- each group planned
// as a hidden batch at the first of its candidate roots that evaluates it
// (single aggregates when a group fits none), and this batch's plan becomes
// the place their results are copied to after every run.
lmf_status plan_per_query(lmf_ctx* c, int batch_id, const lmf_plan_opts& opts) {
  {  // the hidden batches of an earlier per-query plan of this batch give back their memory
    BatchH& B0 = *c->batches[batch_id];
    if (B0.plan)
      for (int id : B0.plan->subs) c->batches[id]->plan.reset();
  }
  lmf_plan_opts o = opts;
  o.root_mode = LMF_ROOT_EXPLICIT;
  o.root_rel = c->root;
  lmf_status s = plan_with_root(c, batch_id, o, c->root);
  if (s != LMF_ERR_UNSUPPORTED) return s;
  BatchH& B = *c->batches[batch_id];
  const int n = (int)B.aggs.size();
  std::vector<int> by_size(c->rels.size());
  for (size_t r = 0; r < by_size.size(); ++r) by_size[r] = (int)r;
  std::stable_sort(by_size.begin(), by_size.end(),
                   [&](int a, int b) { return c->rels[a].nrows > c->rels[b].nrows; });
  auto candidates = [&](const AggH& a) {
    std::vector<int> out;
    auto add = [&](int r) {
      if (r >= 0 && std::find(out.begin(), out.end(), r) == out.end()) out.push_back(r);
    };
    int col = 0;
    for (auto& g : a.gb) add(owner_of(c, g, &col));
    for (auto& f : a.f)
      if (f.kind != LMF_POW) add(owner_of(c, f.attr, &col));
    add(c->root);
    for (int r : by_size) add(r);
    return out;
  };
  // groups keyed by the candidate list, in order of first appearance
  std::vector<std::vector<int>> keys;
  std::vector<std::vector<int>> members;
  for (int a = 0; a < n; ++a) {
    auto k = candidates(B.aggs[a]);
    size_t g = 0;
    while (g < keys.size() && keys[g] != k) ++g;
    if (g == keys.size()) {
      keys.push_back(k);
      members.emplace_back();
    }
    members[g].push_back(a);
  }
  std::vector<int> subs;
  std::vector<std::pair<int, int>> where(n, {-1, -1});  // aggregate -> (hidden batch, index in it)
  auto plan_group = [&](const std::vector<int>& aggs, const std::vector<int>& cand) -> lmf_status {
    const int id = (int)c->batches.size();
    auto hb = std::make_unique<BatchH>();
    for (int a : aggs) hb->aggs.push_back(B.aggs[a]);
    c->batches.push_back(std::move(hb));
    lmf_status st = LMF_ERR_UNSUPPORTED;
    for (int r : cand) {
      lmf_plan_opts q = o;
      q.root_rel = r;
      st = plan_with_root(c, id, q, r);
      if (st != LMF_ERR_UNSUPPORTED) break;
    }
    if (st != LMF_OK) {
      c->batches.pop_back();
      return st;
    }
    for (size_t j = 0; j < aggs.size(); ++j) where[aggs[j]] = {id, (int)j};
    subs.push_back(id);
    return LMF_OK;
  };
  for (size_t g = 0; g < keys.size(); ++g) {
    lmf_status st = plan_group(members[g], keys[g]);
    if (st == LMF_ERR_UNSUPPORTED && members[g].size() > 1) {
      for (int a : members[g]) {
        st = plan_group({a}, keys[g]);
        if (st) return fail(c, st, "aggregate %d fits no root", a);
      }
    } else if (st) {
      return st;
    }
  }
  // this batch's plan: the result arrays in the batch's layout and the copies
  auto P = std::make_unique<Plan>();
  P->opts = opts;
  P->root = c->root;
  P->subs = subs;
  P->agg_dtype.resize(n);
  P->agg_off.resize(n);
  P->agg_n.resize(n);
  for (int a = 0; a < n; ++a) {
    const Plan& S = *c->batches[where[a].first]->plan;
    const int j = where[a].second;
    P->agg_dtype[a] = S.agg_dtype[j];
    P->agg_n[a] = S.agg_n[j];
    if (S.agg_dtype[j] == LMF_I64) {
      P->agg_off[a] = P->n_i64;
      P->n_i64 += S.agg_n[j];
    } else {
      P->agg_off[a] = P->n_f64;
      P->n_f64 += S.agg_n[j];
    }
  }
  Arena& A = P->arena;
  P->status_off = A.take(16);
  P->res_i64_off = A.take((size_t)std::max<int64_t>(1, P->n_i64) * 8);
  P->res_f64_off = A.take((size_t)std::max<int64_t>(1, P->n_f64) * 8);
  P->copies_off = A.take(sizeof(ResultCopy) * (size_t)std::max(1, n));
  A.size = A.used + 256;
  {
    void* base = nullptr;
    if (cudaMalloc(&base, A.size) != cudaSuccess) return fail(c, LMF_ERR_OOM, "per-query result arrays");
    A.base = static_cast<char*>(base);
  }
  CUDA_TRY(c, cudaMemset(A.base, 0, A.size));
  for (int a = 0; a < n; ++a) {
    const Plan& S = *c->batches[where[a].first]->plan;
    const int j = where[a].second;
    const bool i64 = S.agg_dtype[j] == LMF_I64;
    ResultCopy rc;
    rc.src = reinterpret_cast<const long long*>(S.arena.base + (i64 ? S.res_i64_off : S.res_f64_off)) + S.agg_off[j];
    rc.dst = reinterpret_cast<long long*>(A.base + (i64 ? P->res_i64_off : P->res_f64_off)) + P->agg_off[a];
    rc.n = S.agg_n[j];
    P->copies.push_back(rc);
  }
  CUDA_TRY(c, cudaMemcpy(A.base + P->copies_off, P->copies.data(), sizeof(ResultCopy) * P->copies.size(),
                         cudaMemcpyHostToDevice));
  for (int id : subs) P->n_kernels += c->batches[id]->plan->n_kernels;
  P->n_kernels += 1;
  B.plan = std::move(P);
  return LMF_OK;
}

// ev (optional): LMF_STAGES + 1 events recorded on s at the stage boundaries
lmf_status enqueue(lmf_ctx* c, BatchH& B, cudaStream_t s, cudaEvent_t* ev = nullptr) {
  Plan* P = B.plan.get();
  int nk = 0;
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(ev[i], s);
  };
  mark(0);
  // host-resident columns are copied in first
  for (auto& r : c->rels)
    for (auto& col : r.cols)
      if (col.on_host == LMF_HOST_COPY && !col.remap && r.nrows > 0)
        CUDA_TRY(c, cudaMemcpyAsync(col.dev, col.data, (size_t)r.nrows * col.esize(), cudaMemcpyHostToDevice, s));
  CUDA_TRY(c, cudaMemsetAsync(P->arena.base + P->zero_off, 0, P->zero_len, s));
  mark(1);
  // child views, deepest first
  for (int r : P->post) {
    RelPlan& cp = P->rp[r];
    const RelationH& R = c->rels[r];
    GroupH& g = P->groups[cp.group];
    ViewArgs a{};
    a.nrows = R.nrows;
    a.key = static_cast<const int32_t*>(R.cols[R.find(P->key[r])].dptr());
    a.K = g.K;
    a.dst = P->at<uint32_t>(g.rec_off);
    a.dst_stride = g.stride;
    a.cnt_word = cp.slot;
    a.mu_off = g.child_mu_off[cp.slot];
    a.cat_off = g.child_cat_off[cp.slot];
    a.n_own = (int)cp.own_feat.size();
    for (int i = 0; i < a.n_own; ++i)
      a.own[i] = {R.cols[cp.own_feat[i]].dptr(), R.cols[cp.own_feat[i]].dtype == LMF_F64 ? 2 : 1};
    a.n_owncat = (int)cp.own_cat.size();
    for (int i = 0; i < a.n_owncat; ++i) {
      a.owncat[i] = static_cast<const int32_t*>(R.cols[cp.own_cat[i]].dptr());
      a.owncat_dom[i] = R.cols[cp.own_cat[i]].dom;
    }
    a.n_grp = (int)cp.groups.size();
    for (int q = 0; q < a.n_grp; ++q) {
      GroupH& cg = P->groups[cp.groups[q]];
      GroupDesc d;
      d.fk = static_cast<const int32_t*>(R.cols[R.find(cg.fk)].dptr());
      d.rec = P->at<uint32_t>(cg.rec_off);
      d.K = cg.K;
      d.stride = cg.stride;
      d.n_cnt = cg.n_cnt;
      d.n_mu = cg.n_mu;
      d.n_cat = cg.n_cat;
      d.fix = nullptr;
      d.fix_stride = 0;
      a.grp[q] = d;
    }
    a.status = P->at<uint32_t>(P->status_off);
    if (cp.unique) {
      CUDA_TRY(c, launch_view_unique(a, s));
      ++nk;
      continue;
    }
    a.d = cp.d;
    a.dq = cp.d * (cp.d + 1) / 2;
    a.cnt64 = P->at<unsigned long long>(cp.cnt64_off);
    a.S = P->at<long long>(cp.S_off);
    a.Q = P->at<long long>(cp.Q_off);
    for (int i = 0; i < cp.d; ++i) a.s_scale[i] = cp.s_scale[i];
    a.q_scale = cp.q_scale;
    a.n_sc = 0;
    int f0 = (int)cp.own_feat.size();
    for (int q = 0; q < a.n_grp; ++q) {
      GroupH& cg = P->groups[cp.groups[q]];
      for (size_t k = 0; k < cg.children.size(); ++k) {
        RelPlan& ep = P->rp[cg.children[k]];
        if (!ep.unique) {
          a.sc[a.n_sc] = P->at<double>(ep.sc_off);
          a.sc_grp[a.n_sc] = q;
          a.sc_cntword[a.n_sc] = (int)k;
          a.sc_feat0[a.n_sc] = f0;
          a.sc_d[a.n_sc] = ep.d;
          ++a.n_sc;
        }
        f0 += ep.d;
      }
    }
    CUDA_TRY(c, launch_view_general(a, s));
    ViewFinalizeArgs f{};
    f.K = g.K;
    f.d = cp.d;
    f.dq = a.dq;
    f.cnt64 = a.cnt64;
    f.S = a.S;
    f.Q = a.Q;
    for (int i = 0; i < cp.d; ++i) f.s_scale[i] = cp.s_scale[i];
    f.q_scale = cp.q_scale;
    f.dst = a.dst;
    f.dst_stride = g.stride;
    f.cnt_word = cp.slot;
    f.mu_off = a.mu_off;
    f.sc = P->at<double>(cp.sc_off);
    f.status = a.status;
    CUDA_TRY(c, launch_view_finalize(f, s));
    nk += 2;
  }
  for (const FixMeans& f : P->fixm) {
    CUDA_TRY(c, launch_fix_means(f, s));
    ++nk;
  }
  mark(2);
  // root scan: Gram, counts, reverse views, per-row grouped tables (skipped when
  // the batch has only threshold-filtered aggregates)
  if (P->root_scan) {
    if (P->tc && P->jit_tc) {
      void* args[] = {&P->rootp, &P->tc->n_tiles, &P->tc->part};
      CUDA_TRY(c, cudaLaunchKernel(reinterpret_cast<const void*>(P->jit_tc), dim3(P->tc->grid), dim3(128), args,
                                   P->tc->smem, s));
    } else if (P->tc) {
      CUDA_TRY(c, gram_tc_launch(P->tc.get(), P->rootp, s));
    } else if (P->lean) {
      void* args[] = {&P->rootp, &P->n_tiles};
      CUDA_TRY(c, cudaLaunchKernel(reinterpret_cast<const void*>(P->jit_lean), dim3(P->grid), dim3(kLeanT), args,
                                   P->smem, s));
    } else {
      if (P->jit_plain) {
        void* args[] = {&P->rootp, &P->n_tiles};
        CUDA_TRY(c, cudaLaunchKernel(reinterpret_cast<const void*>(P->jit_plain), dim3(P->grid), dim3(256), args,
                                     P->smem, s));
      } else {
        CUDA_TRY(c, launch_root_plain(P->rootp, P->mp, P->grid, P->n_tiles, P->smem, s));
      }
    }
    ++nk;
  }
  mark(3);
  if (P->tree) {
    CUDA_TRY(c, tree_launch(P->tree.get(), P->rootp, s, &nk));
  }
  mark(4);
  if (P->root_scan) {
    if (P->tc) {
      CUDA_TRY(c, gram_tc_combine(P->tc.get(), P->rootp, P->at<double>(P->G_off), P->at<long long>(P->count_off), s));
    } else if (P->lean) {  // the row Gram covers the root's features z[1, 1 + n_x)
      CUDA_TRY(c, launch_combine(P->at<double>(P->part_off), P->grid, P->lean_mpx, P->rootp.m,
                                 P->at<long long>(P->cntp_off), P->at<double>(P->G_off),
                                 P->at<long long>(P->count_off), s, P->rootp.gram_off, P->rootp.gram_n));
    } else {
      CUDA_TRY(c, launch_combine(P->at<double>(P->part_off), P->grid, P->mp, P->rootp.m,
                                 P->at<long long>(P->cntp_off), P->at<double>(P->G_off),
                                 P->at<long long>(P->count_off), s));
    }
    ++nk;
    if (!P->cgram.empty()) {
      CUDA_TRY(c, launch_cross_gram(P->at<CrossGram>(P->cgram_off), (int)P->cgram.size(), P->at<CrossPair>(P->cpair_off),
                                    Plan::kGgChunks, P->rootp, P->at<double>(P->cgram_part_off),
                                    P->at<double>(P->G_off), s));
      nk += 2;
    }
    if (!P->ggram.empty()) {
      CUDA_TRY(c, launch_group_gram(P->at<GroupGram>(P->ggram_off), (int)P->ggram.size(), Plan::kGgChunks, P->rootp,
                                    P->at<double>(P->ggram_part_off), P->at<double>(P->G_off), s));
      nk += 2;
    }
  }
  if (!P->corr.empty()) {
    CUDA_TRY(c, launch_corr(P->arena.base + P->corr_off, (int)P->corr.size(), P->at<double>(P->G_off), P->rootp.m, s));
    ++nk;
  }
  char* aux = static_cast<char*>(P->aux);
  if (!P->rv_items.empty()) {
    CUDA_TRY(c, launch_rv_items(P->at<RvTask>(P->rvtask_off), reinterpret_cast<const RvItem*>(aux + P->aux_rv),
                                (int)P->rv_items.size(), P->rv_item_cells, P->rootp, s));
    ++nk;
  }
  if (P->rv_wide) {
    CUDA_TRY(c, launch_rv_tasks(P->at<RvTask>(P->rvtask_off), P->rv_ranges, P->rootp, P->max_group_K, s));
    ++nk;
  }
  if (!P->cv_pair_items.empty()) {
    CUDA_TRY(c, launch_cat_index(P->at<CatIndex>(P->cat_idx_off), (int)P->cat_idx.size(), P->cat_idx_maxK, P->rootp,
                                 s));
    nk += 3;
    CUDA_TRY(c, launch_cv_pairs(P->at<CatViewTask>(P->cvtask_off), P->at<CatIndex>(P->cat_idx_off),
                                reinterpret_cast<const CvPairItem*>(aux + P->aux_cvp), (int)P->cv_pair_items.size(),
                                P->rootp, s));
    ++nk;
  }
  if (!P->cv_mean_items.empty()) {
    CUDA_TRY(c, launch_cv_means(P->at<CatViewTask>(P->cvtask_off), reinterpret_cast<const CvMeanItem*>(aux + P->aux_cvm),
                                (int)P->cv_mean_items.size(), P->rootp, s));
    ++nk;
  }
  if (!P->out_items.empty()) {
    CUDA_TRY(c, launch_out_map(P->at<OutMap>(P->maps_off), reinterpret_cast<const OutItem*>(aux + P->aux_out),
                               (int)P->out_items.size(), P->at<double>(P->G_off), P->rootp.m,
                               P->at<long long>(P->count_off), P->at<long long>(P->res_i64_off),
                               P->at<double>(P->res_f64_off), s));
    ++nk;
  }
  mark(5);
  P->n_kernels = nk;
  return LMF_OK;
}

// The tree-node histogram pass is autotuned once, on the first run, before any
// graph capture: one plain run fills the per-row buffers, then the tuner times
// its shape candidates on them and keeps the fastest.
lmf_status ensure_tuned(lmf_ctx* c, BatchH& B, cudaStream_t s) {
  Plan* P = B.plan.get();
  if (!P->tree || !tree_needs_tuning(P->tree.get())) return LMF_OK;
  lmf_status st = enqueue(c, B, s);
  if (st) return st;
  CUDA_TRY(c, tree_autotune(P->tree.get(), P->rootp, s));
  CUDA_TRY(c, cudaStreamSynchronize(s));
  return LMF_OK;
}

}  // namespace

extern "C" {

lmf_status lmf_plan_info(lmf_ctx* c, int batch_id, lmf_plan_stats* info) {
  if (!c || !info || batch_id < 0 || batch_id >= (int)c->batches.size()) return LMF_ERR_ARG;
  Plan* P = c->batches[batch_id]->plan.get();
  if (!P) return fail(c, LMF_ERR_STATE, "batch not planned");
  if (!P->subs.empty()) {  // per-query roots: the first root's plan, with the totals of all
    lmf_status st = lmf_plan_info(c, P->subs[0], info);
    if (st) return st;
    info->n_roots = (int32_t)P->subs.size();
    info->n_kernels_per_run = P->n_kernels;
    info->n_gram_aggs = info->n_grouped_aggs = info->n_filtered_aggs = 0;
    info->n_views = 0;
    for (int id : P->subs) {
      const Plan& S = *c->batches[id]->plan;
      info->n_gram_aggs += S.n_gram;
      info->n_grouped_aggs += S.n_grouped;
      info->n_filtered_aggs += S.n_filtered;
      info->n_views += S.n_views;
    }
    info->root_rel = -1;
    return LMF_OK;
  }
  std::memset(info, 0, sizeof(*info));
  info->n_roots = 1;
  info->n_views = P->n_views;
  info->n_probe_groups = P->rootp.n_grp;
  info->z_len = P->rootp.m;
  info->n_gram_aggs = P->n_gram;
  info->n_grouped_aggs = P->n_grouped;
  info->n_filtered_aggs = P->n_filtered;
  info->n_kernels_per_run = P->n_kernels;
  info->unique_keys = P->unique_all ? 1 : 0;
  info->root_grid = P->grid;
  info->precision = P->tc ? LMF_PREC_SPLIT_BF16 : LMF_PREC_PLAIN_FP32;
  info->root_rel = P->root;
  info->merged = P->merge ? 1 : 0;
  if (P->tree) {
    int t5[5];
    tree_shape(P->tree.get(), t5);
    tree_counts(P->tree.get(), &info->tree_nodes, &info->tree_groups);
    info->tree_slices = t5[0];
    info->tree_split_w = t5[1];
    info->tree_node_w = t5[2];
    info->tree_ctas_per_sm = t5[3];
    info->tree_chunk = t5[4];
  }
  info->root_rows = P->rootp.N;
  info->scratch_bytes = (int64_t)P->arena.size;
  info->resident_group = P->rootp.res_cells > 0 ? P->rootp.res_grp : -1;
  info->resident_cells = P->rootp.res_cells;
  info->jit = (P->jit_plain || P->jit_tc || P->jit_lean) ? 1 : 0;
  info->key_level = P->lean ? 1 : 0;
  return LMF_OK;
}

lmf_status lmf_run(lmf_ctx* c, int batch_id, void* cuda_stream) {
  if (!c || batch_id < 0 || batch_id >= (int)c->batches.size()) return fail(c, LMF_ERR_ARG, "run: bad batch id");
  BatchH& B = *c->batches[batch_id];
  Plan* P = B.plan.get();
  if (!P) return fail(c, LMF_ERR_STATE, "run before plan");
  if (P->dry) return fail(c, LMF_ERR_STATE, "run of a plan built for plan choice only");
  cudaSetDevice(c->device);
  cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : c->stream;
  B.last_stream = s;
  if (!P->subs.empty()) {  // per-query roots: every root's plan, then the results copied in
    for (int id : P->subs) {
      lmf_status st = lmf_run(c, id, s);
      if (st) return st;
    }
    CUDA_TRY(c, launch_copy_results(P->at<ResultCopy>(P->copies_off), (int)P->copies.size(), s));
    return LMF_OK;
  }
  {
    lmf_status st = ensure_tuned(c, B, s);
    if (st) return st;
  }
  if (P->opts.batching == LMF_BATCH_GRAPH) {
    if (!P->exec) {
      if (!P->graph_stream) CUDA_TRY(c, cudaStreamCreateWithFlags(&P->graph_stream, cudaStreamNonBlocking));
      CUDA_TRY(c, cudaStreamBeginCapture(P->graph_stream, cudaStreamCaptureModeThreadLocal));
      lmf_status st = enqueue(c, B, P->graph_stream);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(P->graph_stream, &g);
      if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return fail(c, LMF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
      P->graph = g;
      CUDA_TRY(c, cudaGraphInstantiate(&P->exec, g, 0));
    }
    CUDA_TRY(c, cudaGraphLaunch(P->exec, s));
    return LMF_OK;
  }
  return enqueue(c, B, s);
}

lmf_status lmf_run_profiled(lmf_ctx* c, int batch_id, void* cuda_stream, float* stage_ms) {
  if (!c || !stage_ms || batch_id < 0 || batch_id >= (int)c->batches.size())
    return fail(c, LMF_ERR_ARG, "run_profiled: bad argument");
  BatchH& B = *c->batches[batch_id];
  if (!B.plan) return fail(c, LMF_ERR_STATE, "run before plan");
  if (B.plan->dry) return fail(c, LMF_ERR_STATE, "run of a plan built for plan choice only");
  cudaSetDevice(c->device);
  cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : c->stream;
  B.last_stream = s;
  if (!B.plan->subs.empty()) {  // per-query roots: the stages summed over the roots' plans
    for (int i = 0; i < LMF_STAGES; ++i) stage_ms[i] = 0.f;
    for (int id : B.plan->subs) {
      float st_ms[LMF_STAGES];
      lmf_status st = lmf_run_profiled(c, id, s, st_ms);
      if (st) return st;
      for (int i = 0; i < LMF_STAGES; ++i) stage_ms[i] += st_ms[i];
    }
    CUDA_TRY(c, launch_copy_results(B.plan->at<ResultCopy>(B.plan->copies_off), (int)B.plan->copies.size(), s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    return LMF_OK;
  }
  {
    lmf_status st = ensure_tuned(c, B, s);
    if (st) return st;
  }
  struct Events {
    cudaEvent_t e[LMF_STAGES + 1] = {};
    ~Events() {
      for (auto x : e)
        if (x) cudaEventDestroy(x);
    }
  } ev;
  for (auto& e : ev.e) CUDA_TRY(c, cudaEventCreate(&e));
  lmf_status st = enqueue(c, B, s, ev.e);
  if (st == LMF_OK) {
    CUDA_TRY(c, cudaEventSynchronize(ev.e[LMF_STAGES]));
    for (int i = 0; i < LMF_STAGES; ++i) cudaEventElapsedTime(&stage_ms[i], ev.e[i], ev.e[i + 1]);
    if (log_enabled())
      std::fprintf(stderr, "lmf: batch %d run: input %.3f, views %.3f, root scan %.3f, tree %.3f, finalize %.3f ms\n",
                   batch_id, stage_ms[0], stage_ms[1], stage_ms[2], stage_ms[3], stage_ms[4]);
  }
  return st;
}

lmf_status lmf_wait_selftest(lmf_ctx* c) {
  if (!c) return LMF_ERR_ARG;
  cudaSetDevice(c->device);
  uint32_t* d = nullptr;
  CUDA_TRY(c, cudaMalloc(&d, sizeof(uint32_t)));
  uint32_t st = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(uint32_t), c->stream);
  if (e == cudaSuccess) e = gram_tc_wait_selftest(d, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, d, sizeof(st), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  if (e != cudaSuccess) return fail(c, LMF_ERR_CUDA, "wait self-test: %s", cudaGetErrorString(e));
  if (st & kStatusTimeout) return fail(c, LMF_ERR_TIMEOUT, "the bounded wait gave up (as expected)");
  return LMF_OK;
}

lmf_status lmf_sync(lmf_ctx* c, int batch_id) {
  if (!c || batch_id < 0 || batch_id >= (int)c->batches.size()) return fail(c, LMF_ERR_ARG, "sync: bad batch id");
  BatchH& B = *c->batches[batch_id];
  Plan* P = B.plan.get();
  if (!P) return fail(c, LMF_ERR_STATE, "sync before plan");
  cudaSetDevice(c->device);
  for (int id : P->subs) {  // per-query roots: each root's plan reports its own status
    lmf_status st = lmf_sync(c, id);
    if (st) return st;
  }
  cudaStream_t s = B.last_stream ? B.last_stream : c->stream;
  uint32_t st = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&st, P->arena.base + P->status_off, sizeof(st), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(c, cudaStreamSynchronize(s));
  if (st & kStatusTimeout) return fail(c, LMF_ERR_TIMEOUT, "a device wait gave up");
  if (st & kStatusOverflow) return fail(c, LMF_ERR_OVERFLOW, "a subtree count exceeded int32");
  if (st & (kStatusCatRange | kStatusKeyRange)) return fail(c, LMF_ERR_KEY, "category or key out of range (status %u)", st);
  return LMF_OK;
}

lmf_status lmf_result_info(lmf_ctx* c, int batch_id, int agg, int64_t* n_groups, int32_t* dtype, int64_t* offset) {
  if (!c || batch_id < 0 || batch_id >= (int)c->batches.size()) return LMF_ERR_ARG;
  Plan* P = c->batches[batch_id]->plan.get();
  if (!P) return fail(c, LMF_ERR_STATE, "batch not planned");
  if (agg < 0 || agg >= (int)P->agg_n.size()) return fail(c, LMF_ERR_ARG, "bad aggregate index");
  if (n_groups) *n_groups = P->agg_n[agg];
  if (dtype) *dtype = P->agg_dtype[agg];
  if (offset) *offset = P->agg_off[agg];
  return LMF_OK;
}

lmf_status lmf_result_sizes(lmf_ctx* c, int batch_id, int64_t* n_i64, int64_t* n_f64) {
  if (!c || batch_id < 0 || batch_id >= (int)c->batches.size()) return LMF_ERR_ARG;
  Plan* P = c->batches[batch_id]->plan.get();
  if (!P) return fail(c, LMF_ERR_STATE, "batch not planned");
  if (n_i64) *n_i64 = P->n_i64;
  if (n_f64) *n_f64 = P->n_f64;
  return LMF_OK;
}

lmf_status lmf_read_results(lmf_ctx* c, int batch_id, int64_t* dst_i64, double* dst_f64, int dst_is_device,
                            void* cuda_stream) {
  if (!c || batch_id < 0 || batch_id >= (int)c->batches.size()) return LMF_ERR_ARG;
  BatchH& B = *c->batches[batch_id];
  Plan* P = B.plan.get();
  if (!P) return fail(c, LMF_ERR_STATE, "batch not planned");
  cudaSetDevice(c->device);
  cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : (B.last_stream ? B.last_stream : c->stream);
  cudaMemcpyKind k = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (dst_i64 && P->n_i64 > 0)
    CUDA_TRY(c, cudaMemcpyAsync(dst_i64, P->arena.base + P->res_i64_off, P->n_i64 * 8, k, s));
  if (dst_f64 && P->n_f64 > 0)
    CUDA_TRY(c, cudaMemcpyAsync(dst_f64, P->arena.base + P->res_f64_off, P->n_f64 * 8, k, s));
  if (!dst_is_device) CUDA_TRY(c, cudaStreamSynchronize(s));
  return LMF_OK;
}

lmf_status lmf_read_result(lmf_ctx* c, int batch_id, int agg, void* dst) {
  if (!c || !dst || batch_id < 0 || batch_id >= (int)c->batches.size()) return LMF_ERR_ARG;
  BatchH& B = *c->batches[batch_id];
  Plan* P = B.plan.get();
  if (!P) return fail(c, LMF_ERR_STATE, "batch not planned");
  if (agg < 0 || agg >= (int)P->agg_n.size()) return fail(c, LMF_ERR_ARG, "bad aggregate index");
  cudaSetDevice(c->device);
  cudaStream_t s = B.last_stream ? B.last_stream : c->stream;
  size_t base = P->agg_dtype[agg] == LMF_I64 ? P->res_i64_off : P->res_f64_off;
  CUDA_TRY(c, cudaMemcpyAsync(dst, P->arena.base + base + P->agg_off[agg] * 8, P->agg_n[agg] * 8,
                              cudaMemcpyDeviceToHost, s));
  CUDA_TRY(c, cudaStreamSynchronize(s));
  return LMF_OK;
}

}  // extern "C"

// ============================================================================
// plan choice: candidates, features, learned selection
namespace {

constexpr int kPlanFeatures = 26;

void plan_features(lmf_ctx* c, const Plan& P, float* f) {
  double total_rows = 0, max_rows = 1;
  for (auto& r : c->rels) {
    total_rows += (double)r.nrows;
    max_rows = std::max(max_rows, (double)r.nrows);
  }
  const double root_rows = (double)std::max<int64_t>(1, P.rootp.N);
  double rec_bytes = 0, general_work = 0;
  int non_unique = 0, max_mult = 1;
  for (auto& g : P.groups) rec_bytes += (double)g.K * g.stride * 4;
  for (int r : P.post) {
    max_mult = std::max(max_mult, P.mult[r]);
    if (!P.rp[r].unique) {
      ++non_unique;
      general_work += (double)c->rels[r].nrows * (P.rp[r].d * (P.rp[r].d + 1) / 2 + P.rp[r].d + 1);
    }
  }
  double cells = 0;
  for (auto& o : P.maps)
    if (o.kind >= 2) cells += (double)o.n;
  int slots = 0;
  for (int q = 0; q < P.rootp.n_rv; ++q) slots += P.rootp.rv[q].n_slot;
  int fanin = 1;
  for (int r = 0; r < (int)c->rels.size(); ++r)
    if (c->rels[r].parent >= 0) fanin = std::max(fanin, c->rels[r].fk_mult);
  const float v[kPlanFeatures] = {
      (float)std::log2(root_rows + 1), (float)std::log2(total_rows + 1), (float)c->rels.size(),
      (float)P.post.size(), (float)P.rootp.n_grp, (float)P.rootp.m, (float)std::log2(rec_bytes + 1),
      (float)P.n_gram, (float)P.n_grouped, (float)P.n_filtered, (float)std::log2(cells + 1),
      P.unique_all ? 1.f : 0.f, (float)std::log2((double)max_mult + 1), P.tc ? 1.f : 0.f,
      (float)P.grid / (float)std::max(1, c->num_sms), P.merge ? 1.f : 0.f,
      (double)c->rels[P.root].nrows >= max_rows ? 1.f : 0.f, (float)(std::log2(root_rows) - std::log2(max_rows)),
      (float)non_unique, (float)std::log2(general_work + 1), (float)slots, (float)P.direct.size(),
      (float)std::log2((double)fanin + 1), P.tree ? 1.f : 0.f, P.lean ? 1.f : 0.f, (float)P.run_log2};
  std::memcpy(f, v, sizeof(v));
}

std::vector<lmf_plan_opts> plan_candidates(lmf_ctx* c, const BatchH& B, const lmf_plan_opts& base) {
  std::vector<int> roots{c->root};
  const int h = heuristic_root(c, B);
  if (h != roots[0]) roots.push_back(h);
  std::vector<int> by_size;
  for (int r = 0; r < (int)c->rels.size(); ++r) by_size.push_back(r);
  std::stable_sort(by_size.begin(), by_size.end(),
                   [&](int a, int b) { return c->rels[a].nrows > c->rels[b].nrows; });
  for (int r : by_size) {
    if ((int)roots.size() >= 3) break;
    if (std::find(roots.begin(), roots.end(), r) == roots.end()) roots.push_back(r);
  }
  // Gram forms: plain FP32 with key-level blocks, plain FP32 all at the row
  // level, split bf16 on the tensor cores.  Views stay merged per parent key
  // (case (1) of Sec. 3.4): across the plan-choice corpus turning merging off
  // changed no candidate's time by more than 1% (median ratio 1.000), while on
  // a snowflake whose sub-dimensions share a key it costs a gather per view
  struct Form { int prec, flags; };
  const Form forms[] = {{LMF_PREC_PLAIN_FP32, 0}, {LMF_PREC_PLAIN_FP32, LMF_PLAN_ROW_GRAM},
                        {LMF_PREC_SPLIT_BF16, 0}};
  std::vector<lmf_plan_opts> out;
  for (int r : roots)
    for (const Form& f : forms) {
      lmf_plan_opts o = base;
      o.root_mode = LMF_ROOT_EXPLICIT;
      o.root_rel = r;
      o.precision = f.prec;
      o.flags = (base.flags & ~LMF_PLAN_ROW_GRAM) | f.flags;
      o.no_merge = 0;
      out.push_back(o);
    }
  return out;
}

// plan every candidate dry (features, no compile) and return those that plan
lmf_status dry_candidates(lmf_ctx* c, int batch_id, const std::vector<lmf_plan_opts>& cand,
                          std::vector<lmf_plan_opts>* ok, std::vector<float>* feats) {
  BatchH& B = *c->batches[batch_id];
  c->dry = true;
  c->dry_sources.clear();
  for (const lmf_plan_opts& o : cand) {
    if (lmf_plan(c, batch_id, &o) != LMF_OK) continue;
    if (feats) {
      float f[kPlanFeatures];
      plan_features(c, *B.plan, f);
      feats->insert(feats->end(), f, f + kPlanFeatures);
    }
    ok->push_back(o);
  }
  c->dry = false;
  B.plan.reset();
  return LMF_OK;
}

}  // namespace

extern "C" {

lmf_status lmf_plan_features(lmf_ctx* c, int batch_id, float* feat, int n) {
  if (!c || !feat || batch_id < 0 || batch_id >= (int)c->batches.size()) return LMF_ERR_ARG;
  Plan* P = c->batches[batch_id]->plan.get();
  if (!P) return fail(c, LMF_ERR_STATE, "features before plan");
  if (!P->subs.empty()) return fail(c, LMF_ERR_STATE, "a per-query plan has no single set of features");
  if (n < kPlanFeatures) return fail(c, LMF_ERR_ARG, "need %d feature slots", kPlanFeatures);
  plan_features(c, *P, feat);
  return LMF_OK;
}

lmf_status lmf_plan_candidates(lmf_ctx* c, int batch_id, const lmf_plan_opts* base, lmf_plan_opts* out, int max,
                               int* n) {
  if (!c || !n || batch_id < 0 || batch_id >= (int)c->batches.size()) return LMF_ERR_ARG;
  if (!c->joined) return fail(c, LMF_ERR_STATE, "candidates before declare_join");
  lmf_plan_opts b{};
  if (base) b = *base;
  auto cand = plan_candidates(c, *c->batches[batch_id], b);
  *n = (int)cand.size();
  for (int i = 0; i < std::min<int>(max, (int)cand.size()) && out; ++i) out[i] = cand[i];
  return LMF_OK;
}

lmf_status lmf_plan_precompile(lmf_ctx* c, int batch_id, const lmf_plan_opts* base, int threads, int* n_compiled) {
  if (!c || batch_id < 0 || batch_id >= (int)c->batches.size() || threads < 0) return LMF_ERR_ARG;
  if (!c->joined) return fail(c, LMF_ERR_STATE, "precompile before declare_join");
  lmf_plan_opts b{};
  if (base) b = *base;
  auto cand = plan_candidates(c, *c->batches[batch_id], b);
  std::vector<lmf_plan_opts> ok;
  dry_candidates(c, batch_id, cand, &ok, nullptr);
  auto jobs = std::move(c->dry_sources);
  c->dry_sources.clear();
  const int n = jit_kernels_parallel(jobs, threads > 0 ? threads : 8, c->device);
  if (n_compiled) *n_compiled = n;
  return LMF_OK;
}

lmf_status lmf_plan_learned(lmf_ctx* c, int batch_id, lmf_mlp* model, const lmf_plan_opts* base,
                            lmf_plan_opts* chosen) {
  if (!c || batch_id < 0 || batch_id >= (int)c->batches.size()) return LMF_ERR_ARG;
  if (!c->joined) return fail(c, LMF_ERR_STATE, "plan before declare_join");
  lmf_plan_opts b{};
  if (base) {
    b = *base;
  } else {
    b.precision = LMF_PREC_SPLIT_BF16;
    b.batching = LMF_BATCH_GRAPH;
  }
  if (!model) {  // fallback: the root rule of Sec. 3.3 with the base options
    b.root_mode = LMF_ROOT_HEURISTIC;
    lmf_status s = lmf_plan(c, batch_id, &b);
    if (s == LMF_OK && chosen) {
      *chosen = b;
      chosen->root_mode = LMF_ROOT_EXPLICIT;
      chosen->root_rel = c->batches[batch_id]->plan->root;
    }
    return s;
  }
  BatchH& B = *c->batches[batch_id];
  auto cand = plan_candidates(c, B, b);
  std::vector<float> feats;
  std::vector<lmf_plan_opts> ok;
  dry_candidates(c, batch_id, cand, &ok, &feats);
  c->dry_sources.clear();
  if (ok.empty()) return fail(c, LMF_ERR_UNSUPPORTED, "no candidate plan evaluates this batch");
  float *dx = nullptr, *dy = nullptr;
  CUDA_TRY(c, cudaMalloc(&dx, feats.size() * 4));
  CUDA_TRY(c, cudaMalloc(&dy, ok.size() * 4));
  CUDA_TRY(c, cudaMemcpy(dx, feats.data(), feats.size() * 4, cudaMemcpyHostToDevice));
  lmf_status s = lmf_mlp_forward(model, dx, (int)ok.size(), dy);
  std::vector<float> pred(ok.size());
  if (s == LMF_OK) cudaMemcpy(pred.data(), dy, ok.size() * 4, cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dy);
  if (s) return fail(c, s, "cost model forward failed");
  size_t best = 0;
  for (size_t i = 1; i < ok.size(); ++i)
    if (pred[i] < pred[best]) best = i;
  s = lmf_plan(c, batch_id, &ok[best]);
  if (s == LMF_OK && chosen) *chosen = ok[best];
  return s;
}

}  // extern "C"
