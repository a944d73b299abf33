// lmf_internal.h -- plan structures shared by the host planner (lmf_api.cu)
// and the device kernels (lmf_kernels.cu, lmf_gram_tc.cu, lmf_tree.cu).
//
// Vocabulary follows the paper: a *view* is the directional view of a child
// relation towards its parent (Sec. 3.2), keyed by the join key; views that
// leave their children towards the same parent key are merged into one
// record array (merge case (1) of Sec. 3.4) called a *probe group* here.
#pragma once

#ifdef __CUDACC_RTC__  // compiled at plan time by NVRTC: no host headers
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef long long int64_t;
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
#else
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#endif

namespace lmf {

constexpr int kMaxGroups = 8;        // probe groups of one relation (distinct FK columns)
constexpr int kMaxZ = 64;            // length of z = [1, root features, view means]
constexpr int kMaxOwn = 48;          // own continuous columns of one relation
constexpr int kMaxCat = 32;          // categorical words of one record / root row
constexpr int kMaxQ = kMaxZ * (kMaxZ + 1) / 2;
constexpr int kDirInline = 96;        // per-row tables whose descriptors ride in the kernel parameters
constexpr int kMaxCatViews = 64;      // category views of one root scan
constexpr int kLeanT = 256;           // key-level root scan: rows per tile, one per thread

// device status bits (OR-ed by kernels, read by lmf_sync)
constexpr uint32_t kStatusCatRange = 1u;      // category outside [0, domain)
constexpr uint32_t kStatusOverflow = 2u;      // an exact count left its integer range
constexpr uint32_t kStatusTimeout = 4u;       // a bounded device wait gave up
constexpr uint32_t kStatusKeyRange = 8u;      // a child key outside the indexed range

struct Col {
  const void* p;
  int32_t dtype;                     // 0 i32, 1 f32, 2 f64
};

// One merged view record array (probe group).  Record k of a group holds, for
// every child c of the group, its subtree count at word cnt[c] (int32), the
// means of its subtree features (float) and its carried categories (int32).
// Word layout: [n_cnt counts][n_mu means][n_cat categories], stride padded to
// a multiple of 4 words so one record is read with 128-bit loads.
struct GroupDesc {
  const int32_t* fk;                 // foreign-key column of the probing relation
  uint32_t* rec;                     // [K][stride] words
  int32_t K;                         // keys 0..K-1 (direct addressing)
  int32_t stride;                    // words per record
  int32_t n_cnt, n_mu, n_cat;
  // key-level plans: exact fixed-point images of the means the reverse views
  // sum, [K][fix_stride] int64 (fix_stride even: 16-byte records), written
  // once per run from the records by k_fix_means; null when none
  long long* fix;
  int32_t fix_stride;
};

// fixed-point images of a probe group's means (key-level plans)
struct FixMeans {
  GroupDesc g;
  int32_t n;                         // images per key
  int16_t mu_word[kMaxZ];            // record word of each mean
  float scale[kMaxZ];                // fixed-point scale (power of 2) of each
};

// Build of one child relation's section of its parent's group record (A2).
struct ViewArgs {
  int64_t nrows;
  const int32_t* key;                // the child's join key column
  int32_t K;                         // size of the parent group's key space
  uint32_t* dst;                     // parent's group record array
  int32_t dst_stride;
  int32_t cnt_word;                  // word of this child's count
  int32_t mu_off;                    // first mean word of this child's section
  int32_t cat_off;                   // first category word of this child's section
  int32_t n_own;                     // own continuous columns -> first means
  Col own[kMaxOwn];
  int32_t n_owncat;                  // own categorical columns -> first categories
  const int32_t* owncat[kMaxCat];
  int32_t owncat_dom[kMaxCat];
  int32_t n_grp;                     // the child's own probe groups (its children)
  GroupDesc grp[kMaxGroups];
  // general (non-unique) path only
  int32_t d;                         // subtree features of the child
  int32_t dq;                        // d (d + 1) / 2
  unsigned long long* cnt64;         // [K] subtree counts
  long long* S;                      // [K][d] fixed-point sums
  long long* Q;                      // [K][dq] fixed-point second moments
  float s_scale[kMaxOwn + kMaxZ];    // fixed-point scale of S per feature (power of 2)
  double q_scale;                    // fixed-point scale of Q (power of 2)
  // second moments of the grand-children that fan out: per group child
  int32_t n_sc;
  const double* sc[kMaxGroups * 4];  // [K_e][dq_e] within-key scatter of child e
  int32_t sc_grp[kMaxGroups * 4];    // group of e in this relation
  int32_t sc_cntword[kMaxGroups * 4];// count word of e in that group's record
  int32_t sc_feat0[kMaxGroups * 4];  // first subtree feature of e in this child's vector
  int32_t sc_d[kMaxGroups * 4];      // subtree features of e
  uint32_t* status;
};

// finalize of a general view: counts, means and within-key scatter per key
struct ViewFinalizeArgs {
  int32_t K, d, dq;
  const unsigned long long* cnt64;
  const long long* S;
  const long long* Q;
  float s_scale[kMaxOwn + kMaxZ];
  double q_scale;
  uint32_t* dst;                      // parent's group record array
  int32_t dst_stride, cnt_word, mu_off;
  double* sc;                         // [K][dq]
  uint32_t* status;
};

// reverse view of the root towards one probe group: per key of the group,
// SUM(w) and SUM(w * z_s) for the slots s (the view from the root towards a
// dimension, Sec. 3.2 directional views; used for grouped outputs).
struct RevView {
  unsigned long long* hist;          // count of key k at hist[k * hstride]
  long long* R;                      // slot s of key k at R[k * rstride + s]
  int32_t grp;                       // root probe group
  int32_t n_slot;
  int16_t slot_z[kMaxZ];             // z index of each slot
  float slot_scale[kMaxZ];           // fixed-point scale per slot (power of 2)
  // Layout.  Row-level Gram plans: hist [K] and R [K][n_slot] (hstride 1,
  // rstride n_slot).  Key-level plans (RootParams::lean): one record of
  // `stride` int64 words per key, word 0 the count and words 1..n_slot the
  // slots (hist points at word 0, R at word 1, both strides = stride); stride
  // is even so that a record is a whole number of 16-byte units.
  int32_t hstride, rstride;
  int32_t stride;                    // key-level plans: int64 words per key
  int32_t mode;                      // key-level plans: how the scan updates it (kRv*)
};

// update modes of a reverse view in the key-level root scan
constexpr int kRvRuns = 0;           // FP32 sum of every run of equal keys in a warp, one reduction per run
constexpr int kRvResident = 1;       // the CTA's resident key: per-lane sums in registers until the key changes
constexpr int kRvBulk = 2;           // every row's record added by one bulk reduction (cp.reduce.async.bulk)

__host__ __device__ inline unsigned long long rv_hist(const RevView& R, int64_t k) { return R.hist[k * R.hstride]; }
__host__ __device__ inline long long rv_slot(const RevView& R, int64_t k, int s) { return R.R[k * R.rstride + s]; }

// one grouped aggregate accumulated row by row (group-by categories that are
// not all functions of one foreign key)
struct DirectAgg {
  int32_t n_gb;
  int32_t cat[3];                    // positions in the row's category vector
  int32_t dom[3];
  int32_t z;                         // -1: count; else z index of SUM(z)
  float scale;
  long long* out;                    // [cells] fixed-point / counts
  int32_t cache_off;                 // pair tables: first cache cell of its hot x hot block, else -1
  // resident-key form (COUNT tables with one category from the resident probe
  // group): the CTA counts the rows of the current resident key in shared
  // memory over the other categories' cells
  int32_t res_off;                   // first shared counter, -1: not resident
  int32_t res_q;                     // group-by position of the resident group's category
  int32_t res_word;                  // that category's word in the resident group's record
  int32_t res_n;                     // cells: product of the other positions' domains
  int32_t res_lanes;                 // 1: 32 counters per cell, one per lane (no same-address
                                     //    conflicts inside a warp), 0: one counter per cell
  int32_t runs;                      // 1: its cells come in runs of equal values (sum them per warp)
};

// A directional view from the root towards probe group grp that keeps one
// more group-by attribute, the category b of another probe group or of the
// root (Sec. 3.2: a view's group-by holds its join key and the attributes the
// aggregates above it need): V[k][vb] = sum of w over the root rows with key
// k and b = vb.  Every COUNT table (a, b) with a carried by grp is read off it
// by a pass over grp's keys, so a root row makes one update per view instead
// of one per table.
struct CatView {
  int32_t grp;                       // keying probe group
  int32_t bcat;                      // row-category index of b
  int32_t dom;                       // domain of b
  int32_t res_off;                   // grp is the resident group: first of dom shared counters, else -1
  int32_t runs;                      // 1: (key, b) comes in runs (sum them per warp)
  int32_t pad;
  uint32_t* V;                       // [K of grp][dom] counts (w is 0 or 1, fewer than 2^32 rows)
};

// COUNT table (a, b) read off its category view: for every key k,
// T[a(k)][vb] += V[k][vb]
struct CatViewTask {
  int32_t view;                      // index into RootParams::cv
  int32_t a_word;                    // a's word in the keying group's record
  int32_t dom_a;
  int32_t a_first;                   // 1: cells a * dom_b + b, 0: b * dom_a + a
  long long* out;
  // mode 1: SUM of a mean m of the keying group grouped by b alone,
  // T[vb] += V[k][vb] * m(k) (fixed-point, one rounding per cell): the mean
  // is constant over key k, so the view's counts weight it exactly
  int32_t mode;                      // 0: COUNT table (a, b), 1: SUM(m) grouped by b
  int32_t mu_word;                   // mode 1: m's word in the keying group's record
  float scale;                       // mode 1: fixed-point scale of the output
  int32_t fix_idx;                   // mode 1: m's fixed-point image in the keying group's fix records
                                     // (count * image, exact integers), -1: rounded in FP64 per cell
  int32_t cat_idx;                   // mode 0: the CatIndex of (keying group, a_word)
  int32_t pad;
};

// Gram entries taken at the key level from a reverse view R keyed by probe
// group g (the aggregate at the root of g, Sec. 3.3):
//   G[za][zb] = sum over keys k of R[k][s] / scale_s * m_i(k)
// where slot s holds sum w z_a over the root rows with key k and m_i is mean i
// of group g (constant over key k; i = -1: the constant 1, giving SUM(z_a)).
struct CrossPair {
  int16_t s, i;                      // reverse-view slot, mean index (-1: 1)
  int16_t za, zb;                    // Gram entry
};
struct CrossGram {
  int32_t rv;                        // index into RootParams::rv
  int32_t grp;                       // probe group (the view's key)
  int32_t mu_word;                   // record word of mean 0
  int32_t npair;
  int32_t pair_off;                  // first pair in the pair table
  int32_t part_off;                  // first partial: [npair][n_parts]
};

// Gram block of one probe group's view means, taken at the key level: for z
// slots i, j of the group (i = -1: the constant 1),
//   G[i][j] = sum over root rows of w z_i z_j = sum over keys k of hist(k) m_i(k) m_j(k)
// since z_i = m_i(k) on every row with key k (the aggregate evaluated at the
// group's own root, Sec. 3.3, over the view of counts from the root).  FP64
// over the keys, in a fixed order: no FP32 rounding repeated over a run of
// equal keys.
struct GroupGram {
  int32_t grp;                       // probe group
  int32_t rv;                        // reverse view holding hist(k)
  int32_t n;                         // means of the group (z slots zoff .. zoff + n - 1)
  int32_t zoff;
  int32_t mu_word;                   // record word of the first mean
  int32_t npair;                     // (n + 1)(n + 2)/2 - 1 pairs (i <= j, not both -1)
  int32_t part_off;                  // first partial of this block: [npair][n_parts]
  int32_t pad;
};

struct OmegaAcc {                    // SUM over root rows of w / cnt_e per key of e
  int32_t grp;
  int32_t cnt_word;
  unsigned long long* omega;         // [K]
};

struct RootParams {
  int64_t N;                         // root rows
  int32_t n_grp;
  GroupDesc grp[kMaxGroups];
  int32_t grp_zoff[kMaxGroups];      // z index of the group's first mean
  int32_t grp_catoff[kMaxGroups];    // row-category index of the group's first category
  int32_t n_x;                       // root continuous columns: z[1 + i]
  Col x[kMaxZ];
  int32_t n_rcat;                    // root categorical columns, after the groups' ones
  const int32_t* rcat[kMaxCat];
  int32_t rcat_dom[kMaxCat];
  int32_t n_rowcat;                  // length of the row's category vector
  int32_t m;                         // length of z
  double* gram_part;                 // [grid][MP * MP]
  long long* cnt_part;               // [grid]
  int32_t n_rv;
  RevView rv[kMaxGroups];
  int32_t n_direct;
  DirectAgg dir[kDirInline];         // the first kDirInline per-row tables (constant bank)
  const DirectAgg* direct;           // device array of all n_direct (read for d >= kDirInline)
  int32_t n_om;
  OmegaAcc om[kMaxGroups * 4];
  int32_t n_cv;
  CatView cv[kMaxCatViews];
  uint32_t* status;
  // per-CTA shared-memory cache of the hot cells of pair-count tables (Zipf-hot
  // category values), 32-bit counters flushed once per CTA
  int32_t cache_cells;               // 0: no cache
  int32_t hot_h;                     // hot values per category (pair tables use hot_h^2 cells)
  const int8_t* hot_lut;             // concatenated per-category value -> hot index, -1 cold
  int32_t hot_lut_off[kMaxCat];      // per row category: offset into hot_lut, -1 none
  long long* const* cache_dst;       // [cache_cells]: global cell each cache cell flushes to
  // resident key: when the root is sorted on the foreign key of probe group
  // res_grp (long runs of one key, the trie order of the scan in Sec. 3.5),
  // every CTA scans one contiguous range of tiles and keeps the resident-form
  // tables of the current key in res_cells shared 32-bit counters; 0: off
  int32_t res_grp;
  int32_t res_cells;
  int32_t unit_w;                    // 1: every w is 0 or 1 (unique child keys)
  int32_t fold;                      // rows per FP32 chain of the plain Gram before it is
                                     // folded into the two-float accumulator (0: once per tile)
  // key-level plans (lmf_root_lean.cuh): the row-level Gram covers only
  // z[gram_off, gram_off + gram_n) (the root's own features); every block
  // with a view mean is taken at the key level from the reverse views
  int32_t lean;
  int32_t gram_off, gram_n;
  int32_t res_rv;                    // reverse view of the resident key (kRvResident), -1: none
  int16_t fix_of_z[kMaxZ];           // key-level plans: index of z's fixed-point image in its group's
                                     // fix records, -1: none (the row pass converts the value itself)
};

// answering a grouped aggregate from a reverse view: loop over the group's keys
struct RvTask {
  int32_t rv;                        // index into RootParams::rv
  int32_t n_gb;
  int32_t cat_word[3];               // category words in the group record
  int32_t dom[3];
  int32_t mode;                      // 0 count, 1 reverse-view slot, 2 hist * mean
  int32_t slot;                      // mode 1
  int32_t mu_word;                   // mode 2
  float scale;                       // modes 1, 2
  long long* out;                    // [cells]
  int32_t fix_idx;                   // mode 2: the mean's fixed-point image in the group's fix records
                                     // (hist * image, exact integers), -1: rounded in FP64 per key
  int32_t soff;                      // first cell of its output in the block's shared table (grouped
                                     // launch), -1: accumulated straight into `out`
  int64_t cells;
};

// one block of the grouped launch of the reverse-view tasks: tasks [t0, t1)
// of view rv (sharing one shared-memory table of `cells` int64) over the
// keys [k0, k1)
struct RvItem {
  int32_t rv, t0, t1, cells;
  int64_t k0, k1;
};

// the keys of a probe group listed by the value of one of their categories
// (rebuilt every run from the group's records): cnt[v] keys carry value v,
// perm[start[v] ..] are those keys (in no particular order), cnt[dom] the
// number of keys with a category inside [0, dom)
struct CatIndex {
  int32_t grp, a_word, dom, pad;
  uint32_t* cnt;                     // [dom + 1], zeroed every run
  uint32_t* start;                   // [dom + 1]
  int32_t* perm;                     // [K of grp]
};

// one block of a COUNT table read off a category view: the keys at positions
// [p0, p1) of the task's category index (so runs of keys with one value a of
// the table's row category), view cells b0 .. b0 + blockDim - 1 of each
struct CvPairItem {
  int32_t task, b0, pad0, pad1;
  int64_t p0, p1;
};

// one block of the SUM(m) grouped by b tables of a category view: the view's
// mean tasks [t0, t1) (at most kCvMeanTasks) over its keys [k0, k1), view
// cells b0 .. b0 + blockDim - 1
constexpr int kCvMeanTasks = 16;
struct CvMeanItem {
  int32_t view, t0, t1, b0;
  int64_t k0, k1;
};

// within-key scatter of a fanning-out root child e:  G[e's block] += sum_k omega[k] Sc_e[k]
struct CorrTask {
  const unsigned long long* omega;
  const double* sc;
  int32_t K, d, zoff;
};

// final placement of one aggregate's result
struct OutMap {
  int32_t kind;                      // 0 COUNT, 1 Gram entry, 2 grouped count, 3 grouped sum,
                                     // 4 filtered count, 5 filtered sum
  int32_t i, j;                      // Gram entry (kind 1)
  int64_t n;                         // cells
  int64_t dst;                       // offset in the int64 or float64 result array
  const long long* src;              // kinds 2, 3: fixed-point cells
  double inv_scale;                  // kind 3
};

#ifndef __CUDACC_RTC__
// ---------------------------------------------------------------------------
// kernel launchers (lmf_kernels.cu)
cudaError_t launch_view_unique(const ViewArgs& a, cudaStream_t s);
cudaError_t launch_view_general(const ViewArgs& a, cudaStream_t s);
cudaError_t launch_view_finalize(const ViewFinalizeArgs& a, cudaStream_t s);
cudaError_t launch_root_plain(const RootParams& p, int mp, int grid, int64_t n_tiles,
                              size_t smem, cudaStream_t s);
size_t root_plain_smem(int mp, int n_rowcat, int cache_cells = 0, int res_cells = 0, bool unit_w = false);
cudaError_t root_plain_prepare(int mp, size_t smem);
int root_plain_tile_rows();
cudaError_t launch_combine(const double* part, int grid, int mp, int m, const long long* cnt_part,
                           double* G, long long* count, cudaStream_t s, int off = 0, int n = -1);
cudaError_t launch_cross_gram(const CrossGram* cg, int n_cg, const CrossPair* pairs, int n_parts,
                              const RootParams& p, double* part, double* G, cudaStream_t s);
cudaError_t launch_fix_means(const FixMeans& f, cudaStream_t s);
// grouped launches of the key-level tasks (shared-memory tables per block)
cudaError_t launch_rv_items(const RvTask* tasks, const RvItem* items, int n_items, int max_cells,
                            const RootParams& p, cudaStream_t s);
// one aggregate's results copied from a per-root plan into the batch's arrays
struct ResultCopy {
  const long long* src;              // int64 or float64 words (copied as bits)
  long long* dst;
  int64_t n;
};
cudaError_t launch_copy_results(const ResultCopy* items, int n_items, cudaStream_t s);
cudaError_t launch_cat_index(const CatIndex* idx, int n_idx, int64_t max_K, const RootParams& p, cudaStream_t s);
cudaError_t launch_cv_pairs(const CatViewTask* tasks, const CatIndex* idx, const CvPairItem* items, int n_items,
                            const RootParams& p, cudaStream_t s);
cudaError_t launch_cv_means(const CatViewTask* tasks, const CvMeanItem* items, int n_items, const RootParams& p,
                            cudaStream_t s);
cudaError_t launch_corr(const void* tasks_dev, int n, double* G, int m, cudaStream_t s);
// tasks sorted by their view; view v owns tasks [begin[v], begin[v + 1])
struct TaskRanges {
  int32_t n_views;
  int32_t begin[kMaxCatViews + 1];
};
cudaError_t launch_rv_tasks(const RvTask* tasks, const TaskRanges& rg, const RootParams& p,
                            int max_K, cudaStream_t s);
cudaError_t launch_cv_tasks(const CatViewTask* tasks, const TaskRanges& rg, const RootParams& p, int64_t max_cells,
                            cudaStream_t s);
cudaError_t launch_group_gram(const GroupGram* gg, int n_gg, int n_parts, const RootParams& p, double* part,
                              double* G, cudaStream_t s);
// a range of one map's cells placed by one block
struct OutItem {
  int32_t map, pad;
  int64_t c0, c1;
};
cudaError_t launch_out_map(const OutMap* maps, const OutItem* items, int n_items, const double* G, int m,
                           const long long* count, long long* res_i64, double* res_f64, cudaStream_t s);
cudaError_t launch_colmaxabs(const Col* cols, int n, int64_t nrows, double* out, cudaStream_t s);
cudaError_t launch_key_stats(const int32_t* key, int64_t n, unsigned int* hist, int K,
                             int* minmax, cudaStream_t s);
// *out += number of adjacent unequal pairs of key[0, n) (*out zeroed by the caller)
cudaError_t launch_key_changes(const int32_t* key, int64_t n, unsigned long long* out, cudaStream_t s);
#endif  // __CUDACC_RTC__

}  // namespace lmf
