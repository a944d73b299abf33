// lmf_tree_dev.cuh -- device side of the tree pass (threshold-filtered
// aggregates, lmf_tree.cu): the plan's device tables, the exact warp and
// global reductions, the node search and the pass's body, shared by the
// kernel compiled with the library and the one compiled for a plan at plan
// time (NVRTC).
#pragma once

#include "lmf_rowpass.cuh"

namespace lmf {

constexpr int kTreeMaxMom = 8;
constexpr int kTreeResNodes = 256;  // nodes whose resident-key sums fit the shared table
constexpr uint16_t kNoNode = 0xFFFF;

struct TreePred {
  int16_t z;
  int16_t op;     // 0: x <= thr, 1: x > thr
  float thr;
};

struct TreeDt {
  int16_t z;
  int16_t leaf;                // 1: left/right are the candidate range [left, left + right)
  float thr;
  int32_t left, right;
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

// The tree pass's body (see the kernels in lmf_tree.cu): Row provides the
// row pass (z and w of a root row: root_row_z for the interpreted kernel, a
// pass generated for the plan for the compiled one) and the node search.
template <class Row, int MP>
__device__ __forceinline__ void tree_body(const RootParams& p, const TreeDev& d) {
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
    if (row < r_end) w = Row::row(p, row, zrow, crow);
    // the row's cells of resident splits go to the shared sums
    const bool row_res = resident && w != 0 && res_key >= 0 && static_cast<long long>(RG.fk[row]) == res_key;
    long long mv[kTreeMaxMom];
    bool have = false;
    for (int g = 0; g < d.n_groups; ++g) {
      const int n = w != 0 ? Row::node(d, g, zrow) : static_cast<int>(kNoNode);
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

// the interpreted row pass and node search
template <int MP>
struct InterpTreeRow {
  static __device__ __forceinline__ long long row(const RootParams& p, int64_t r, float* zrow, int32_t* crow) {
    return root_row_z<MP>(p, r, zrow, crow);
  }
  static __device__ __forceinline__ int node(const TreeDev& d, int g, const float* zrow) {
    return tree_node_of(d, g, zrow);
  }
};

}  // namespace lmf
