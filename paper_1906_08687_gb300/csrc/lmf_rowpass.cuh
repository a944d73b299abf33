// lmf_rowpass.cuh -- the per-row part of the root scan shared by the plain and
// the tensor-core kernels: follow the root row's foreign keys into the merged
// view records (the view lookups of the multi-output plan, Sec. 3.5), build
// z = [1, root features, view means] and the join multiplicity w, and apply the
// row's grouped updates (reverse views towards the dimensions, Sec. 3.2, and
// per-row grouped tables).
#pragma once

#include "lmf_internal.h"

namespace lmf {

__device__ __forceinline__ float rp_load_f(const Col& c, int64_t i) {
  return c.dtype == 2 ? static_cast<float>(static_cast<const double*>(c.p)[i])
                      : static_cast<const float*>(c.p)[i];
}
// Reductions whose old value nobody reads: `red` carries no return value, so
// the issuing warp never waits for the memory system to answer.
__device__ __forceinline__ void rp_red_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void rp_add_ll(long long* p, long long v) {
  rp_red_u64(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}
__device__ __forceinline__ void rp_red_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void rp_red_shared_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))), "r"(v)
               : "memory");
}
// exact fixed-point image of w * x (x * scale is a power-of-two scaling)
__device__ __forceinline__ long long rp_fixp(long long w, float x, float scale) {
  return w * __float2ll_rn(x * scale);
}

__device__ __forceinline__ void rp_put_word(float* zrow, int32_t* crow, const RootParams& p, int g, int w,
                                            uint32_t v, long long& cnt) {
  const GroupDesc& G = p.grp[g];
  if (w < G.n_cnt) {
    cnt *= static_cast<long long>(v);
  } else if (w < G.n_cnt + G.n_mu) {
    zrow[p.grp_zoff[g] + (w - G.n_cnt)] = __uint_as_float(v);
  } else if (w < G.n_cnt + G.n_mu + G.n_cat) {
    crow[p.grp_catoff[g] + (w - G.n_cnt - G.n_mu)] = static_cast<int32_t>(v);
  }
}

// Fills zrow[0, MP) (z, zero padded; all zero when the row does not join) and
// crow[0, n_rowcat); returns w (0 when the row is outside the relation or one of
// its foreign keys dangles).
template <int MP>
__device__ __forceinline__ long long root_row_z(const RootParams& p, int64_t row, float* zrow, int32_t* crow) {
#pragma unroll
  for (int i = 0; i < MP; ++i) zrow[i] = 0.f;
  if (row >= p.N) return 0;
  long long w = 1;
  zrow[0] = 1.f;
  for (int i = 0; i < p.n_x; ++i) zrow[1 + i] = rp_load_f(p.x[i], row);
  for (int g = 0; g < p.n_grp; ++g) {
    const GroupDesc& G = p.grp[g];
    const int32_t fk = G.fk[row];
    if (fk < 0 || fk >= G.K) {
      w = 0;
      continue;
    }
    const uint4* rec = reinterpret_cast<const uint4*>(G.rec + (int64_t)fk * G.stride);
    const int nw = G.n_cnt + G.n_mu + G.n_cat;
    for (int q = 0; q < (nw + 3) / 4; ++q) {
      const uint4 v = __ldg(rec + q);
      rp_put_word(zrow, crow, p, g, 4 * q + 0, v.x, w);
      rp_put_word(zrow, crow, p, g, 4 * q + 1, v.y, w);
      rp_put_word(zrow, crow, p, g, 4 * q + 2, v.z, w);
      rp_put_word(zrow, crow, p, g, 4 * q + 3, v.w, w);
    }
  }
  for (int i = 0; i < p.n_rcat; ++i) {
    int32_t v = p.rcat[i][row];
    if (v < 0 || v >= p.rcat_dom[i]) {
      atomicOr(p.status, kStatusCatRange);
      v = 0;
    }
    crow[p.n_rowcat - p.n_rcat + i] = v;
  }
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < MP; ++i) zrow[i] = 0.f;
  }
  return w;
}

// Runs of equal update targets among the 32 consecutive rows of a warp.  On a
// fact relation sorted by its join attributes (the scan order of Sec. 3.5) the
// rows of one key are contiguous, so a run's updates are summed with shuffles
// and only its first lane issues the atomics.  Integer sums are exact in any
// order, so this changes the number of atomics, never a result.
constexpr unsigned kFullWarp = 0xffffffffu;
constexpr int kRunMaxHeads = 24;  // fewer runs than this in a warp: sum them first

struct WarpRuns {
  bool head;       // first lane of its run
  bool sum;        // warp-uniform: the runs are summed before the atomics
  int end;         // one past the last lane of this lane's run
  unsigned heads;  // lanes that start a run
};

__device__ __forceinline__ WarpRuns warp_runs(long long key) {
  const int lane = threadIdx.x & 31;
  const long long prev = __shfl_up_sync(kFullWarp, key, 1);
  WarpRuns r;
  r.head = lane == 0 || key != prev;
  const unsigned hm = __ballot_sync(kFullWarp, r.head);
  r.heads = hm;
  r.sum = __popc(hm) <= kRunMaxHeads;
  const unsigned above = hm & ~((2u << lane) - 1u);
  r.end = above ? __ffs(above) - 1 : 32;
  return r;
}

// total of v over lanes [lane, end) of the run (complete in the run's head)
__device__ __forceinline__ long long warp_run_sum(const WarpRuns& r, long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long o = __shfl_down_sync(kFullWarp, v, d);
    if (lane + d < r.end) v += o;
  }
  return v;
}

__device__ __forceinline__ void rp_direct_add(const RootParams& p, const DirectAgg& A, int64_t cell,
                                              const int32_t* crow, long long v, uint32_t* cache) {
  if (cache && A.cache_off >= 0) {  // a pair-count table: 32-bit counter cells
    const int ha = __ldg(p.hot_lut + p.hot_lut_off[A.cat[0]] + crow[A.cat[0]]);
    const int hb = __ldg(p.hot_lut + p.hot_lut_off[A.cat[1]] + crow[A.cat[1]]);
    if (ha >= 0 && hb >= 0) {
      rp_red_shared_u32(cache + A.cache_off + ha * p.hot_h + hb, static_cast<uint32_t>(v));
      return;
    }
  }
  rp_add_ll(A.out + cell, v);
}

// ---- resident key ----------------------------------------------------------
// A root sorted on its join attributes (Sec. 3.5: the scan sees the relation as
// a trie, first attribute outermost) holds one value of its first attribute
// over long runs.  A COUNT table with one category from that attribute's probe
// group then gets, for the whole run, one fixed value at that position: the CTA
// counts the run's rows in shared memory over the other positions' cells (the
// table's row for the current key) and adds them to the table when the key
// changes.  Counters are 32-bit: a CTA holds a key for fewer than 2^32 rows.

// a row's counter within a resident table: the cell of the other positions
// (last fastest), times 32 plus the lane for lane-private counters
__device__ __forceinline__ int res_index(const DirectAgg& A, const int32_t* crow) {
  int idx = 0;
  for (int q = 0; q < A.n_gb; ++q)
    if (q != A.res_q) idx = idx * A.dom[q] + crow[A.cat[q]];
  return A.res_lanes ? idx * 32 + static_cast<int>(threadIdx.x & 31) : idx;
}

// adds the counters of resident key k to their tables and clears them; every
// thread of the CTA calls this
__device__ __forceinline__ void root_res_flush(const RootParams& p, uint32_t* hist, long long k) {
  if (k < 0) return;  // no row counted under "no key"
  for (int v = 0; v < p.n_cv; ++v) {
    const CatView& C = p.cv[v];
    if (C.res_off < 0) continue;
    for (int i = threadIdx.x; i < C.dom; i += blockDim.x) {
      const uint32_t n = hist[C.res_off + i];
      if (n == 0u) continue;
      hist[C.res_off + i] = 0u;
      rp_red_u32(C.V + k * C.dom + i, n);
    }
  }
  const GroupDesc& G = p.grp[p.res_grp];
  for (int d = 0; d < p.n_direct; ++d) {
    const DirectAgg& A = d < kDirInline ? p.dir[d] : p.direct[d];
    if (A.res_off < 0) continue;
    const int32_t a = static_cast<int32_t>(G.rec[k * G.stride + A.res_word]);
    for (int i = threadIdx.x; i < A.res_n; i += blockDim.x) {
      uint32_t v = 0u;
      if (A.res_lanes) {
        uint32_t* h = hist + A.res_off + i * 32;
        for (int l = 0; l < 32; ++l) {
          v += h[l];
          h[l] = 0u;
        }
      } else {
        v = hist[A.res_off + i];
        hist[A.res_off + i] = 0u;
      }
      if (v == 0u) continue;
      int rem = i;
      int64_t cell = 0, mult = 1;
      for (int q = A.n_gb - 1; q >= 0; --q) {
        int val = a;
        if (q != A.res_q) {
          val = rem % A.dom[q];
          rem /= A.dom[q];
        }
        cell += static_cast<int64_t>(val) * mult;
        mult *= A.dom[q];
      }
      rp_red_u64(reinterpret_cast<unsigned long long*>(A.out + cell), v);
    }
  }
}

// at the start of a tile: make the key of the tile's first row resident,
// flushing the previous one; every thread of the CTA calls this and holds the
// same key
__device__ __forceinline__ void root_res_advance(const RootParams& p, int64_t row0, uint32_t* hist,
                                                 long long& key) {
  long long nk = -1;
  if (row0 < p.N) {
    const GroupDesc& G = p.grp[p.res_grp];
    const int32_t f = G.fk[row0];
    nk = (f >= 0 && f < G.K) ? f : -1;
  }
  if (nk == key) return;
  __syncthreads();  // the counts of earlier tiles are in
  root_res_flush(p, hist, key);
  __syncthreads();  // cleared before the next tile counts
  key = nk;
}

// one per-row table for the warp's rows (every lane calls this; fres is the
// row's resident-group key, -2 when no key is resident or the row is dead)
__device__ __forceinline__ void root_direct_one(const RootParams& p, const DirectAgg& A, int64_t row,
                                                const float* zrow, const int32_t* crow, long long w,
                                                uint32_t* cache, uint32_t* res_hist, long long res_key,
                                                long long fres) {
  const bool live = w != 0;
  if (A.res_off >= 0 && res_key >= 0) {  // resident form (warp-uniform branch)
    if (!live) return;
    if (fres == res_key) {
      rp_red_shared_u32(res_hist + A.res_off + res_index(A, crow), static_cast<uint32_t>(w));
    } else {
      int64_t cell = 0;
      for (int k = 0; k < A.n_gb; ++k) cell = cell * A.dom[k] + crow[A.cat[k]];
      rp_direct_add(p, A, cell, crow, w, cache);
    }
    return;
  }
  int64_t cell = -1;
  if (live) {
    cell = 0;
    for (int k = 0; k < A.n_gb; ++k) cell = cell * A.dom[k] + crow[A.cat[k]];
  }
  const long long v = live ? (A.z < 0 ? w : rp_fixp(w, zrow[A.z], A.scale)) : 0ll;
  if (!A.runs) {
    if (live) rp_direct_add(p, A, cell, crow, v, cache);
    return;
  }
  const WarpRuns q = warp_runs(cell);  // warp-uniform: A.runs is
  if (!q.sum) {
    if (live) rp_direct_add(p, A, cell, crow, v, cache);
    return;
  }
  const long long t = warp_run_sum(q, v);
  if (q.head && live) rp_direct_add(p, A, cell, crow, t, cache);
}

// Reverse view R for the warp's 32 rows, slot-parallel: lane s sums slot s
// over the rows of each run of equal keys and issues one reduction per run, so
// one instruction updates a key's consecutive slots (a few L2 sectors instead
// of one sector per row and slot).  zw: the warp's z rows, ldz floats apart
// (zero for dead rows); fk: this lane's key, -1 when dead.
// the key's join count of every run, issued by the run's first lane
__device__ __forceinline__ void rv_count_runs(const WarpRuns& q, bool unit_w, long long fk, long long w,
                                              unsigned long long* hist) {
  const int lane = threadIdx.x & 31;
  if (unit_w) {
    const unsigned live = __ballot_sync(kFullWarp, w != 0);
    if (q.head && fk >= 0) {
      const unsigned run = (q.end == 32 ? 0xffffffffu : ((1u << q.end) - 1u)) & ~((1u << lane) - 1u);
      rp_red_u64(hist + fk, static_cast<unsigned long long>(__popc(live & run)));
    }
  } else {
    const long long h = warp_run_sum(q, w);
    if (q.head && fk >= 0 && h != 0) rp_red_u64(hist + fk, static_cast<unsigned long long>(h));
  }
}

// slot s of a reverse view with n_slot slots per key (this lane's slot when
// `slot`; zi its z index, sc its fixed-point scale): sum over each run's rows,
// one reduction per run
__device__ __forceinline__ void rv_slot_runs(const WarpRuns& q, bool unit_w, long long fk, long long w,
                                             const float* zw, int ldz, bool slot, int zi, float sc, long long* R,
                                             int n_slot, int s) {
  long long acc = 0;
  if (unit_w && q.heads == 1u) {  // one run over the whole warp (warp-uniform): one reduction
#pragma unroll 8
    for (int j = 0; j < 32; ++j) acc += __float2ll_rn(zw[j * ldz + zi] * sc);
    const long long k0 = __shfl_sync(kFullWarp, fk, 0);
    if (slot && k0 >= 0 && acc != 0) rp_add_ll(R + k0 * n_slot + s, acc);
    return;
  }
#pragma unroll 4
  for (int j = 0; j < 32; ++j) {
    if (unit_w) {  // w is 0 or 1 and z is zero for dead rows
      acc += __float2ll_rn(zw[j * ldz + zi] * sc);
    } else {
      acc += rp_fixp(__shfl_sync(kFullWarp, w, j), zw[j * ldz + zi], sc);
    }
    if (j == 31 || ((q.heads >> (j + 1)) & 1u)) {  // row j ends a run (warp-uniform)
      const long long kj = __shfl_sync(kFullWarp, fk, j);
      if (slot && kj >= 0 && acc != 0) rp_add_ll(R + kj * n_slot + s, acc);
      acc = 0;
    }
  }
}

__device__ __forceinline__ void root_rv_slots(const RootParams& p, const RevView& R, long long fk, long long w,
                                              const float* zw, int ldz) {
  const int lane = threadIdx.x & 31;
  const WarpRuns q = warp_runs(fk);
  rv_count_runs(q, p.unit_w != 0, fk, w, R.hist);
  for (int s0 = 0; s0 < R.n_slot; s0 += 32) {
    const int s = s0 + lane;
    const bool slot = s < R.n_slot;
    rv_slot_runs(q, p.unit_w != 0, fk, w, zw, ldz, slot, slot ? R.slot_z[s] : 0, slot ? R.slot_scale[s] : 0.f, R.R,
                 R.n_slot, s);
  }
}

// category view C for the warp's rows (every lane calls this): fk is the row's
// key of C's group (-1 when dead), b its category value
__device__ __forceinline__ void root_cv_one(const CatView& C, long long fk, int b, long long w, uint32_t* res_hist,
                                            long long res_key) {
  const bool live = w != 0;
  if (C.res_off >= 0 && res_key >= 0) {  // resident form (warp-uniform branch)
    if (!live) return;
    if (fk == res_key) rp_red_shared_u32(res_hist + C.res_off + b, static_cast<uint32_t>(w));
    else rp_red_u32(C.V + fk * C.dom + b, static_cast<uint32_t>(w));
    return;
  }
  const long long cell = live ? fk * C.dom + b : -1ll;
  if (C.runs) {  // warp-uniform
    const WarpRuns q = warp_runs(cell);
    if (q.sum) {
      const long long t = warp_run_sum(q, w);
      if (q.head && live) rp_red_u32(C.V + cell, static_cast<uint32_t>(t));
      return;
    }
  }
  if (live) rp_red_u32(C.V + cell, static_cast<uint32_t>(w));
}

// Grouped updates of the warp's 32 rows; every lane of the warp calls this,
// w == 0 marks a row that does not join (or lies past the relation's end).
// cache (may be null) holds the CTA's counters for the hot cells of
// pair-count tables, res_hist those of the resident key res_key (-1: none).
__device__ __forceinline__ void root_row_grouped(const RootParams& p, int64_t row, const float* zrow, int ldz,
                                                 const int32_t* crow, long long w, uint32_t* cache,
                                                 uint32_t* res_hist, long long res_key) {
  const bool live = w != 0;
  const long long fres = (live && res_key >= 0) ? static_cast<long long>(p.grp[p.res_grp].fk[row]) : -2ll;
  for (int r = 0; r < p.n_rv; ++r) {
    const RevView& R = p.rv[r];
    const long long fk = live ? static_cast<long long>(p.grp[R.grp].fk[row]) : -1ll;
    root_rv_slots(p, R, fk, w, zrow - (threadIdx.x & 31) * ldz, ldz);
  }
  for (int v = 0; v < p.n_cv; ++v) {
    const CatView& C = p.cv[v];
    const long long fk = live ? static_cast<long long>(p.grp[C.grp].fk[row]) : -1ll;
    root_cv_one(C, fk, live ? crow[C.bcat] : 0, w, res_hist, res_key);
  }
  const int n_inline = p.n_direct < kDirInline ? p.n_direct : kDirInline;
  for (int d = 0; d < n_inline; ++d) root_direct_one(p, p.dir[d], row, zrow, crow, w, cache, res_hist, res_key, fres);
  for (int d = kDirInline; d < p.n_direct; ++d)
    root_direct_one(p, p.direct[d], row, zrow, crow, w, cache, res_hist, res_key, fres);
  if (!live) return;
  for (int o = 0; o < p.n_om; ++o) {
    const OmegaAcc& O = p.om[o];
    const GroupDesc& G = p.grp[O.grp];
    const int32_t fk = G.fk[row];
    const long long ce = static_cast<long long>(G.rec[(int64_t)fk * G.stride + O.cnt_word]);
    rp_red_u64(O.omega + fk, static_cast<unsigned long long>(w / ce));
  }
}

// the CTA's cache of 32-bit counters (hot cells, then the resident-key
// counters): zero at start, flush to the global int64 cells at the end
__device__ __forceinline__ void root_cache_zero(const RootParams& p, uint32_t* cache) {
  const int n = p.cache_cells + p.res_cells;
  for (int i = threadIdx.x; i < n; i += blockDim.x) cache[i] = 0u;
}
__device__ __forceinline__ void root_cache_flush(const RootParams& p, const uint32_t* cache) {
  for (int i = threadIdx.x; i < p.cache_cells; i += blockDim.x) {
    const unsigned long long v = cache[i];
    if (v) rp_red_u64(reinterpret_cast<unsigned long long*>(p.cache_dst[i]), v);
  }
}

// every lane of the warp calls this (root_row_grouped is warp-cooperative)
template <int MP>
__device__ __forceinline__ long long root_row_pass(const RootParams& p, int64_t row, float* zrow, int ldz,
                                                   int32_t* crow, uint32_t* cache, uint32_t* res_hist,
                                                   long long res_key) {
  const long long w = root_row_z<MP>(p, row, zrow, crow);
  __syncwarp();  // the warp's z rows are in shared memory for the slot-parallel sums
  root_row_grouped(p, row, zrow, ldz, crow, w, cache, res_hist, res_key);
  return w;
}

// the row pass that reads the plan's descriptors at run time
struct GenericRowPass {
  static __device__ __forceinline__ int fold(const RootParams& p) { return p.fold; }
  template <int MP>
  static __device__ __forceinline__ long long run(const RootParams& p, int64_t row, float* zrow, int ldz,
                                                  int32_t* crow, uint32_t* cache, uint32_t* res_hist,
                                                  long long res_key) {
    return root_row_pass<MP>(p, row, zrow, ldz, crow, cache, res_hist, res_key);
  }
};

}  // namespace lmf
